// The bottom of the V-cycle in one thread block.
//
// On the small levels (n <= 64 cells per side) every kernel of the V-cycle is
// latency bound: a launch costs more than its work.  k_tail runs the whole
// V-cycle below a given level (Alg. 1 applied recursively, Sec. 3.2) inside
// one 1024-thread block, with every level's u, F and node tags in shared
// memory and __syncthreads() between the colour phases: for each level
// nu1 smoothing steps (one 4-colour Gauss-Seidel sweep, Sec. 4.1, then eta
// sweeps over the cut-cell vertices, Sec. 5.3), residual and restriction
// R = P^T (Sec. 5.1), recursion, the exact coarsest solve (dense inverse),
// prolongation P, nu2 smoothing steps.  It reads F and writes u of its top
// level in that level's padded global layout, so it slots in where the
// multi-block kernels leave off.  The arithmetic and the colour order are
// those of the multi-block kernels.
#include "tail.cuh"

namespace {

constexpr int kThreads = 1024;

struct Grid {
  int n, S;             // cells per side, bordered side n + 3
};

template <class T>
struct Smem {
  T* U[MG_TAIL_MAX_LEVELS];
  T* F[MG_TAIL_MAX_LEVELS];
  int16_t* G[MG_TAIL_MAX_LEVELS];   // -2 not a DOF, -1 interior, >= 0 boundary row
  const T* rows[MG_TAIL_MAX_LEVELS];  // boundary rows (shared or global memory)
  uint16_t* BL[MG_TAIL_MAX_LEVELS];   // boundary nodes' bordered positions, by colour
  int* off;                           // [level][5]: colour offsets into BL
  T* R;                             // residual of the level being restricted
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

template <class T>
__device__ void carve(const TailArgs<T>& a, unsigned char* base, Smem<T>& s) {
  size_t off = 0;
  for (int k = 0; k < a.nlev; ++k) {
    int S = a.n[k] + 3;
    s.U[k] = reinterpret_cast<T*>(base + off); off = align16(off + (size_t)S * S * sizeof(T));
    s.F[k] = reinterpret_cast<T*>(base + off); off = align16(off + (size_t)S * S * sizeof(T));
    s.G[k] = reinterpret_cast<int16_t*>(base + off); off = align16(off + (size_t)S * S * 2);
  }
  s.R = reinterpret_cast<T*>(base + off);
  off = align16(off + (size_t)(a.n[0] + 3) * (a.n[0] + 3) * sizeof(T));
  for (int k = 0; k < a.nlev; ++k) {
    if (a.rows_in_smem) {
      s.rows[k] = reinterpret_cast<const T*>(base + off);
      off = align16(off + (size_t)a.n_bnd[k] * MG_ROW * sizeof(T));
    } else {
      s.rows[k] = a.rows[k];
    }
  }
  for (int k = 0; k < a.nlev; ++k) {
    s.BL[k] = reinterpret_cast<uint16_t*>(base + off);
    off = align16(off + (size_t)a.n_bnd[k] * sizeof(uint16_t));
  }
}

// one colour phase; boundary_only restricts it to the cut-cell vertices.
// Interior nodes of the colour are found by scanning the colour's lattice,
// boundary nodes come from the level's colour-sorted list.
template <class T>
__device__ __forceinline__ void colour_phase(const TailArgs<T>& a, const Smem<T>& s, int k, int c,
                                             bool boundary_only) {
  const int n = a.n[k], S = n + 3;
  T* U = s.U[k];
  const T* F = s.F[k];
  if (!boundary_only) {
    const int ci = c & 1, cj = c >> 1;
    const int wa = (n + 1 - ci + 1) / 2, wb = (n + 1 - cj + 1) / 2;
    const int16_t* G = s.G[k];
    for (int it = threadIdx.x; it < wa * wb; it += blockDim.x) {
      int b = it / wa, aa = it - b * wa;
      int q = (2 * b + cj + 1) * S + (2 * aa + ci + 1);
      if (G[q] != -1) continue;
      const T* Up = U + q;
      T sum = ((Up[-1] + Up[1]) + (Up[-S] + Up[S])) +
              ((Up[-S - 1] + Up[-S + 1]) + (Up[S - 1] + Up[S + 1]));
      U[q] = (T(3) * F[q] + sum) * T(0.125);
    }
  }
  const int e0 = s.off[k * 5 + c], e1 = s.off[k * 5 + c + 1];
  const uint16_t* BL = s.BL[k];
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    int q = BL[e];
    const T* R = s.rows[k] + (size_t)s.G[k][q] * MG_ROW;
    const T* Up = U + q;
    T acc = R[0] * Up[-S - 1] + R[1] * Up[-S] + R[2] * Up[-S + 1] + R[3] * Up[-1] +
            R[4] * Up[0] + R[5] * Up[1] + R[6] * Up[S - 1] + R[7] * Up[S] + R[8] * Up[S + 1];
    U[q] = Up[0] + (F[q] - acc) * R[9];
  }
  __syncthreads();
}

template <class T>
__device__ void smooth(const TailArgs<T>& a, const Smem<T>& s, int k) {
  for (int c = 0; c < 4; ++c) colour_phase(a, s, k, c, false);
  for (int e = 0; e < a.eta; ++e)
    for (int c = 0; c < 4; ++c) colour_phase(a, s, k, c, true);
}

template <class T>
__device__ void residual_restrict(const TailArgs<T>& a, const Smem<T>& s, int k) {
  const int n = a.n[k], S = n + 3;
  const T* U = s.U[k];
  const T* F = s.F[k];
  const int16_t* G = s.G[k];
  for (int q = threadIdx.x; q < S * S; q += blockDim.x) {
    int tag = G[q];
    T r = T(0);
    if (tag != -2) {
      const T* Up = U + q;
      if (tag == -1) {
        T s8 = ((Up[-1] + Up[1]) + (Up[-S] + Up[S])) +
               ((Up[-S - 1] + Up[-S + 1]) + (Up[S - 1] + Up[S + 1]));
        r = F[q] - (T(8) * Up[0] - s8) * T(1.0 / 3.0);
      } else {
        const T* R = s.rows[k] + (size_t)tag * MG_ROW;
        T acc = R[0] * Up[-S - 1] + R[1] * Up[-S] + R[2] * Up[-S + 1] + R[3] * Up[-1] +
                R[4] * Up[0] + R[5] * Up[1] + R[6] * Up[S - 1] + R[7] * Up[S] + R[8] * Up[S + 1];
        r = F[q] - acc;
      }
    }
    s.R[q] = r;
  }
  __syncthreads();
  const int nc = a.n[k + 1], Sc = nc + 3;
  T* Fc = s.F[k + 1];
  for (int p = threadIdx.x; p < (nc + 1) * (nc + 1); p += blockDim.x) {
    int J = p / (nc + 1), I = p - J * (nc + 1);
    const T* R = s.R + (2 * J + 1) * S + (2 * I + 1);
    T rc = R[0] + T(0.5) * ((R[-1] + R[1]) + (R[-S] + R[S])) +
           T(0.25) * ((R[-S - 1] + R[-S + 1]) + (R[S - 1] + R[S + 1]));
    Fc[(J + 1) * Sc + (I + 1)] = rc;
  }
  __syncthreads();
}

template <class T>
__device__ void prolong(const TailArgs<T>& a, const Smem<T>& s, int k) {
  const int n = a.n[k], S = n + 3, Sc = a.n[k + 1] + 3;
  T* U = s.U[k];
  const T* E = s.U[k + 1];
  const int16_t* G = s.G[k];
  for (int p = threadIdx.x; p < (n + 1) * (n + 1); p += blockDim.x) {
    int j = p / (n + 1), i = p - j * (n + 1);
    int q = (j + 1) * S + (i + 1);
    if (G[q] == -2) continue;
    const T* e = E + ((j >> 1) + 1) * Sc + ((i >> 1) + 1);
    T v;
    if (!(i & 1) && !(j & 1)) v = e[0];
    else if (!(j & 1)) v = T(0.5) * (e[0] + e[1]);
    else if (!(i & 1)) v = T(0.5) * (e[0] + e[Sc]);
    else v = T(0.25) * ((e[0] + e[1]) + (e[Sc] + e[Sc + 1]));
    U[q] += v;
  }
  __syncthreads();
}

// u = A^{-1} F on the coarsest level: one warp per row group, lanes split
// the columns, warp-shuffle sums (fp64 accumulation)
template <class T>
__device__ void coarsest(const TailArgs<T>& a, const Smem<T>& s, int k) {
  const int n = a.n[k], S = n + 3, m = (n + 1) * (n + 1);
  const T* F = s.F[k];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int p = warp; p < m; p += nwarp) {
    double x = 0.0;
    for (int c = lane; c < m; c += 32) {
      int cj = c / (n + 1), ci = c - cj * (n + 1);
      x += a.Ainv[(size_t)c * m + p] * (double)F[(cj + 1) * S + (ci + 1)];
    }
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) {
      int j = p / (n + 1), i = p - j * (n + 1);
      s.U[k][(j + 1) * S + (i + 1)] = (T)x;
    }
  }
  __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(kThreads, 1) k_tail(TailArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<T> s;
  carve(a, smem_raw, s);
  // tags, F of the top level, u of the top level (or 0), zero everywhere else;
  // loads are issued in batches of 4 per thread before any shared store
  for (int k = 0; k < a.nlev; ++k) {
    const int n = a.n[k], S = n + 3;
    const Layout& L = a.L[k];
    constexpr int B = 4;
    for (int q0 = threadIdx.x; q0 < S * S; q0 += B * blockDim.x) {
      uint16_t cd[B];
      T u[B], f[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        int q = q0 + b * blockDim.x;
        int j = q / S - 1, i = q % S - 1;
        bool in = q < S * S && i >= 0 && j >= 0 && i <= n && j <= n;
        size_t g = in ? L.idx(i, j) : 0;
        cd[b] = in ? a.code[k][g] : (uint16_t)0;
        f[b] = (in && k == 0) ? a.F0[g] : T(0);
        u[b] = (in && k == 0 && a.load_u0) ? a.u0[g] : T(0);
      }
#pragma unroll
      for (int b = 0; b < B; ++b) {
        int q = q0 + b * blockDim.x;
        if (q >= S * S) continue;
        int j = q / S - 1, i = q % S - 1;
        int tag = -2;
        if (cd[b] == 1) tag = -1;
        else if (cd[b] >= 2) tag = a.tile_base[k][L.tile_of(i, j)] + cd[b] - 2;
        s.G[k][q] = (int16_t)tag;
        s.U[k][q] = cd[b] ? u[b] : T(0);
        s.F[k][q] = f[b];
      }
    }
    if (a.rows_in_smem) {
      T* dst = const_cast<T*>(s.rows[k]);
      for (int e = threadIdx.x; e < a.n_bnd[k] * MG_ROW; e += blockDim.x) dst[e] = a.rows[k][e];
    }
  }
  // colour-sorted boundary lists: count, offsets, fill
  __shared__ int s_cnt[MG_TAIL_MAX_LEVELS * 4];
  __shared__ int s_off[MG_TAIL_MAX_LEVELS * 5];
  s.off = s_off;
  if (threadIdx.x < MG_TAIL_MAX_LEVELS * 4) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int k = 0; k < a.nlev; ++k) {
    const int n = a.n[k], S = n + 3;
    for (int q = threadIdx.x; q < S * S; q += blockDim.x) {
      if (s.G[k][q] < 0) continue;
      int j = q / S - 1, i = q % S - 1;
      atomicAdd(&s_cnt[k * 4 + (i & 1) + 2 * (j & 1)], 1);
    }
  }
  __syncthreads();
  if (threadIdx.x < a.nlev) {
    int k = threadIdx.x, acc = 0;
    for (int c = 0; c < 4; ++c) {
      s_off[k * 5 + c] = acc;
      acc += s_cnt[k * 4 + c];
      s_cnt[k * 4 + c] = s_off[k * 5 + c];      // fill cursor
    }
    s_off[k * 5 + 4] = acc;
  }
  __syncthreads();
  for (int k = 0; k < a.nlev; ++k) {
    const int n = a.n[k], S = n + 3;
    for (int q = threadIdx.x; q < S * S; q += blockDim.x) {
      if (s.G[k][q] < 0) continue;
      int j = q / S - 1, i = q % S - 1;
      int e = atomicAdd(&s_cnt[k * 4 + (i & 1) + 2 * (j & 1)], 1);
      s.BL[k][e] = (uint16_t)q;
    }
  }
  __syncthreads();
  const int K = a.nlev;
  for (int k = 0; k + 1 < K; ++k) {
    for (int r = 0; r < a.nu1; ++r) smooth(a, s, k);
    residual_restrict(a, s, k);
  }
  coarsest(a, s, K - 1);
  for (int k = K - 2; k >= 0; --k) {
    prolong(a, s, k);
    for (int r = 0; r < a.nu2; ++r) smooth(a, s, k);
  }
  const int n = a.n[0], S = n + 3;
  for (int p = threadIdx.x; p < (n + 1) * (n + 1); p += blockDim.x) {
    int j = p / (n + 1), i = p - j * (n + 1);
    a.u0[a.L[0].idx(i, j)] = s.U[0][(j + 1) * S + (i + 1)];
  }
}

}  // namespace

size_t tail_smem_bytes(const int* n, int nlev, size_t elem) {
  size_t off = 0;
  for (int k = 0; k < nlev; ++k) {
    size_t S = (size_t)n[k] + 3;
    off = align16(off + S * S * elem);
    off = align16(off + S * S * elem);
    off = align16(off + S * S * 2);
  }
  size_t S0 = (size_t)n[0] + 3;
  return align16(off + S0 * S0 * elem);
}

size_t tail_rows_bytes(const int* n_bnd, int nlev, size_t elem) {
  size_t off = 0;
  for (int k = 0; k < nlev; ++k) off = align16(off + (size_t)n_bnd[k] * MG_ROW * elem);
  return off;
}

size_t tail_list_bytes(const int* n_bnd, int nlev) {
  size_t off = 0;
  for (int k = 0; k < nlev; ++k) off = align16(off + (size_t)n_bnd[k] * sizeof(uint16_t));
  return off;
}

template <class T>
cudaError_t configure_tail(size_t smem) {
  return cudaFuncSetAttribute(k_tail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <class T>
void launch_tail(const TailArgs<T>& a, size_t smem, cudaStream_t st) {
  k_tail<T><<<1, kThreads, smem, st>>>(a);
}

template cudaError_t configure_tail<float>(size_t);
template cudaError_t configure_tail<double>(size_t);
template void launch_tail<float>(const TailArgs<float>&, size_t, cudaStream_t);
template void launch_tail<double>(const TailArgs<double>&, size_t, cudaStream_t);
