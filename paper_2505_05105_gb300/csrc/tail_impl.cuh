// Device code of the single-block V-cycle on the smallest levels, shared by
// k_tail (tail.cu) and the batched solver (batch.cu).  See tail.cu.
#pragma once

#include "tail.cuh"
#include "bandreg.cuh"

namespace {


constexpr int kTailThreads = 1024;

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Per-level pointers and sizes, kept in shared memory: indexing the kernel
// parameters or a local array by a runtime level would go through the stack.
template <class T>
struct Smem {
  int n[MG_TAIL_MAX_LEVELS];
  int nb[MG_TAIL_MAX_LEVELS];             // boundary rows per level
  T* U[MG_TAIL_MAX_LEVELS];
  T* F[MG_TAIL_MAX_LEVELS];
  const int16_t* G[MG_TAIL_MAX_LEVELS];   // -2 not a DOF, -1 interior, >= 0 boundary row
  const T* rows[MG_TAIL_MAX_LEVELS];      // boundary rows (shared or global memory)
  const uint16_t* BL[MG_TAIL_MAX_LEVELS]; // boundary nodes' bordered positions, by colour
  const int* off;                         // [level][5]: colour offsets into BL
  const double* Ainv;                     // coarsest inverse (shared or global memory)
  T* R;                                   // residual of the level being restricted
};

// Level data used by the phases of one level, loaded once per smoothing step.
template <class T>
struct Lvl {
  int n, S, nb;
  T* U;
  const T* F;
  const int16_t* G;
  const T* rows;
  const uint16_t* BL;
  int o[5];
};

// a listed node's bordered position (checked builds: its stencil inside the
// (n + 3)^2 array)
__device__ __forceinline__ int tail_pos(int q, int S) {
  (void)S;
  return MG_CHECKED(q >= S + 1 && q < S * S - S - 1) ? q : S + 1;
}

template <class T>
__device__ __forceinline__ Lvl<T> level(const Smem<T>& s, int k) {
  Lvl<T> v;
  v.n = s.n[k];
  v.S = v.n + 3;
  v.nb = s.nb[k];
  v.U = s.U[k];
  v.F = s.F[k];
  v.G = s.G[k];
  v.rows = s.rows[k];
  v.BL = s.BL[k];
#pragma unroll
  for (int c = 0; c < 5; ++c) v.o[c] = s.off[k * 5 + c];
  return v;
}

// one colour phase of the full sweep: interior nodes of the colour by
// scanning the colour's lattice (a warp per lattice row), boundary nodes from
// the level's colour-sorted list.
template <class T>
__device__ __forceinline__ void colour_phase(const Lvl<T>& v, int c, bool boundary_only) {
  const int n = v.n, S = v.S;
  T* U = v.U;
  if (!boundary_only) {
    const int ci = c & 1, cj = c >> 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = cj + 2 * warp; j <= n; j += 2 * nw) {
      for (int i = ci + 2 * lane; i <= n; i += 64) {
        const int q = (j + 1) * S + (i + 1);
        if (v.G[q] != -1) continue;
        const T* Up = U + q;
        T sum = ((Up[-1] + Up[1]) + (Up[-S] + Up[S])) +
                ((Up[-S - 1] + Up[-S + 1]) + (Up[S - 1] + Up[S + 1]));
        U[q] = (T(3) * v.F[q] + sum) * T(0.125);
      }
    }
  }
  const int e0 = c == 0 ? v.o[0] : c == 1 ? v.o[1] : c == 2 ? v.o[2] : v.o[3];
  const int e1 = c == 0 ? v.o[1] : c == 1 ? v.o[2] : c == 2 ? v.o[3] : v.o[4];
  // boundary nodes from the last threads, whose warps have the fewest (on the
  // small levels no) interior rows: both kinds of work run side by side
  for (int e = e0 + (int)(blockDim.x - 1 - threadIdx.x); e < e1; e += blockDim.x) {
    const int q = tail_pos(v.BL[e], v.S);
    const T* R = v.rows + (size_t)checked_row(v.G[q], v.nb) * MG_ROW;
    const T* Up = U + q;
    T acc = R[0] * Up[-S - 1] + R[1] * Up[-S] + R[2] * Up[-S + 1] + R[3] * Up[-1] +
            R[4] * Up[0] + R[5] * Up[1] + R[6] * Up[S - 1] + R[7] * Up[S] + R[8] * Up[S + 1];
    U[q] = Up[0] + (v.F[q] - acc) * R[9];
  }
  __syncthreads();
}

// one smoothing step: the full 4-colour sweep, then the eta sweeps over the
// cut-cell vertices on as many warps as the longest colour list needs, each
// thread's nodes in registers (REG: their rows too, for blocks small enough
// to hold them)
template <class T, bool REG = false>
__device__ void smooth(const TailArgs<T>& a, const Smem<T>& s, int k) {
  const Lvl<T> v = level(s, k);
  for (int c = 0; c < 4; ++c) colour_phase(v, c, false);
  if (a.eta <= 0) return;
  int mc = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) mc = max(mc, v.o[c + 1] - v.o[c]);
  const int nw = min((int)(blockDim.x >> 5), max(1, (mc + 31) / 32));
  if ((int)(threadIdx.x >> 5) < nw) {
    auto extra = [&](int e) {
      const int q = tail_pos(v.BL[e], v.S);
      const T* w = v.rows + (size_t)checked_row(v.G[q], v.nb) * MG_ROW;
      const T* Up = v.U + q;
      const int S = v.S;
      T acc = w[0] * Up[-S - 1] + w[1] * Up[-S] + w[2] * Up[-S + 1] + w[3] * Up[-1] +
              w[4] * Up[0] + w[5] * Up[1] + w[6] * Up[S - 1] + w[7] * Up[S] + w[8] * Up[S + 1];
      v.U[q] = Up[0] + (v.F[q] - acc) * w[9];
    };
    if constexpr (REG) {
      auto fetch = [&](int e, T* w, int& p) {
        const int q = tail_pos(v.BL[e], v.S);
        const T* R = v.rows + (size_t)checked_row(v.G[q], v.nb) * MG_ROW;
#pragma unroll
        for (int kk = 0; kk < MG_ROW; ++kk) w[kk] = R[kk];
        w[MG_ROW] = v.F[q];
        p = q;
      };
      band_phases_reg<T>(v.U, v.S, v.o, a.eta, 32 * nw, fetch, extra);
    } else {
      auto fetch = [&](int e, int& r, T& f, int& p) {
        const int q = tail_pos(v.BL[e], v.S);
        r = checked_row(v.G[q], v.nb);
        f = v.F[q];
        p = q;
      };
      band_phases_idx<T>(v.U, v.S, v.rows, v.o, a.eta, 32 * nw, fetch, extra);
    }
  }
  __syncthreads();
}

// the transposed smoothing step (transposed V-cycle): the eta sweeps over
// the cut-cell vertices first, then the full sweep, all colours in the
// reverse order
template <class T>
__device__ void smooth_transposed(const TailArgs<T>& a, const Smem<T>& s, int k) {
  const Lvl<T> v = level(s, k);
  if (a.eta > 0) {
    int mc = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) mc = max(mc, v.o[c + 1] - v.o[c]);
    const int nw = min((int)(blockDim.x >> 5), max(1, (mc + 31) / 32));
    if ((int)(threadIdx.x >> 5) < nw) {
      auto fetch = [&](int e, int& r, T& f, int& p) {
        const int q = tail_pos(v.BL[e], v.S);
        r = checked_row(v.G[q], v.nb);
        f = v.F[q];
        p = q;
      };
      auto extra = [&](int e) {
        const int q = tail_pos(v.BL[e], v.S);
        const T* w = v.rows + (size_t)checked_row(v.G[q], v.nb) * MG_ROW;
        const T* Up = v.U + q;
        const int S = v.S;
        T acc = w[0] * Up[-S - 1] + w[1] * Up[-S] + w[2] * Up[-S + 1] + w[3] * Up[-1] +
                w[4] * Up[0] + w[5] * Up[1] + w[6] * Up[S - 1] + w[7] * Up[S] + w[8] * Up[S + 1];
        v.U[q] = Up[0] + (v.F[q] - acc) * w[9];
      };
      band_phases_idx<T, decltype(fetch), decltype(extra), true>(v.U, v.S, v.rows, v.o, a.eta,
                                                                 32 * nw, fetch, extra);
    }
    __syncthreads();
  }
  for (int c = 3; c >= 0; --c) colour_phase(v, c, false);
}

template <class T>
__device__ void residual_restrict(const Smem<T>& s, int k) {
  const Lvl<T> v = level(s, k);
  const int S = v.S;
  for (int q = threadIdx.x; q < S * S; q += blockDim.x) {
    const int tag = v.G[q];
    T r = T(0);
    if (tag != -2) {
      const T* Up = v.U + q;
      if (tag == -1) {
        T s8 = ((Up[-1] + Up[1]) + (Up[-S] + Up[S])) +
               ((Up[-S - 1] + Up[-S + 1]) + (Up[S - 1] + Up[S + 1]));
        r = v.F[q] - (T(8) * Up[0] - s8) * T(1.0 / 3.0);
      } else {
        const T* R = v.rows + (size_t)checked_row(tag, v.nb) * MG_ROW;
        T acc = R[0] * Up[-S - 1] + R[1] * Up[-S] + R[2] * Up[-S + 1] + R[3] * Up[-1] +
                R[4] * Up[0] + R[5] * Up[1] + R[6] * Up[S - 1] + R[7] * Up[S] + R[8] * Up[S + 1];
        r = v.F[q] - acc;
      }
    }
    s.R[q] = r;
  }
  __syncthreads();
  const int nc = s.n[k + 1], Sc = nc + 3;
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
__device__ void prolong(const Smem<T>& s, int k) {
  const int n = s.n[k], S = n + 3, Sc = s.n[k + 1] + 3;
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

// u = A^{-1} F on the coarsest level in fp64.  fp64 instructions are costly
// on this part (a warp's fp64 instruction occupies the SM's fp64 pipe for
// many cycles), so the solve issues as few as it can: F is converted once,
// the columns are split into K slices whose partial row sums go to scratch
// space (the residual buffer R, free at this point), and one pass adds the
// K partials of each row.  With too little scratch, one thread per row.
// The inverse is stored by columns.
template <class T>
__device__ void coarsest(const Smem<T>& s, int k, size_t r_bytes) {
  const int n = s.n[k], S = n + 3, W = n + 1, m = W * W;
  const T* F = s.F[k];
  const double* Ainv = s.Ainv;
  T* U = s.U[k];
  double* fd = reinterpret_cast<double*>(s.R);            // F in fp64, then the partials
  const int cap = (int)(r_bytes / sizeof(double));
  const int K = min((int)blockDim.x / m, cap / m - 1);
  if (K < 1) {
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
      double x = 0.0;
      for (int c = 0; c < m; ++c) {
        const int cj = c / W, ci = c - cj * W;
        x = fma(Ainv[(size_t)c * m + p], (double)F[(cj + 1) * S + ci + 1], x);
      }
      const int j = p / W, i = p - j * W;
      U[(j + 1) * S + (i + 1)] = (T)x;
    }
    __syncthreads();
    return;
  }
  double* part = fd + m;
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    const int cj = c / W, ci = c - cj * W;
    fd[c] = (double)F[(cj + 1) * S + ci + 1];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < K * m; t += blockDim.x) {
    const int sl = t / m, p = t - sl * m;
    double x = 0.0;
    for (int c = sl; c < m; c += K) x = fma(Ainv[(size_t)c * m + p], fd[c], x);
    part[sl * m + p] = x;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < m; p += blockDim.x) {
    double x = part[p];
    for (int sl = 1; sl < K; ++sl) x += part[sl * m + p];
    const int j = p / W, i = p - j * W;
    U[(j + 1) * S + (i + 1)] = (T)x;
  }
  __syncthreads();
}

// The whole V-cycle below level a.lay (see the file comment of tail.cu) by
// one block of blockDim.x <= 1024 threads, in the shared memory at smem_raw
// (128-byte aligned, a.lay.total bytes).  Callable repeatedly by the same
// block.  load_u0: start from the top level's u in global memory (else from
// zero; a.load_u0 is not read); load_image = false keeps the static image a
// previous call of the same problem left in shared memory.
template <class T, bool REG = false>
__device__ void tail_vcycle(const TailArgs<T>& a, unsigned char* smem_raw, bool load_u0,
                            bool load_image) {
  // order this block's earlier generic accesses of the shared memory before
  // the bulk copies below; a previous call may still be reading the table
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  __shared__ Smem<T> s;
  __shared__ uint64_t bar;
  __shared__ int bad;
  const TailLayout& lay = a.lay;
  const int K = lay.nlev;
  // the residual buffer: (n_0 + 3)^2 values of the top level
  const size_t s_rbytes = (size_t)(lay.n[0] + 3) * (lay.n[0] + 3) * sizeof(T);
  if (threadIdx.x == 0) {
    for (int k = 0; k < K; ++k) {
      s.n[k] = lay.n[k];
      s.nb[k] = lay.n_bnd[k];
      s.U[k] = reinterpret_cast<T*>(smem_raw + lay.U[k]);
      s.F[k] = reinterpret_cast<T*>(smem_raw + lay.F[k]);
      s.G[k] = reinterpret_cast<const int16_t*>(smem_raw + lay.G[k]);
      s.BL[k] = reinterpret_cast<const uint16_t*>(smem_raw + lay.BL[k]);
      s.rows[k] = lay.rows_in_smem ? reinterpret_cast<const T*>(smem_raw + lay.rows[k])
                                   : a.rows[k];
    }
    s.off = reinterpret_cast<const int*>(smem_raw + lay.off);
    s.Ainv = lay.ainv_in_smem ? reinterpret_cast<const double*>(smem_raw + lay.Ainv) : a.Ainv;
    s.R = reinterpret_cast<T*>(smem_raw + lay.R);
    mbar_init(&bar, 1);
    bad = load_image && !bulk_ok(smem_raw, a.image, lay.image_bytes);
  }
  __syncthreads();
  // the static image: one bulk copy (in pieces of at most 64 KB)
  if (threadIdx.x == 0) {
    if (!load_image) {
      mbar_arrive_expect_tx(&bar, 0);
    } else if (!bad) {
      mbar_arrive_expect_tx(&bar, (uint32_t)lay.image_bytes);
      for (size_t o = 0; o < lay.image_bytes; o += 65536) {
        const size_t nb = lay.image_bytes - o < 65536 ? lay.image_bytes - o : 65536;
        bulk_load(smem_raw + o, a.image + o, (uint32_t)nb, &bar);
      }
    } else {
      atomicOr(a.err, DEV_ERR_ALIGN);
      mbar_arrive_expect_tx(&bar, 0);
    }
  }
  // meanwhile: u and F of every level start at zero, then (once the
  // previous kernel is done) the top level's F and u from global memory, all
  // loads of a thread in flight at once
  {
    T* dyn = reinterpret_cast<T*>(smem_raw + lay.U[0]);
    const size_t nd = (lay.R - lay.U[0]) / sizeof(T);
    for (size_t q = threadIdx.x; q < nd; q += blockDim.x) dyn[q] = T(0);
  }
  __syncthreads();
  griddep_wait();
  {
    const int n = lay.n[0], S = n + 3, W = n + 1;
    constexpr int B = 6;
    for (int p0 = threadIdx.x; p0 < W * W; p0 += B * blockDim.x) {
      T f[B], u[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int p = p0 + b * blockDim.x;
        const int j = p / W, i = p - j * W;
        const bool in = p < W * W;
        const size_t g = in ? a.L0.idx(i, j) : 0;
        f[b] = in ? a.F0[g] : T(0);
        u[b] = (in && load_u0) ? a.u0[g] : T(0);
      }
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int p = p0 + b * blockDim.x;
        if (p >= W * W) continue;
        const int j = p / W, i = p - j * W;
        s.F[0][(j + 1) * S + (i + 1)] = f[b];
        s.U[0][(j + 1) * S + (i + 1)] = u[b];
      }
    }
  }
  const bool ok = mbar_wait(&bar, 0, a.wait_polls);
  if (__syncthreads_or(!ok || bad)) {
    if (threadIdx.x == 0 && !ok) {
      atomicOr(a.err, DEV_ERR_TIMEOUT);
      mbar_wait(&bar, 0);        // bounded: let copies still in flight land
    }
    __syncthreads();
    return;
  }
  if (threadIdx.x == 0) mbar_inval(&bar);
  if (!a.transposed) {
    for (int k = 0; k + 1 < K; ++k) {
      for (int r = 0; r < a.nu1; ++r) smooth<T, REG>(a, s, k);
      residual_restrict(s, k);
    }
    coarsest(s, K - 1, s_rbytes);
    for (int k = K - 2; k >= 0; --k) {
      prolong(s, k);
      for (int r = 0; r < a.nu2; ++r) smooth<T, REG>(a, s, k);
    }
  } else {
    // the transposed cycle: the same steps in the reverse order, each
    // transposed (nu2 transposed steps down, nu1 up)
    for (int k = 0; k + 1 < K; ++k) {
      for (int r = 0; r < a.nu2; ++r) smooth_transposed(a, s, k);
      residual_restrict(s, k);
    }
    coarsest(s, K - 1, s_rbytes);
    for (int k = K - 2; k >= 0; --k) {
      prolong(s, k);
      for (int r = 0; r < a.nu1; ++r) smooth_transposed(a, s, k);
    }
  }
  const int n = lay.n[0], S = n + 3;
  for (int p = threadIdx.x; p < (n + 1) * (n + 1); p += blockDim.x) {
    int j = p / (n + 1), i = p - j * (n + 1);
    a.u0[a.L0.idx(i, j)] = s.U[0][(j + 1) * S + (i + 1)];
  }
}


}  // namespace
