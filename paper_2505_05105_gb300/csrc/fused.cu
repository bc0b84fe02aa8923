// One whole smoothing step per kernel on the intermediate levels.
//
// Between the fine level (bandwidth bound, separate kernels) and the tail
// block (n <= 64) the levels are small enough that launch and phase latency
// dominate.  k_smooth_step does one smoothing step -- a 4-colour Gauss-Seidel
// sweep (Sec. 4.1) followed by eta colour sweeps over the cut-cell vertices
// (Sec. 5.3) -- for one 64 x 32 tile, redundantly on a halo of
// HS = 4 eta + 7 nodes: after 4 + 4 eta colour phases a stale halo value can
// have spread at most 4 + 4 eta nodes inwards, so the owned tile and two more
// rings are exact.  Optionally it
//   * starts from u = 0 (first smoothing step on a coarse level),
//   * adds the prolongated correction P e_2h while loading u (Sec. 5.1), and
//   * computes r = F - A u on the owned nodes plus one ring and restricts it,
//     F_2h = P^T r, for the 32 x 16 coarse block the tile covers.
// This replaces 8 launches per level (3 sweeps, 3 band sweeps, restriction,
// prolongation) by 3.
#include "fused.cuh"

namespace {

constexpr int kThreads = 512;

__host__ __device__ inline int halo_of(int eta) { return 4 * eta + 7; }

// elements of the shared area used for the coarse correction (prolongation)
// and later for the restriction staging (owned tile plus one ring)
__host__ __device__ inline int e_size(int RX, int RY) {
  int a = (RX / 2 + 3) * (RY / 2 + 3), b = (MG_TX + 2) * (MG_TY + 2);
  return a > b ? a : b;
}

// capacity of each colour's boundary list; a region with more boundary nodes
// of one colour (far beyond smooth interfaces) falls back to scanning
constexpr int kListCap = 512;
__host__ __device__ inline int list_cap(int, int) { return kListCap; }

template <class T, bool ZERO_IN, bool PROLONG, bool RESTRICT>
__global__ void __launch_bounds__(kThreads)
k_smooth_step(FusedArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int HS = halo_of(a.eta);
  const int RX = MG_TX + 2 * HS, RY = MG_TY + 2 * HS;
  T* sU = reinterpret_cast<T*>(smem_raw);
  T* sF = sU + RX * RY;
  T* sE = sF + RX * RY;        // coarse correction region, then restriction staging
  const int EX = RX / 2 + 3, EY = RY / 2 + 3;
  uint16_t* sC = reinterpret_cast<uint16_t*>(sE + e_size(RX, RY));
  const int LCAP = list_cap(RX, RY);
  int* sRow = reinterpret_cast<int*>(sC + ((RX * RY + 1) & ~1));   // [4][LCAP]
  uint16_t* sL = reinterpret_cast<uint16_t*>(sRow + 4 * LCAP);      // [4][LCAP]
  __shared__ int cnt[4];
  __shared__ int overflow;
  const Layout& L = a.L;
  const int n = L.n;
  const int t = a.tiles[blockIdx.x];
  const int i0 = (t % L.ntx) * MG_TX, j0 = (t / L.ntx) * MG_TY;
  const int ri0 = i0 - HS, rj0 = j0 - HS;

  if (PROLONG) {
    // coarse nodes (I, J) covering the region: I in [floor(ri0/2), ...]
    const int ci0 = (ri0 >> 1) - 1, cj0 = (rj0 >> 1) - 1;
    const int nc = a.Lc.n;
    for (int p = threadIdx.x; p < EX * EY; p += blockDim.x) {
      int y = p / EX, x = p - y * EX;
      int I = ci0 + x, J = cj0 + y;
      bool in = I >= 0 && J >= 0 && I <= nc && J <= nc;
      sE[p] = in ? a.ec[a.Lc.idx(I, J)] : T(0);
    }
    __syncthreads();
  }
  {
    constexpr int B = 4;
    const int ci0 = (ri0 >> 1) - 1, cj0 = (rj0 >> 1) - 1;
    for (int p0 = threadIdx.x; p0 < RX * RY; p0 += B * blockDim.x) {
      uint16_t cd[B];
      T f[B], u[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        int p = p0 + b * blockDim.x;
        int y = p / RX, x = p - y * RX;
        int gi = ri0 + x, gj = rj0 + y;
        bool in = p < RX * RY && gi >= 0 && gj >= 0 && gi <= n && gj <= n;
        size_t g = in ? L.idx(gi, gj) : 0;
        cd[b] = in ? a.code[g] : (uint16_t)0;
        f[b] = in ? a.F[g] : T(0);
        u[b] = (in && !ZERO_IN) ? a.uin[g] : T(0);
      }
#pragma unroll
      for (int b = 0; b < B; ++b) {
        int p = p0 + b * blockDim.x;
        if (p >= RX * RY) continue;
        T uv = u[b];
        if (PROLONG && cd[b]) {
          int y = p / RX, x = p - y * RX;
          int gi = ri0 + x, gj = rj0 + y;
          const T* e = sE + ((gj >> 1) - cj0) * EX + ((gi >> 1) - ci0);
          T v;
          if (!(gi & 1) && !(gj & 1)) v = e[0];
          else if (!(gj & 1)) v = T(0.5) * (e[0] + e[1]);
          else if (!(gi & 1)) v = T(0.5) * (e[0] + e[EX]);
          else v = T(0.25) * ((e[0] + e[1]) + (e[EX] + e[EX + 1]));
          uv += v;
        }
        sC[p] = cd[b];
        sF[p] = f[b];
        sU[p] = uv;
      }
    }
  }
  __syncthreads();

  // boundary nodes of the region (not on its rim), by colour, with rows
  if (threadIdx.x < 4) cnt[threadIdx.x] = 0;
  if (threadIdx.x == 0) overflow = 0;
  __syncthreads();
  for (int p = threadIdx.x; p < RX * RY; p += blockDim.x) {
    uint16_t cd = sC[p];
    if (cd < 2) continue;
    int y = p / RX, x = p - y * RX;
    if (x == 0 || y == 0 || x == RX - 1 || y == RY - 1) continue;
    int gi = ri0 + x, gj = rj0 + y;
    int c = (gi & 1) + 2 * (gj & 1);
    int pos = atomicAdd(&cnt[c], 1);
    if (pos < LCAP) {
      sL[c * LCAP + pos] = (uint16_t)p;
      sRow[c * LCAP + pos] = a.tile_base[L.tile_of(gi, gj)] + cd - 2;
    } else {
      overflow = 1;
    }
  }
  __syncthreads();
  const bool scan = overflow != 0;     // uniform across the block

  // 4 full colour phases over the region interior
  for (int c = 0; c < 4; ++c) {
    // first x >= 1 with (ri0 + x) of the colour's parity, then every other one
    const int x0 = 2 - (((c & 1) - ri0) & 1), y0 = 2 - (((c >> 1) - rj0) & 1);
    const int wa = (RX - 2 - x0) / 2 + 1, wb = (RY - 2 - y0) / 2 + 1;
    for (int it = threadIdx.x; it < wa * wb; it += blockDim.x) {
      int b = it / wa, aa = it - b * wa;
      int p = (y0 + 2 * b) * RX + x0 + 2 * aa;
      uint16_t cd = sC[p];
      if (cd == 0 || (cd >= 2 && !scan)) continue;   // listed boundary nodes below
      const T* Up = sU + p;
      if (cd == 1) {
        T s8 = ((Up[-1] + Up[1]) + (Up[-RX] + Up[RX])) +
               ((Up[-RX - 1] + Up[-RX + 1]) + (Up[RX - 1] + Up[RX + 1]));
        sU[p] = (T(3) * sF[p] + s8) * T(0.125);
      } else {
        int gi = ri0 + x0 + 2 * aa, gj = rj0 + y0 + 2 * b;
        const T* R = a.rows + (size_t)(a.tile_base[L.tile_of(gi, gj)] + cd - 2) * MG_ROW;
        T acc = R[0] * Up[-RX - 1] + R[1] * Up[-RX] + R[2] * Up[-RX + 1] + R[3] * Up[-1] +
                R[4] * Up[0] + R[5] * Up[1] + R[6] * Up[RX - 1] + R[7] * Up[RX] +
                R[8] * Up[RX + 1];
        sU[p] = Up[0] + (sF[p] - acc) * R[9];
      }
    }
    // same colour's boundary nodes (same-colour nodes never interact)
    const int m = scan ? 0 : cnt[c];
    for (int e = threadIdx.x; e < m; e += blockDim.x) {
      int p = sL[c * LCAP + e];
      const T* R = a.rows + (size_t)sRow[c * LCAP + e] * MG_ROW;
      const T* Up = sU + p;
      T acc = R[0] * Up[-RX - 1] + R[1] * Up[-RX] + R[2] * Up[-RX + 1] + R[3] * Up[-1] +
              R[4] * Up[0] + R[5] * Up[1] + R[6] * Up[RX - 1] + R[7] * Up[RX] +
              R[8] * Up[RX + 1];
      sU[p] = Up[0] + (sF[p] - acc) * R[9];
    }
    __syncthreads();
  }
  // 4 eta phases on the cut-cell vertices only
  for (int ph = 0; ph < 4 * a.eta; ++ph) {
    const int c = ph & 3;
    if (scan) {
      const int x0 = 2 - (((c & 1) - ri0) & 1), y0 = 2 - (((c >> 1) - rj0) & 1);
      const int wa = (RX - 2 - x0) / 2 + 1, wb = (RY - 2 - y0) / 2 + 1;
      for (int it = threadIdx.x; it < wa * wb; it += blockDim.x) {
        int b = it / wa, aa = it - b * wa;
        int x = x0 + 2 * aa, y = y0 + 2 * b;
        int p = y * RX + x;
        uint16_t cd = sC[p];
        if (cd < 2) continue;
        const T* R =
            a.rows + (size_t)(a.tile_base[L.tile_of(ri0 + x, rj0 + y)] + cd - 2) * MG_ROW;
        const T* Up = sU + p;
        T acc = R[0] * Up[-RX - 1] + R[1] * Up[-RX] + R[2] * Up[-RX + 1] + R[3] * Up[-1] +
                R[4] * Up[0] + R[5] * Up[1] + R[6] * Up[RX - 1] + R[7] * Up[RX] +
                R[8] * Up[RX + 1];
        sU[p] = Up[0] + (sF[p] - acc) * R[9];
      }
      __syncthreads();
      continue;
    }
    const int m = cnt[c];
    for (int e = threadIdx.x; e < m; e += blockDim.x) {
      int p = sL[c * LCAP + e];
      const T* R = a.rows + (size_t)sRow[c * LCAP + e] * MG_ROW;
      const T* Up = sU + p;
      T acc = R[0] * Up[-RX - 1] + R[1] * Up[-RX] + R[2] * Up[-RX + 1] + R[3] * Up[-1] +
              R[4] * Up[0] + R[5] * Up[1] + R[6] * Up[RX - 1] + R[7] * Up[RX] +
              R[8] * Up[RX + 1];
      sU[p] = Up[0] + (sF[p] - acc) * R[9];
    }
    __syncthreads();
  }

  for (int it = threadIdx.x; it < MG_TX * MG_TY; it += blockDim.x) {
    int rr = it / MG_TX, ii = it - rr * MG_TX;
    a.uout[L.idx(i0 + ii, j0 + rr)] = sU[(HS + rr) * RX + HS + ii];
  }

  if (RESTRICT) {
    // residual on the owned nodes plus one ring, kept in sF (no longer needed)
    T* sR = sF;
    __syncthreads();
    for (int it = threadIdx.x; it < (MG_TX + 2) * (MG_TY + 2); it += blockDim.x) {
      int rr = it / (MG_TX + 2), ii = it - rr * (MG_TX + 2);
      int x = HS - 1 + ii, y = HS - 1 + rr;
      int p = y * RX + x;
      uint16_t cd = sC[p];
      T r = T(0);
      if (cd) {
        const T* Up = sU + p;
        if (cd == 1) {
          T s8 = ((Up[-1] + Up[1]) + (Up[-RX] + Up[RX])) +
                 ((Up[-RX - 1] + Up[-RX + 1]) + (Up[RX - 1] + Up[RX + 1]));
          r = sF[p] - (T(8) * Up[0] - s8) * T(1.0 / 3.0);
        } else {
          int gi = ri0 + x, gj = rj0 + y;
          const T* R = a.rows + (size_t)(a.tile_base[L.tile_of(gi, gj)] + cd - 2) * MG_ROW;
          T acc = R[0] * Up[-RX - 1] + R[1] * Up[-RX] + R[2] * Up[-RX + 1] + R[3] * Up[-1] +
                  R[4] * Up[0] + R[5] * Up[1] + R[6] * Up[RX - 1] + R[7] * Up[RX] +
                  R[8] * Up[RX + 1];
          r = sF[p] - acc;
        }
      }
      sE[it] = r;     // staging: (MG_TX + 2) x (MG_TY + 2)
    }
    __syncthreads();
    (void)sR;
    const Layout& Lc = a.Lc;
    const int I0 = i0 / 2, J0 = j0 / 2;
    const int SX = MG_TX + 2;
    for (int it = threadIdx.x; it < (MG_TX / 2) * (MG_TY / 2); it += blockDim.x) {
      int cy = it / (MG_TX / 2), cx = it - cy * (MG_TX / 2);
      int I = I0 + cx, J = J0 + cy;
      if (I > Lc.n || J > Lc.n) continue;
      const T* R = sE + (2 * cy + 1) * SX + (2 * cx + 1);
      T rc = R[0] + T(0.5) * ((R[-1] + R[1]) + (R[-SX] + R[SX])) +
             T(0.25) * ((R[-SX - 1] + R[-SX + 1]) + (R[SX - 1] + R[SX + 1]));
      a.Fc[Lc.idx(I, J)] = rc;
    }
  }
}

}  // namespace

size_t fused_smem_bytes(int eta, size_t elem) {
  int HS = halo_of(eta);
  int RX = MG_TX + 2 * HS, RY = MG_TY + 2 * HS;
  return (size_t)RX * RY * 2 * elem + (size_t)e_size(RX, RY) * elem +
         (size_t)((RX * RY + 1) & ~1) * sizeof(uint16_t) +
         4 * (size_t)list_cap(RX, RY) * (sizeof(int) + sizeof(uint16_t));
}

template <class T>
cudaError_t configure_fused(size_t smem) {
  cudaError_t e;
#define MG_CFG(Z, P, R)                                                                       \
  e = cudaFuncSetAttribute(k_smooth_step<T, Z, P, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                           (int)smem);                                                        \
  if (e != cudaSuccess) return e;
  MG_CFG(true, false, false)
  MG_CFG(false, false, false)
  MG_CFG(false, false, true)
  MG_CFG(true, false, true)
  MG_CFG(false, true, false)
  MG_CFG(false, true, true)
#undef MG_CFG
  return cudaSuccess;
}

template <class T>
void launch_smooth_step(const FusedArgs<T>& a, int ntiles, bool zero_in, bool prolong,
                        bool restrict_, size_t smem, cudaStream_t st) {
  if (!ntiles) return;
  if (zero_in && !prolong && !restrict_)
    k_smooth_step<T, true, false, false><<<ntiles, kThreads, smem, st>>>(a);
  else if (zero_in && !prolong && restrict_)
    k_smooth_step<T, true, false, true><<<ntiles, kThreads, smem, st>>>(a);
  else if (!zero_in && !prolong && !restrict_)
    k_smooth_step<T, false, false, false><<<ntiles, kThreads, smem, st>>>(a);
  else if (!zero_in && !prolong && restrict_)
    k_smooth_step<T, false, false, true><<<ntiles, kThreads, smem, st>>>(a);
  else if (!zero_in && prolong && !restrict_)
    k_smooth_step<T, false, true, false><<<ntiles, kThreads, smem, st>>>(a);
  else
    k_smooth_step<T, false, true, true><<<ntiles, kThreads, smem, st>>>(a);
}

template cudaError_t configure_fused<float>(size_t);
template cudaError_t configure_fused<double>(size_t);
template void launch_smooth_step<float>(const FusedArgs<float>&, int, bool, bool, bool, size_t,
                                        cudaStream_t);
template void launch_smooth_step<double>(const FusedArgs<double>&, int, bool, bool, bool, size_t,
                                         cudaStream_t);
