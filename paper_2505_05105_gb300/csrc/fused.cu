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
//   * adds the prolongated correction P e_2h after loading u (Sec. 5.1), and
//   * computes r = F - A u on the owned nodes plus one ring and restricts it,
//     F_2h = P^T r, for the 32 x 16 coarse block the tile covers.
// This replaces 8 launches per level (3 sweeps, 3 band sweeps, restriction,
// prolongation) by 3.
//
// Latency is what counts here, so: u, F and the codes of the region arrive
// by three TMA box copies on one mbarrier; meanwhile the block stages the
// matrix row and F of the region's boundary nodes (cut-cell vertices, from a
// list built at setup, grouped by colour) in shared memory.  The colour
// phases then run from shared memory only, the full phases with several
// lattice nodes in flight per thread, the band phases on as few warps as
// cover the longest colour list.
#include "fused.cuh"
#include "bandreg.cuh"

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kXL = 3;               // 32-node lattice chunks per region row (RX <= 190)

__host__ __device__ inline int halo_of(int eta) { return 4 * eta + 7; }
__host__ __device__ inline int region_x(int eta) { return MG_TX + 2 * halo_of(eta); }
__host__ __device__ inline int region_y(int eta) { return MG_TY + 2 * halo_of(eta); }
__host__ __device__ inline int box_x(int eta) { return tma_box_w(region_x(eta)); }
__host__ __device__ inline size_t a128(size_t b) { return (b + 127) & ~(size_t)127; }

// elements of the shared area used for the coarse correction (prolongation)
// and later for the restriction staging (owned tile plus one ring)
__host__ __device__ inline int e_size(int RX, int RY) {
  int a = (RX / 2 + 3) * (RY / 2 + 3), b = (MG_TX + 2) * (MG_TY + 2);
  return a > b ? a : b;
}

// listed boundary nodes whose row and F are staged in shared memory
template <class T> struct FusedCap;
template <> struct FusedCap<float> { static constexpr int value = 512; };
template <> struct FusedCap<double> { static constexpr int value = 256; };
constexpr int kNS = MG_ROW;          // staged values per node: the row
// tiles around the owned one whose boundary-row bases a region can need:
// x offsets -1..1 (HS < MG_TX), y offsets -2..2 (HS < 2 MG_TY)
constexpr int kTBX = 3, kTBY = 5;

template <class T>
struct Carve {
  T *sUb, *sFb, *sE, *sS;
  uint16_t* sCb;
  int* sP;
};

template <class T>
__host__ __device__ inline size_t carve(unsigned char* base, int eta, Carve<T>* c) {
  const int BX = box_x(eta), BY = region_y(eta);
  const int RC = FusedCap<T>::value;
  size_t off = 0;
  auto take = [&](size_t bytes) { unsigned char* p = base + off; off += a128(bytes); return p; };
  unsigned char* u = take((size_t)BX * BY * sizeof(T));
  unsigned char* f = take((size_t)BX * BY * sizeof(T));
  unsigned char* cd = take((size_t)BX * BY * sizeof(uint16_t));
  unsigned char* e = take((size_t)e_size(region_x(eta), BY) * sizeof(T));
  unsigned char* s = take((size_t)kNS * RC * sizeof(T));
  unsigned char* pp = take((size_t)RC * sizeof(int));
  if (c) {
    c->sUb = reinterpret_cast<T*>(u);
    c->sFb = reinterpret_cast<T*>(f);
    c->sCb = reinterpret_cast<uint16_t*>(cd);
    c->sE = reinterpret_cast<T*>(e);
    c->sS = reinterpret_cast<T*>(s);
    c->sP = reinterpret_cast<int*>(pp);
  }
  return off;
}

template <class T>
__device__ __forceinline__ T row_update(const T* w, const T* Up, T f, int RS) {
  T acc = w[0] * Up[-RS - 1] + w[1] * Up[-RS] + w[2] * Up[-RS + 1] + w[3] * Up[-1] +
          w[4] * Up[0] + w[5] * Up[1] + w[6] * Up[RS - 1] + w[7] * Up[RS] + w[8] * Up[RS + 1];
  return Up[0] + (f - acc) * w[9];
}

template <class T, bool ZERO_IN, bool PROLONG, bool RESTRICT>
__global__ void __launch_bounds__(kThreads)
k_smooth_step(FusedArgs<T> a, const __grid_constant__ FusedMaps maps) {
  griddep_launch_next();
  constexpr int RC = FusedCap<T>::value;
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  unsigned char* smem_raw = smem_align128(smem_dyn);
  const int HS = halo_of(a.eta);
  const int RX = region_x(a.eta), RY = region_y(a.eta);
  const int RS = box_x(a.eta);                 // shared row stride (TMA box width)
  Carve<T> cv;
  carve<T>(smem_raw, a.eta, &cv);
  __shared__ uint64_t bar;
  __shared__ int sTB[kTBX * kTBY];
  __shared__ int gs[6];
  const Layout& L = a.L;
  const int t = a.tiles[blockIdx.x];
  const int tx = t % L.ntx, ty = t / L.ntx;
  const int i0 = tx * MG_TX, j0 = ty * MG_TY;
  const int ri0 = i0 - HS, rj0 = j0 - HS;
  const int ax = tma_floor(ri0 + MG_G), ay = rj0 + MG_G;   // box origin, padded coordinates
  const int ox = ri0 + MG_G - ax;                          // region column 0 inside the box
  T* sU = cv.sUb + ox;
  T* sF = cv.sFb + ox;
  const uint16_t* sC = cv.sCb + ox;
  T* sE = cv.sE;
  T* sS = cv.sS;
  int* sP = cv.sP;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto row_base = [&](int gi, int gj) {
    return sTB[((gj / MG_TY) - ty + 2) * kTBX + (gi / MG_TX) - tx + 1];
  };

  __shared__ int bad;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    bad = !(tma_box_ok(cv.sFb, ax) && tma_box_ok(cv.sCb, ax) && tma_box_ok(cv.sUb, ax));
  }
  __syncthreads();
  // static data first (codes, row bases, lists, rows): it may overlap the
  // end of the previous kernel
  if (threadIdx.x == 0) {
    if (!bad) {
      const uint32_t bytes =
          (uint32_t)((size_t)RS * RY * ((ZERO_IN ? 1 : 2) * sizeof(T) + sizeof(uint16_t)));
      mbar_arrive_expect_tx(&bar, bytes);
      tma_load_2d(cv.sCb, &maps.code, ax, ay, &bar);
    } else {
      atomicOr(a.err, DEV_ERR_ALIGN);
      mbar_arrive_expect_tx(&bar, 0);
    }
  }
  if (threadIdx.x < kTBX * kTBY) {
    int ux = tx + threadIdx.x % kTBX - 1, uy = ty + threadIdx.x / kTBX - 2;
    sTB[threadIdx.x] =
        (ux >= 0 && uy >= 0 && ux < L.ntx && uy < L.nty) ? a.tile_base[uy * L.ntx + ux] : 0;
  }
  const int e0 = a.loff[5 * t];
  if (threadIdx.x < 6) gs[threadIdx.x] = a.loff[5 * t + threadIdx.x] - e0;
  const int m = a.loff[5 * t + 4] - e0;        // colour groups only: the rim is never updated
  // rows of the first RC listed nodes
  for (int e = threadIdx.x; e < m && e < RC; e += blockDim.x) {
    const int2 en = a.lent[e0 + e];
    const int x = en.x & 0xffff, y = en.x >> 16;
    const T* R = a.rows + (size_t)en.y * MG_ROW;
    T v[MG_ROW];
#pragma unroll
    for (int k = 0; k < MG_ROW; ++k) v[k] = R[k];
#pragma unroll
    for (int k = 0; k < MG_ROW; ++k) sS[k * RC + e] = v[k];
    sP[e] = y * RS + x;
  }
  // then the data of the previous kernels: F, u, the coarse correction
  griddep_wait();
  if (threadIdx.x == 0 && !bad) {
    tma_load_2d(cv.sFb, &maps.F, ax, ay, &bar);
    if (!ZERO_IN) tma_load_2d(cv.sUb, &maps.u[a.uin_map], ax, ay, &bar);
  }
  const int ci0 = (ri0 >> 1) - 1, cj0 = (rj0 >> 1) - 1;
  const int EX = RX / 2 + 3, EY = RY / 2 + 3;
  if (PROLONG) {
    // coarse nodes (I, J) covering the region, all loads of a thread in flight
    const int nc = a.Lc.n;
    constexpr int B = 8;
    for (int q0 = threadIdx.x; q0 < EX * EY; q0 += B * kThreads) {
      T v[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int q = q0 + b * kThreads;
        const int y = q / EX, x = q - y * EX;
        const int I = ci0 + x, J = cj0 + y;
        const bool in = q < EX * EY && I >= 0 && J >= 0 && I <= nc && J <= nc;
        v[b] = in ? a.ec[a.Lc.idx(I, J)] : T(0);
      }
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int q = q0 + b * kThreads;
        if (q < EX * EY) sE[q] = v[b];
      }
    }
  }
  if (ZERO_IN)
    for (int q = threadIdx.x; q < RS * RY; q += blockDim.x) cv.sUb[q] = T(0);
  const bool ok = mbar_wait(&bar, 0);
  if (__syncthreads_or(!ok || bad)) {
    if (threadIdx.x == 0 && !ok) {
      atomicOr(a.err, DEV_ERR_TIMEOUT);
      mbar_wait(&bar, 0);        // bounded: let copies still in flight land
    }
    __syncthreads();
    return;
  }

  if (PROLONG) {
    // u += P e_2h on the region's DOFs: per region row all corrections are
    // computed before any is added (several nodes in flight per thread)
    constexpr int kXB = 5;           // 32-column chunks per region row (RX <= 160)
    for (int y = warp; y < RY; y += kWarps) {
      const int gj = rj0 + y;
      T v[kXB];
#pragma unroll
      for (int k = 0; k < kXB; ++k) {
        const int x = lane + 32 * k;
        v[k] = T(0);
        if (x < RX && sC[y * RS + x]) {
          const int gi = ri0 + x;
          const T* e = sE + ((gj >> 1) - cj0) * EX + ((gi >> 1) - ci0);
          if (!(gi & 1) && !(gj & 1)) v[k] = e[0];
          else if (!(gj & 1)) v[k] = T(0.5) * (e[0] + e[1]);
          else if (!(gi & 1)) v[k] = T(0.5) * (e[0] + e[EX]);
          else v[k] = T(0.25) * ((e[0] + e[1]) + (e[EX] + e[EX + 1]));
        }
      }
#pragma unroll
      for (int k = 0; k < kXB; ++k) {
        const int x = lane + 32 * k;
        if (x < RX) sU[y * RS + x] += v[k];
      }
    }
    __syncthreads();
  }

  // one listed node of colour c, entry e
  auto listed = [&](int e) {
    T w[MG_ROW + 1];
    int p;
    if (e < RC) {
      p = sP[e];
#pragma unroll
      for (int k = 0; k < MG_ROW; ++k) w[k] = sS[k * RC + e];
    } else {
      const int2 en = a.lent[e0 + e];
      p = (en.x >> 16) * RS + (en.x & 0xffff);
      const T* R = a.rows + (size_t)en.y * MG_ROW;
#pragma unroll
      for (int k = 0; k < MG_ROW; ++k) w[k] = R[k];
    }
    w[MG_ROW] = sF[p];
    sU[p] = row_update(w, sU + p, w[MG_ROW], RS);
  };

  // 4 full colour phases over the region interior: interior nodes by
  // scanning the colour's lattice (a warp per lattice row, kXL nodes in
  // flight per thread), boundary nodes from the list (same-colour nodes
  // never interact)
  for (int c = 0; c < 4; ++c) {
    // first x >= 1 with (ri0 + x) of the colour's parity, then every other one
    const int x0 = 2 - (((c & 1) - ri0) & 1), y0 = 2 - (((c >> 1) - rj0) & 1);
    const int nxl = (RX - x0) / 2, nyl = (RY - y0) / 2;   // lattice nodes with x, y <= R - 2
    for (int yl0 = warp; yl0 < nyl; yl0 += 2 * kWarps) {
      // two lattice rows, kXL nodes each, all loads before any store
      T val[2 * kXL];
      int pp[2 * kXL];
      bool dd[2 * kXL];
#pragma unroll
      for (int k = 0; k < 2 * kXL; ++k) {
        const int yl = yl0 + (k / kXL) * kWarps, xl = lane + 32 * (k % kXL);
        const int p = (y0 + 2 * yl) * RS + x0 + 2 * xl;
        pp[k] = p;
        dd[k] = yl < nyl && xl < nxl && sC[p] == 1;
        val[k] = T(0);
        if (dd[k]) {
          const T* Up = sU + p;
          T s8 = ((Up[-1] + Up[1]) + (Up[-RS] + Up[RS])) +
                 ((Up[-RS - 1] + Up[-RS + 1]) + (Up[RS - 1] + Up[RS + 1]));
          val[k] = (T(3) * sF[p] + s8) * T(0.125);
        }
      }
#pragma unroll
      for (int k = 0; k < 2 * kXL; ++k)
        if (dd[k]) sU[pp[k]] = val[k];
    }
    for (int e = gs[c] + threadIdx.x; e < gs[c + 1]; e += blockDim.x) listed(e);
    __syncthreads();
  }
  // 4 eta phases on the cut-cell vertices only, on nw warps, each thread's
  // nodes in registers
  {
    int g[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) g[c] = gs[c];
    int mc = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) mc = max(mc, g[c + 1] - g[c]);
    const int nw = min(kWarps, max(1, (mc + 31) / 32));
    if (warp < nw && a.eta > 0) {
      auto stage = [&](int e, T* w, int& p) {
        if (e < RC) {
          p = sP[e];
#pragma unroll
          for (int k = 0; k < MG_ROW; ++k) w[k] = sS[k * RC + e];
        } else {
          const int2 en = a.lent[e0 + e];
          p = (en.x >> 16) * RS + (en.x & 0xffff);
          const T* R = a.rows + (size_t)en.y * MG_ROW;
#pragma unroll
          for (int k = 0; k < MG_ROW; ++k) w[k] = R[k];
        }
        w[MG_ROW] = sF[p];
      };
      band_phases_reg<T>(sU, RS, g, a.eta, 32 * nw, stage, listed);
    }
    __syncthreads();
  }

  // owned tile out
  for (int rr = warp; rr < MG_TY; rr += kWarps)
    for (int ii = lane; ii < MG_TX; ii += 32)
      a.uout[L.idx(i0 + ii, j0 + rr)] = sU[(HS + rr) * RS + HS + ii];

  if (RESTRICT) {
    // residual on the owned nodes plus one ring, staged in sE
    constexpr int SX = MG_TX + 2;
    for (int rr = warp; rr < MG_TY + 2; rr += kWarps) {
      for (int ii = lane; ii < SX; ii += 32) {
        const int x = HS - 1 + ii, y = HS - 1 + rr;
        const int p = y * RS + x;
        const uint16_t cd = sC[p];
        T r = T(0);
        if (cd) {
          const T* Up = sU + p;
          if (cd == 1) {
            T s8 = ((Up[-1] + Up[1]) + (Up[-RS] + Up[RS])) +
                   ((Up[-RS - 1] + Up[-RS + 1]) + (Up[RS - 1] + Up[RS + 1]));
            r = sF[p] - (T(8) * Up[0] - s8) * T(1.0 / 3.0);
          } else {
            const T* R = a.rows + (size_t)(row_base(ri0 + x, rj0 + y) + cd - 2) * MG_ROW;
            T acc = R[0] * Up[-RS - 1] + R[1] * Up[-RS] + R[2] * Up[-RS + 1] + R[3] * Up[-1] +
                    R[4] * Up[0] + R[5] * Up[1] + R[6] * Up[RS - 1] + R[7] * Up[RS] +
                    R[8] * Up[RS + 1];
            r = sF[p] - acc;
          }
        }
        sE[rr * SX + ii] = r;
      }
    }
    __syncthreads();
    const Layout& Lc = a.Lc;
    const int I0 = i0 / 2, J0 = j0 / 2;
    for (int it = threadIdx.x; it < (MG_TX / 2) * (MG_TY / 2); it += blockDim.x) {
      const int cy = it / (MG_TX / 2), cx = it - cy * (MG_TX / 2);
      const int I = I0 + cx, J = J0 + cy;
      if (I > Lc.n || J > Lc.n) continue;
      const T* R = sE + (2 * cy + 1) * SX + (2 * cx + 1);
      T rc = R[0] + T(0.5) * ((R[-1] + R[1]) + (R[-SX] + R[SX])) +
             T(0.25) * ((R[-SX - 1] + R[-SX + 1]) + (R[SX - 1] + R[SX + 1]));
      a.Fc[Lc.idx(I, J)] = rc;
    }
  }
}

}  // namespace

int fused_box_x(int eta) { return box_x(eta); }
int fused_box_y(int eta) { return region_y(eta); }
int fused_halo(int eta) { return halo_of(eta); }

size_t fused_smem_bytes(int eta, size_t elem) {
  return kSmemSlack +
         (elem == 8 ? carve<double>(nullptr, eta, nullptr) : carve<float>(nullptr, eta, nullptr));
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
void launch_smooth_step(const FusedArgs<T>& a, const FusedMaps& maps, int ntiles, bool zero_in,
                        bool prolong, bool restrict_, size_t smem, cudaStream_t st) {
  if (!ntiles) return;
  if (zero_in && !prolong && !restrict_)
    launch_pdl(k_smooth_step<T, true, false, false>, ntiles, kThreads, smem, st, a, maps);
  else if (zero_in && !prolong && restrict_)
    launch_pdl(k_smooth_step<T, true, false, true>, ntiles, kThreads, smem, st, a, maps);
  else if (!zero_in && !prolong && !restrict_)
    launch_pdl(k_smooth_step<T, false, false, false>, ntiles, kThreads, smem, st, a, maps);
  else if (!zero_in && !prolong && restrict_)
    launch_pdl(k_smooth_step<T, false, false, true>, ntiles, kThreads, smem, st, a, maps);
  else if (!zero_in && prolong && !restrict_)
    launch_pdl(k_smooth_step<T, false, true, false>, ntiles, kThreads, smem, st, a, maps);
  else
    launch_pdl(k_smooth_step<T, false, true, true>, ntiles, kThreads, smem, st, a, maps);
}

template cudaError_t configure_fused<float>(size_t);
template cudaError_t configure_fused<double>(size_t);
template void launch_smooth_step<float>(const FusedArgs<float>&, const FusedMaps&, int, bool, bool,
                                        bool, size_t, cudaStream_t);
template void launch_smooth_step<double>(const FusedArgs<double>&, const FusedMaps&, int, bool,
                                         bool, bool, size_t, cudaStream_t);
