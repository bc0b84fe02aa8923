// V-cycle kernels (Alg. 1 applied recursively, Sec. 3.2) for one level of
// the ghost-FEM hierarchy, templated on the arithmetic type T (double or
// float).  All are matrix-free stencil passes over 64 x 32 node tiles:
//
//   k_gs_sweep        one Gauss-Seidel sweep (Sec. 4.1), 4 colours
//                     (i mod 2, j mod 2) in the order (0,0),(1,0),(0,1),(1,1),
//                     temporally blocked in shared memory with a 4-node halo;
//                     reads u_in, writes u_out (ping-pong buffers)
//   k_band            the eta extra sweeps restricted to the vertices of cut
//                     cells (Sec. 5.3), 4 eta colour phases per 32 x 32 band
//                     tile with a (4 eta + 1)-node halo, in place
//   k_resid_restrict  r = F - A u and r_2h = P^T r (Sec. 5.1 weights 1, 1/2,
//                     1/4), optionally with ||r||_inf and ||r||_2^2
//   k_residual        r = F - A u on one level with norms, optional scaled
//                     copy of r in another precision (refinement residual)
//   k_prolong         u += P e_2h on the DOFs (bilinear interpolation)
//   k_coarse_solve    u = A^{-1} F on the coarsest level (dense inverse)
//   k_rhs             F = M f + G g (Eq. disc_rhs with Q1 interpolants)
#include "cycle.cuh"
#include "bandreg.cuh"
#include "rhs_impl.cuh"

namespace {

constexpr int SW_H = 4;
constexpr int SW_RX = MG_TX + 2 * SW_H;   // 72
constexpr int SW_RY = MG_TY + 2 * SW_H;   // 40
constexpr int SW_PX = SW_RX / 2;          // 36
constexpr int SW_PY = SW_RY / 2;          // 20
constexpr int SW_PLANE = SW_PX * SW_PY;   // nodes per parity plane
constexpr int kThreads = 256;

template <class T>
__device__ __forceinline__ const T* row_of(const OpArgs<T>& op, int i, int j, int cd) {
  int t = op.L.tile_of(i, j);
  if (!MG_CHECKED(t >= 0 && t < op.L.ntx * op.L.nty)) t = 0;
  const int r = checked_row(op.tile_base[t] + cd - 2, op.n_rows);
  return op.rows + (size_t)r * MG_ROW;
}

// MODE: kSweepPlain (u from uin), kSweepZero (u = 0: first pre-smoothing
// step), kSweepProlong (u = uin + P e_2h: the prolongation of Sec. 5.1,
// added while loading, with the same arithmetic as k_prolong).

// REV: the colours in the reverse order (1,1), (0,1), (1,0), (0,0): the
// transposed sweep of the transposed V-cycle.
template <class T, int MODE, bool REV = false>
__global__ void __launch_bounds__(kThreads)
k_gs_sweep(OpArgs<T> op, const int* __restrict__ tiles, const T* __restrict__ uin,
           T* __restrict__ uout, const T* __restrict__ F, T* __restrict__ bval, Layout Lc,
           const T* __restrict__ ec) {
  griddep_launch_next();
  griddep_wait();
  typedef typename Vec2<T>::type T2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sU = reinterpret_cast<T*>(smem_raw);            // [4][PY][PX] parity planes
  T* sF = sU + 4 * SW_PLANE;
  uint16_t* sC = reinterpret_cast<uint16_t*>(sF + 4 * SW_PLANE);

  const int t = tiles[blockIdx.x];
  const int i0 = (t % op.L.ntx) * MG_TX, j0 = (t / op.L.ntx) * MG_TY;
  const int ri0 = i0 - SW_H, rj0 = j0 - SW_H;        // both even

  constexpr int B = 3;
  for (int it0 = threadIdx.x; it0 < SW_RY * SW_PX; it0 += B * blockDim.x) {
    T2 f2[B], u2[B];
    uint32_t c2[B];
    T e00[B], e10[B], e01[B], e11[B];   // coarse values around the node pair
#pragma unroll
    for (int b = 0; b < B; ++b) {
      int it = it0 + b * blockDim.x;
      int rj = it / SW_PX, a = it - rj * SW_PX;
      bool ok = it < SW_RY * SW_PX;
      size_t g = ok ? op.L.idx(ri0 + 2 * a, rj0 + rj) : op.L.idx(0, 0);
      f2[b] = *reinterpret_cast<const T2*>(F + g);
      if (MODE != kSweepZero) u2[b] = *reinterpret_cast<const T2*>(uin + g);
      c2[b] = *reinterpret_cast<const uint32_t*>(op.code + g);
      if (MODE == kSweepProlong) {
        // fine nodes (2I, j) and (2I+1, j), I = (ri0 + 2a) / 2, J = j / 2:
        // E(I, J), E(I+1, J) and, for odd j, the row J+1
        const int gi = ri0 + 2 * a, gj = rj0 + rj;
        const bool in = ok && gi >= 0 && gj >= 0 && gi <= op.L.n && gj <= op.L.n;
        const T* E = ec + (in ? Lc.idx(gi >> 1, gj >> 1) : Lc.idx(0, 0));
        e00[b] = E[0];
        e10[b] = E[1];
        e01[b] = (gj & 1) ? E[Lc.pitch] : T(0);
        e11[b] = (gj & 1) ? E[Lc.pitch + 1] : T(0);
      }
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
      int it = it0 + b * blockDim.x;
      if (it >= SW_RY * SW_PX) continue;
      int rj = it / SW_PX, a = it - rj * SW_PX;
      int pl = (rj & 1) * 2 * SW_PLANE + (rj >> 1) * SW_PX + a;
      const uint16_t c0 = (uint16_t)(c2[b] & 0xffffu), c1 = (uint16_t)(c2[b] >> 16);
      T u0 = MODE == kSweepZero ? T(0) : u2[b].x;
      T u1 = MODE == kSweepZero ? T(0) : u2[b].y;
      if (MODE == kSweepProlong) {
        // same association as k_prolong: u + e with e the bilinear average
        if ((rj0 + rj) & 1) {
          if (c0) u0 = u0 + T(0.5) * (e00[b] + e01[b]);
          if (c1) u1 = u1 + T(0.25) * ((e00[b] + e10[b]) + (e01[b] + e11[b]));
        } else {
          if (c0) u0 = u0 + e00[b];
          if (c1) u1 = u1 + T(0.5) * (e00[b] + e10[b]);
        }
      }
      sF[pl] = f2[b].x;
      sF[pl + SW_PLANE] = f2[b].y;
      sU[pl] = u0;
      sU[pl + SW_PLANE] = u1;
      sC[pl] = c0;
      sC[pl + SW_PLANE] = c1;
    }
  }
  __syncthreads();

#pragma unroll 1
  for (int k = 0; k < 4; ++k) {
    const int col = REV ? 3 - k : k;
    const int ci = col & 1, cj = col >> 1;
    T* P = sU + (cj * 2 + ci) * SW_PLANE;
    const T* PXn = sU + (cj * 2 + (ci ^ 1)) * SW_PLANE;
    const T* PYn = sU + ((cj ^ 1) * 2 + ci) * SW_PLANE;
    const T* PDn = sU + ((cj ^ 1) * 2 + (ci ^ 1)) * SW_PLANE;
    const T* PF = sF + (cj * 2 + ci) * SW_PLANE;
    const uint16_t* PC = sC + (cj * 2 + ci) * SW_PLANE;
    const int lo = k + 1, hix = SW_RX - 1 - k, hiy = SW_RY - 1 - k;
    for (int it = threadIdx.x; it < SW_PLANE; it += blockDim.x) {
      int b = it / SW_PX, a = it - b * SW_PX;
      int ri = 2 * a + ci, rj = 2 * b + cj;
      if (ri < lo || ri >= hix || rj < lo || rj >= hiy) continue;
      uint16_t cd = PC[it];
      if (cd == 0) continue;
      int xm = a + ci - 1, xp = a + ci, ym = b + cj - 1, yp = b + cj;
      T w = PXn[b * SW_PX + xm], e = PXn[b * SW_PX + xp];
      T s = PYn[ym * SW_PX + a], n = PYn[yp * SW_PX + a];
      T sw = PDn[ym * SW_PX + xm], se = PDn[ym * SW_PX + xp];
      T nw = PDn[yp * SW_PX + xm], ne = PDn[yp * SW_PX + xp];
      T f = PF[it];
      T unew;
      if (cd == 1) {
        // interior row: 8/3 u_p - 1/3 (sum of 8 neighbours) = F_p
        unew = (T(3) * f + ((w + e) + (s + n)) + ((sw + se) + (nw + ne))) * T(0.125);
      } else {
        const T* R = row_of(op, ri0 + ri, rj0 + rj, cd);
        T uc = P[it];
        T acc = R[0] * sw + R[1] * s + R[2] * se + R[3] * w + R[4] * uc + R[5] * e +
                R[6] * nw + R[7] * n + R[8] * ne;
        unew = uc + (f - acc) * R[9];
      }
      P[it] = unew;
    }
    __syncthreads();
  }

  const int base = op.tile_base[t];
  for (int it = threadIdx.x; it < MG_TY * (MG_TX / 2); it += blockDim.x) {
    int rr = it / (MG_TX / 2), a2 = it - rr * (MG_TX / 2);
    int rj = SW_H + rr, a = SW_H / 2 + a2;
    int pl = (rj & 1) * 2 * SW_PLANE + (rj >> 1) * SW_PX + a;
    T2 v;
    v.x = sU[pl];
    v.y = sU[pl + SW_PLANE];
    *reinterpret_cast<T2*>(uout + op.L.idx(i0 + 2 * a2, j0 + rr)) = v;
    if (bval) {
      uint16_t c0 = sC[pl], c1 = sC[pl + SW_PLANE];
      if (c0 >= 2) bval[checked_row(base + c0 - 2, op.n_rows)] = v.x;
      if (c1 >= 2) bval[checked_row(base + c1 - 2, op.n_rows)] = v.y;
    }
  }
}

// Extra Gauss-Seidel sweeps on the cut-cell vertices (boundary nodes).  Each
// block owns the boundary nodes of a 32 x 32 band tile and recomputes the
// 4 eta colour phases redundantly on a halo of 4 eta + 1 nodes, so the owned
// values equal those of the global sweep.  Boundary values are read from
// bval (written by the preceding full sweep) and never from u, which other
// blocks update concurrently.  The region's boundary nodes come from a list
// built at setup (grouped by colour, rim last), so the block only
//   1. loads u of the region with one TMA box copy and, meanwhile, stages
//      row, F and bval of its first BandCap<T> listed nodes,
//   2. overwrites the listed nodes with bval,
//   3. runs the 4 eta colour phases on as many warps as the longest colour
//      has 32-node groups (one warp syncs with __syncwarp, more with a
//      named barrier),
//   4. writes the owned listed nodes back.
template <class T> struct BandCap;
template <> struct BandCap<float> { static constexpr int value = 384; };
template <> struct BandCap<double> { static constexpr int value = 256; };
constexpr int kBandNS = MG_ROW + 2;    // staged per node: row, F, bval
// 4 warps: the colour phases need at most a few (a 66 x 66 region holds a few
// hundred boundary nodes), and small blocks let every band tile of a
// 4096^2 level be resident at once (one wave)
constexpr int kBandThreads = 128;

__host__ __device__ constexpr int band_halo(int eta) { return 4 * eta + 1; }
__host__ __device__ constexpr int band_region(int eta) { return 32 + 2 * band_halo(eta); }
__host__ __device__ inline size_t band_a128(size_t b) { return (b + 127) & ~(size_t)127; }

template <class T, bool REV = false>
__global__ void __launch_bounds__(kBandThreads)
k_band(OpArgs<T> op, const int* __restrict__ btiles, int nbx, int eta, T* __restrict__ u,
       const T* __restrict__ F, const T* __restrict__ bval, const int* __restrict__ boff,
       const int2* __restrict__ bent, const __grid_constant__ BandMaps maps, int umap,
       unsigned* err, unsigned wait_polls) {
  constexpr int EC = BandCap<T>::value;
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  unsigned char* smem_raw = smem_align128(smem_dyn);
  const int H = band_halo(eta);
  const int RB = band_region(eta);
  const int RS = tma_box_w(RB);                        // shared row stride (TMA box width)
  T* sUb = reinterpret_cast<T*>(smem_raw);             // [RB][RS] TMA box
  T* sS = reinterpret_cast<T*>(smem_raw + band_a128((size_t)RS * RB * sizeof(T)));  // [NS][EC]
  int* sP = reinterpret_cast<int*>(sS + kBandNS * EC); // [EC] region positions
  __shared__ uint64_t bar;
  __shared__ int gs[6];
  const int b = blockIdx.x;
  const int bt = btiles[b];
  const int bi0 = (bt % nbx) * 32 - H, bj0 = (bt / nbx) * 32 - H;
  const int ax = tma_floor(bi0 + MG_G);
  T* sU = sUb + (bi0 + MG_G - ax);                     // region (x, y) at sU[y RS + x]
  __shared__ int bad;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    bad = !tma_box_ok(sUb, ax);
  }
  const int e0 = boff[5 * b];
  if (threadIdx.x < 6) gs[threadIdx.x] = boff[5 * b + threadIdx.x] - e0;
  const int m = boff[5 * b + 5] - e0;                  // all groups, rim included
  const int nrim0 = boff[5 * b + 4] - e0;              // first rim entry
  // 1a. static part of the listed nodes (rows, positions): before the wait
  //     for the previous kernel
  for (int e = threadIdx.x; e < m && e < EC; e += blockDim.x) {
    const int2 en = bent[e0 + e];
    const int2 xy = region_pos(en, e < nrim0, RB, RB);
    const int x = xy.x, y = xy.y;
    T v[MG_ROW];
    if (e < nrim0) {
      const T* R = op.rows + (size_t)checked_row(en.y, op.n_rows) * MG_ROW;
#pragma unroll
      for (int k = 0; k < MG_ROW; ++k) v[k] = R[k];
    } else {
#pragma unroll
      for (int k = 0; k < MG_ROW; ++k) v[k] = T(0);
    }
#pragma unroll
    for (int k = 0; k < MG_ROW; ++k) sS[k * EC + e] = v[k];
    sP[e] = y * RS + x;
  }
  __syncthreads();
  griddep_wait();
  // dependents launch only now: when the next kernel starts, everything
  // before this one has completed (see band_independent)
  griddep_launch_next();
  if (threadIdx.x == 0) {
    if (!bad) {
      mbar_arrive_expect_tx(&bar, (uint32_t)((size_t)RS * RB * sizeof(T)));
      tma_load_2d(sUb, &maps.u[umap], ax, bj0 + MG_G, &bar);
    } else {
      atomicOr(err, DEV_ERR_ALIGN);
      mbar_arrive_expect_tx(&bar, 0);
    }
  }
  // 1b. F and bval of the listed nodes, while the TMA runs
  for (int e = threadIdx.x; e < m && e < EC; e += blockDim.x) {
    const int2 en = bent[e0 + e];
    const int2 xy = region_pos(en, e < nrim0, RB, RB);
    const int x = xy.x, y = xy.y;
    const T f = e < nrim0 ? F[op.L.idx(bi0 + x, bj0 + y)] : T(0);
    const T bv = bval[checked_row(en.y, op.n_rows)];
    sS[MG_ROW * EC + e] = f;
    sS[(MG_ROW + 1) * EC + e] = bv;
  }
  const bool ok = mbar_wait(&bar, 0, wait_polls);
  if (__syncthreads_or(!ok || bad)) {
    if (threadIdx.x == 0 && !ok) {
      atomicOr(err, DEV_ERR_TIMEOUT);
      mbar_wait(&bar, 0);        // bounded: let a copy still in flight land
    }
    __syncthreads();
    return;
  }
  // 2. boundary values from bval
  for (int e = threadIdx.x; e < m; e += blockDim.x) {
    if (e < EC) {
      sU[sP[e]] = sS[(MG_ROW + 1) * EC + e];
    } else {
      const int2 en = bent[e0 + e];
      const int2 xy = region_pos(en, e < nrim0, RB, RB);
      sU[xy.y * RS + xy.x] = bval[checked_row(en.y, op.n_rows)];
    }
  }
  __syncthreads();
  // 3. 4 eta colour phases on nw warps, each thread's nodes in registers
  int g[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) g[c] = gs[c];
  int mc = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) mc = max(mc, g[c + 1] - g[c]);
  const int nw = min((int)(blockDim.x >> 5), max(1, (mc + 31) / 32));
  if ((int)(threadIdx.x >> 5) < nw) {
    auto fetch = [&](int e, T* w, int& p) {
      if (e < EC) {
        p = sP[e];
#pragma unroll
        for (int k = 0; k <= MG_ROW; ++k) w[k] = sS[k * EC + e];
      } else {
        const int2 en = bent[e0 + e];
        const int2 xy = region_pos(en, true, RB, RB);
        const int x = xy.x, y = xy.y;
        p = y * RS + x;
        const T* R = op.rows + (size_t)checked_row(en.y, op.n_rows) * MG_ROW;
#pragma unroll
        for (int k = 0; k < MG_ROW; ++k) w[k] = R[k];
        w[MG_ROW] = F[op.L.idx(bi0 + x, bj0 + y)];
      }
    };
    auto extra = [&](int e) {
      T w[MG_ROW + 1];
      int p;
      fetch(e, w, p);
      const T* Up = sU + p;
      T acc = w[0] * Up[-RS - 1] + w[1] * Up[-RS] + w[2] * Up[-RS + 1] + w[3] * Up[-1] +
              w[4] * Up[0] + w[5] * Up[1] + w[6] * Up[RS - 1] + w[7] * Up[RS] +
              w[8] * Up[RS + 1];
      sU[p] = Up[0] + (w[MG_ROW] - acc) * w[9];
    };
    band_phases_reg<T, decltype(fetch), decltype(extra), REV>(sU, RS, g, eta, 32 * nw, fetch,
                                                               extra);
  }
  __syncthreads();
  // 4. owned listed nodes back to u
  for (int e = threadIdx.x; e < nrim0; e += blockDim.x) {
    int x, y;
    if (e < EC) {
      const int p = sP[e];
      y = p / RS;
      x = p - y * RS;
    } else {
      const int2 xy = region_pos(bent[e0 + e], true, RB, RB);
      x = xy.x;
      y = xy.y;
    }
    if (x >= H && x < H + 32 && y >= H && y < H + 32)
      u[op.L.idx(bi0 + x, bj0 + y)] = sU[y * RS + x];
  }
}

// Residual of one node from a plain 2D shared-memory region (row stride RS).
template <class T, int RS>
__device__ __forceinline__ T node_residual(const OpArgs<T>& op, const T* Up, uint16_t cd, T f,
                                           int gi, int gj) {
  if (cd == 0) return T(0);
  if (cd == 1) {
    T s8 = ((Up[-1] + Up[1]) + (Up[-RS] + Up[RS])) +
           ((Up[-RS - 1] + Up[-RS + 1]) + (Up[RS - 1] + Up[RS + 1]));
    return f - (T(8) * Up[0] - s8) * T(1.0 / 3.0);
  }
  const T* R = row_of(op, gi, gj, cd);
  T acc = R[0] * Up[-RS - 1] + R[1] * Up[-RS] + R[2] * Up[-RS + 1] + R[3] * Up[-1] +
          R[4] * Up[0] + R[5] * Up[1] + R[6] * Up[RS - 1] + R[7] * Up[RS] + R[8] * Up[RS + 1];
  return f - acc;
}

constexpr int RR_X = 68, RR_Y = 36;   // region of a 64 x 32 fine block with 2-node halo

template <class T, bool NORM>
__global__ void __launch_bounds__(kThreads)
k_resid_restrict(OpArgs<T> op, const T* __restrict__ u, const T* __restrict__ F, Layout Lc,
                 const int* __restrict__ ctiles, T* __restrict__ Fc, double* __restrict__ norms,
                 const uint8_t* __restrict__ touch) {
  griddep_launch_next();
  if (!band_independent(touch)) griddep_wait();
  typedef typename Vec2<T>::type T2;
  __shared__ __align__(16) T sU[RR_Y * RR_X];
  __shared__ __align__(16) T sR[RR_Y * RR_X];
  __shared__ uint16_t sC[RR_Y * RR_X];
  const int t = ctiles[blockIdx.x >> 2], sub = blockIdx.x & 3;
  const int I0 = (t % Lc.ntx) * MG_TX + (sub & 1) * 32;
  const int J0 = (t / Lc.ntx) * MG_TY + (sub >> 1) * 16;
  if (I0 > Lc.n || J0 > Lc.n) return;
  const int fi0 = 2 * I0 - 2, fj0 = 2 * J0 - 2;
  {
    constexpr int B = 4;
    for (int it0 = threadIdx.x; it0 < RR_Y * (RR_X / 2); it0 += B * blockDim.x) {
      T2 u2[B], f2[B];
      uint32_t c2[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        int it = it0 + b * blockDim.x;
        int rj = it / (RR_X / 2), a = it - rj * (RR_X / 2);
        size_t g = it < RR_Y * (RR_X / 2) ? op.L.idx(fi0 + 2 * a, fj0 + rj) : op.L.idx(0, 0);
        u2[b] = __ldcg(reinterpret_cast<const T2*>(u + g));
        f2[b] = __ldcg(reinterpret_cast<const T2*>(F + g));
        c2[b] = *reinterpret_cast<const uint32_t*>(op.code + g);
      }
#pragma unroll
      for (int b = 0; b < B; ++b) {
        int it = it0 + b * blockDim.x;
        if (it >= RR_Y * (RR_X / 2)) continue;
        int rj = it / (RR_X / 2), a = it - rj * (RR_X / 2);
        sU[rj * RR_X + 2 * a] = u2[b].x;
        sU[rj * RR_X + 2 * a + 1] = u2[b].y;
        sR[rj * RR_X + 2 * a] = f2[b].x;       // F, replaced by r below
        sR[rj * RR_X + 2 * a + 1] = f2[b].y;
        sC[rj * RR_X + 2 * a] = (uint16_t)(c2[b] & 0xffffu);
        sC[rj * RR_X + 2 * a + 1] = (uint16_t)(c2[b] >> 16);
      }
    }
  }
  __syncthreads();
  unsigned long long vmax = 0ull;
  double vsum = 0.0;
  // r = F - A u in place of F (the restriction below reads only these nodes)
  for (int it = threadIdx.x; it < (RR_Y - 2) * (RR_X - 2); it += blockDim.x) {
    int rj = 1 + it / (RR_X - 2), ri = 1 + it % (RR_X - 2);
    int p = rj * RR_X + ri;
    uint16_t cd = sC[p];
    T r = T(0);
    if (cd) {
      int gi = fi0 + ri, gj = fj0 + rj;
      r = node_residual<T, RR_X>(op, sU + p, cd, sR[p], gi, gj);
    }
    sR[p] = r;
    if (NORM && ri >= 2 && ri < RR_X - 2 && rj >= 2 && rj < RR_Y - 2) {
      double rd = (double)r;
      max_abs(vmax, rd);
      vsum += rd * rd;
    }
  }
  __syncthreads();
  for (int it = threadIdx.x; it < 32 * 16; it += blockDim.x) {
    int cy = it / 32, cx = it - cy * 32;
    int I = I0 + cx, J = J0 + cy;
    if (I > Lc.n || J > Lc.n) continue;
    const T* R = sR + (2 * cy + 2) * RR_X + (2 * cx + 2);
    T rc = R[0] + T(0.5) * ((R[-1] + R[1]) + (R[-RR_X] + R[RR_X])) +
           T(0.25) * ((R[-RR_X - 1] + R[-RR_X + 1]) + (R[RR_X - 1] + R[RR_X + 1]));
    Fc[Lc.idx(I, J)] = rc;
  }
  if (NORM) block_norms_to_global(vmax, vsum, norms);
}

// One flag per block of a later launch: does the block's input region hold a
// boundary node (code >= 2) of the level with layout L?  The regions are
// those of k_gs_sweep_f32 (64 x 32 tile, 4-node halo), of the coarse nodes
// its prolongation reads, and of k_resid_restrict (RR_X x RR_Y).  The
// prolongation window is a superset: a flag set without need only makes a
// block wait.
__global__ void k_touch_flags(int mode, Layout L, const uint16_t* __restrict__ code,
                              const int* __restrict__ tiles, int tpr, uint8_t* __restrict__ flag) {
  __shared__ int any;
  const int b = blockIdx.x;
  int x0, y0, w, h;
  if (mode == TOUCH_RESTRICT) {
    const int t = tiles[b >> 2], sub = b & 3;
    const int I0 = (t % tpr) * MG_TX + (sub & 1) * 32, J0 = (t / tpr) * MG_TY + (sub >> 1) * 16;
    x0 = 2 * I0 - 2;
    y0 = 2 * J0 - 2;
    w = RR_X;
    h = RR_Y;
  } else {
    const int t = tiles[b];
    const int ri0 = (t % tpr) * MG_TX - 4, rj0 = (t / tpr) * MG_TY - 4;
    if (mode == TOUCH_SWEEP) {
      x0 = ri0;
      y0 = rj0;
      w = MG_TX + 8;
      h = MG_TY + 8;
    } else {
      // fine nodes gi in [ri0, ri0 + MG_TX + 8) read coarse nodes gi / 2 .. gi / 2 + 2
      x0 = (ri0 >> 1) - 1;
      y0 = (rj0 >> 1) - 1;
      w = (MG_TX + 8) / 2 + 4;
      h = (MG_TY + 8) / 2 + 4;
    }
  }
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  int hit = 0;
  for (int p = threadIdx.x; p < w * h; p += blockDim.x) {
    const int gi = x0 + p % w, gj = y0 + p / w;
    if (gi >= 0 && gj >= 0 && gi <= L.n && gj <= L.n && code[L.idx(gi, gj)] >= 2) hit = 1;
  }
  if (hit) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) flag[b] = (uint8_t)any;
}

template <class T, class TR>
__global__ void __launch_bounds__(kThreads)
k_residual(OpArgs<T> op, const int* __restrict__ tiles, const T* __restrict__ u,
           const T* __restrict__ F, TR* __restrict__ rout, T scale, double* __restrict__ norms,
           int l2, double* __restrict__ part) {
  griddep_launch_next();
  griddep_wait();
  typedef typename Vec2<T>::type T2;
  __shared__ __align__(16) T sU[RR_Y * RR_X];
  __shared__ uint16_t sC[RR_Y * RR_X];
  const int t = tiles[blockIdx.x];
  const int i0 = (t % op.L.ntx) * MG_TX, j0 = (t / op.L.ntx) * MG_TY;
  const int fi0 = i0 - 2, fj0 = j0 - 2;
  {
    constexpr int B = 4;
    for (int it0 = threadIdx.x; it0 < RR_Y * (RR_X / 2); it0 += B * blockDim.x) {
      T2 u2[B];
      uint32_t c2[B];
#pragma unroll
      for (int b = 0; b < B; ++b) {
        int it = it0 + b * blockDim.x;
        int rj = it / (RR_X / 2), a = it - rj * (RR_X / 2);
        size_t g = it < RR_Y * (RR_X / 2) ? op.L.idx(fi0 + 2 * a, fj0 + rj) : op.L.idx(0, 0);
        u2[b] = __ldcg(reinterpret_cast<const T2*>(u + g));
        c2[b] = *reinterpret_cast<const uint32_t*>(op.code + g);
      }
#pragma unroll
      for (int b = 0; b < B; ++b) {
        int it = it0 + b * blockDim.x;
        if (it >= RR_Y * (RR_X / 2)) continue;
        int rj = it / (RR_X / 2), a = it - rj * (RR_X / 2);
        sU[rj * RR_X + 2 * a] = u2[b].x;
        sU[rj * RR_X + 2 * a + 1] = u2[b].y;
        sC[rj * RR_X + 2 * a] = (uint16_t)(c2[b] & 0xffffu);
        sC[rj * RR_X + 2 * a + 1] = (uint16_t)(c2[b] >> 16);
      }
    }
  }
  __syncthreads();
  // Interior rows 8/3 u_p - 1/3 (sum of the 8 neighbours) are (9 u_p - box)
  // / 3 with box the 3 x 3 sum, taken separably: row sums of three nodes for
  // the owned columns on the owned rows and one more above and below (sH),
  // then three of them per node -- 6 fp64 operations per node instead of 10,
  // this kernel being bound by the fp64 rate.
  __shared__ __align__(16) T sH[(MG_TY + 2) * MG_TX];
  __shared__ uint16_t s_list[MG_TY * MG_TX];
  __shared__ int s_nl;
  if (threadIdx.x == 0) s_nl = 0;
  for (int it = threadIdx.x; it < (MG_TY + 2) * MG_TX; it += blockDim.x) {
    const int y = it / MG_TX, x = it - y * MG_TX;     // region row y + 1, column x + 2
    const T* r = sU + (y + 1) * RR_X + x + 2;
    sH[it] = (r[-1] + r[0]) + r[1];
  }
  __syncthreads();
  unsigned long long vmax = 0ull;
  double vsum = 0.0;
  auto finish = [&](size_t g, T r) {
    double rd = (double)r;
    max_abs(vmax, rd);
    if (l2) vsum += rd * rd;
    // for an fp32 output with a power-of-two scale (the refinement's sigma)
    // the scaling is exact in fp32 after the rounding to fp32, one fp64
    // instruction fewer per node (identical unless r is below the fp32
    // normal range)
    if (rout) {
      if (sizeof(TR) < sizeof(T)) rout[g] = (TR)r * (TR)scale;
      else rout[g] = (TR)(r * scale);
    }
  };
  // interior nodes here (unrolled so that several nodes' loads of F are in
  // flight at once); boundary nodes go to a list and are done after, a
  // thread each, so that their row products do not hold up whole warps
  // (s_nl was cleared before the barrier above).  With the l2 sum they stay
  // in place: the list's order varies from run to run, and so would the
  // sum's last bits.
#pragma unroll 4
  for (int it = threadIdx.x; it < MG_TY * MG_TX; it += blockDim.x) {
    int rr = it / MG_TX, ii = it - rr * MG_TX;
    int p = (rr + 2) * RR_X + ii + 2;
    uint16_t cd = sC[p];
    if (cd >= 2 && !l2) {
      s_list[atomicAdd(&s_nl, 1)] = (uint16_t)it;
      continue;
    }
    const int gi = i0 + ii, gj = j0 + rr;
    size_t g = op.L.idx(gi, gj);
    T r = T(0);
    if (cd == 1) {
      const T* h = sH + it;                            // rows rr .. rr + 2 of sH
      const T box = (h[0] + h[MG_TX]) + h[2 * MG_TX];
      r = fma(fma(T(9), sU[p], -box), T(-1.0 / 3.0), F[g]);
    } else if (cd >= 2) {
      r = node_residual<T, RR_X>(op, sU + p, cd, F[g], gi, gj);
    }
    finish(g, r);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < s_nl; e += blockDim.x) {
    const int it = s_list[e];
    const int rr = it / MG_TX, ii = it - rr * MG_TX;
    const int p = (rr + 2) * RR_X + ii + 2;
    const int gi = i0 + ii, gj = j0 + rr;
    const size_t g = op.L.idx(gi, gj);
    finish(g, node_residual<T, RR_X>(op, sU + p, sC[p], F[g], gi, gj));
  }
  if (norms) {
    if (part) block_norms_partial(vmax, vsum, norms, part + blockIdx.x);
    else block_norms_to_global(vmax, vsum, norms);
  }
}

// norms[1] = the sum of part[0 .. n - 1] in a fixed order (one block)
__global__ void __launch_bounds__(kThreads) k_sum_partials(const double* __restrict__ part, int n,
                                                           double* __restrict__ norms) {
  griddep_launch_next();
  griddep_wait();
  __shared__ double s[kThreads];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += kThreads) v += part[i];
  s[threadIdx.x] = v;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) norms[1] = s[0];
}

template <class T>
__global__ void __launch_bounds__(kThreads)
k_prolong(OpArgs<T> op, const int* __restrict__ tiles, T* __restrict__ uf, Layout Lc,
          const T* __restrict__ ec) {
  griddep_launch_next();
  griddep_wait();
  const int t = tiles[blockIdx.x];
  const int i0 = (t % op.L.ntx) * MG_TX, j0 = (t / op.L.ntx) * MG_TY;
  constexpr int B = MG_TX * MG_TY / kThreads;     // 8 nodes per thread, loads batched
  uint16_t cd[B];
  T uu[B];
#pragma unroll
  for (int b = 0; b < B; ++b) {
    int it = threadIdx.x + b * blockDim.x;
    int rr = it / MG_TX, ii = it - rr * MG_TX;
    size_t g = op.L.idx(i0 + ii, j0 + rr);
    cd[b] = op.code[g];
    uu[b] = uf[g];
  }
#pragma unroll
  for (int b = 0; b < B; ++b) {
    if (cd[b] == 0) continue;
    int it = threadIdx.x + b * blockDim.x;
    int rr = it / MG_TX, ii = it - rr * MG_TX;
    int i = i0 + ii, j = j0 + rr;
    const T* E = ec + Lc.idx(i >> 1, j >> 1);
    T e;
    if (!(i & 1) && !(j & 1)) e = E[0];
    else if (!(j & 1)) e = T(0.5) * (E[0] + E[1]);
    else if (!(i & 1)) e = T(0.5) * (E[0] + E[Lc.pitch]);
    else e = T(0.25) * ((E[0] + E[1]) + (E[Lc.pitch] + E[Lc.pitch + 1]));
    uf[op.L.idx(i, j)] = uu[b] + e;
  }
}

// bval[r] = u at boundary node r (bnode[r] = i | j << 16): the snapshot the
// band kernel reads when no full sweep has just written it (transposed step)
template <class T>
__global__ void k_gather_bval(Layout L, const int* __restrict__ bnode, int nb,
                              const T* __restrict__ u, T* __restrict__ bval) {
  griddep_launch_next();
  griddep_wait();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nb) return;
  const int p = bnode[r];
  bval[r] = u[L.idx(p & 0xffff, p >> 16)];
}

template <class T>
__global__ void k_coarse_solve(Layout Lc, const double* __restrict__ Ainv, const T* __restrict__ Fc,
                               T* __restrict__ uc) {
  griddep_launch_next();
  griddep_wait();
  extern __shared__ double sF[];
  const int n = Lc.n, m = (n + 1) * (n + 1);
  for (int p = threadIdx.x; p < m; p += blockDim.x)
    sF[p] = (double)Fc[Lc.idx(p % (n + 1), p / (n + 1))];
  __syncthreads();
  for (int p = threadIdx.x; p < m; p += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < m; ++c) s += Ainv[(size_t)c * m + p] * sF[c];
    uc[Lc.idx(p % (n + 1), p / (n + 1))] = (T)s;
  }
}

// F = M f + G g on one active tile per block (rhs_impl.cuh), with ||F||_inf
__global__ void __launch_bounds__(kThreads)
k_rhs(RhsArgs a, const int* __restrict__ tiles, const double* __restrict__ f,
      const double* __restrict__ g, double* __restrict__ F, double* __restrict__ norms) {
  block_norms_to_global(rhs_tile(a, tiles[blockIdx.x], f, g, F), 0.0, norms);
}

// Adjoint of the right-hand side map (f, g) -> F = M f + G g (Eq. disc_rhs):
// for w on the DOFs (padded layout, zero elsewhere) dLdf = M^T w = M w (the
// mass matrices are symmetric) and dLdg = G^T w, on one active tile.
// Interior nodes take the separable mass stencil of k_rhs and no G term;
// vertices of cut cells sum the cells one by one with column `av` of Mk, Gk.
__global__ void __launch_bounds__(kThreads)
k_rhs_adj(RhsArgs a, const int* __restrict__ tiles, const double* __restrict__ w,
          double* __restrict__ dLdf, double* __restrict__ dLdg, double* __restrict__ dLdn) {
  __shared__ double sw[RHS_Y * RHS_X];       // w on the tile plus one ring
  __shared__ double st[RHS_Y * MG_TX];       // row pass w(i-1) + 4 w(i) + w(i+1)
  const int n = a.L.n;
  const int t = tiles[blockIdx.x];
  const int i0 = (t % a.L.ntx) * MG_TX, j0 = (t / a.L.ntx) * MG_TY;
  for (int q = threadIdx.x; q < RHS_Y * RHS_X; q += blockDim.x) {
    const int y = q / RHS_X, x = q - y * RHS_X;
    sw[q] = w[a.L.idx(i0 - 1 + x, j0 - 1 + y)];        // zero margin: no checks needed
  }
  __syncthreads();
  for (int q = threadIdx.x; q < RHS_Y * MG_TX; q += blockDim.x) {
    const int y = q / MG_TX, x = q - y * MG_TX;
    const double* r = sw + y * RHS_X + x;
    st[q] = fma(4.0, r[1], r[0] + r[2]);
  }
  __syncthreads();
  const double h2 = a.h * a.h / 36.0;
  for (int q = threadIdx.x; q < MG_TY * MG_TX; q += blockDim.x) {
    const int y = q / MG_TX, x = q - y * MG_TX;
    const int i = i0 + x, j = j0 + y;
    const size_t gk = a.L.idx(i, j);
    const uint16_t cd = a.code[gk];
    double sf = 0.0, sg = 0.0, sn = 0.0;
    if (cd == 1) {
      const double* c = st + y * MG_TX + x;
      sf = h2 * fma(4.0, c[MG_TX], c[0] + c[2 * MG_TX]);
    } else if (cd || (a.box && i <= n && j <= n && (i == 0 || j == 0 || i == n || j == n))) {
      // (a strong box node: f and g there still enter the load of its
      // neighbours through M and G)
      for (int k = 0; k < 4; ++k) {
        const int dx = k & 1, dy = k >> 1;
        const int ic = i - 1 + dx, jc = j - 1 + dy;
        if (ic < 0 || jc < 0 || ic >= n || jc >= n) continue;
        const size_t c = (size_t)jc * n + ic;
        const uint8_t cl = a.cls[c];
        if (cl == CELL_EXT) continue;
        const int av = (1 - dx) + 2 * (1 - dy);
        const double* wv = sw + (y + dy) * RHS_X + (x + dx);
        const double wb[4] = {wv[0], wv[1], wv[RHS_X], wv[RHS_X + 1]};
        if (cl == CELL_INT) {
          for (int b = 0; b < 4; ++b) {
            int wgt = (b == av) ? 4 : ((b ^ av) == 3 ? 1 : 2);
            sf += h2 * wgt * wb[b];
          }
        } else {
          const double* Mk = a.Mk + (size_t)a.cell_cut[c] * 16;
          const double* Gk = a.Gk + (size_t)a.cell_cut[c] * 16;
          for (int b = 0; b < 4; ++b) {
            sf += Mk[b * 4 + av] * wb[b];
            sg += Gk[b * 4 + av] * wb[b];
          }
          if (dLdn && a.Nk) {
            const double* Nk = a.Nk + (size_t)a.cell_cut[c] * 16;
            for (int b = 0; b < 4; ++b) sn += Nk[b * 4 + av] * wb[b];
          }
        }
      }
    }
    if (a.box && !cd && (i == 0 || j == 0 || i == n || j == n) && i <= n && j <= n) {
      // a strong Dirichlet box node: g_q enters F as - A_pq g_q, so its
      // gradient is - sum over the adjacent cells of A_K(p, q) w_p
      for (int k = 0; k < 4; ++k) {
        const int dx = k & 1, dy = k >> 1;
        const int ic = i - 1 + dx, jc = j - 1 + dy;
        if (ic < 0 || jc < 0 || ic >= n || jc >= n) continue;
        const size_t c = (size_t)jc * n + ic;
        const uint8_t cl = a.cls[c];
        if (cl == CELL_EXT) continue;
        const int av = (1 - dx) + 2 * (1 - dy);
        const double* wv = sw + (y + dy) * RHS_X + (x + dx);
        const double wb[4] = {wv[0], wv[1], wv[RHS_X], wv[RHS_X + 1]};
        for (int b = 0; b < 4; ++b) {
          const int bi = ic + (b & 1), bj = jc + (b >> 1);
          if (bi == 0 || bj == 0 || bi == n || bj == n) continue;     // box nodes: w = 0
          const double e = cl == CELL_INT
                               ? ((b == av) ? 4.0 / 6.0 : ((b ^ av) == 3 ? -2.0 / 6.0 : -1.0 / 6.0))
                               : a.Ke[(size_t)a.cell_cut[c] * 16 + b * 4 + av];
          sg -= e * wb[b];
        }
      }
    }
    if (dLdf) dLdf[gk] = sf;
    if (dLdg) dLdg[gk] = sg;
    if (dLdn) dLdn[gk] = sn;
  }
}

// User layout (row-major (n+1)^2) -> padded layout, zero on nodes that are
// not DOFs; flags NaN/Inf in a DOF entry (err) and any nonzero DOF value
// (nz).  One block per node row (blockIdx.x = j), kIoUnroll nodes of a
// thread in flight; the checks are integer tests on the bit patterns (no
// fp64 instructions) and one atomic per block at most.
constexpr int kIoUnroll = 4;
template <class T>
__global__ void __launch_bounds__(kThreads)
k_pack(Layout L, const uint16_t* __restrict__ code, const double* __restrict__ src,
       T* __restrict__ dst, unsigned* err, unsigned* nz) {
  const int n = L.n, j = blockIdx.x;
  const size_t row = L.idx(0, j);
  const double* s = src + (size_t)j * (n + 1);
  bool bad = false, any = false;
  for (int i0 = threadIdx.x; i0 <= n; i0 += kIoUnroll * blockDim.x) {
    uint16_t cd[kIoUnroll];
    double v[kIoUnroll];
#pragma unroll
    for (int k = 0; k < kIoUnroll; ++k) {
      const int i = i0 + k * (int)blockDim.x;
      cd[k] = i <= n ? code[row + i] : 0;
    }
    // entries off the DOFs are neither read nor checked
#pragma unroll
    for (int k = 0; k < kIoUnroll; ++k) v[k] = cd[k] ? s[i0 + k * (int)blockDim.x] : 0.0;
#pragma unroll
    for (int k = 0; k < kIoUnroll; ++k) {
      const int i = i0 + k * (int)blockDim.x;
      if (i > n) continue;
      bad |= !finite_bits(v[k]);
      any |= abs_bits(v[k]) != 0ull;
      dst[row + i] = (T)v[k];
    }
  }
  bad = __syncthreads_or(bad);
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    if (err && bad) atomicOr(err, DEV_ERR_NAN);
    if (nz && any) atomicOr(nz, 1u);
  }
}

// Padded layout -> user layout, zero on nodes that are not DOFs (box: the
// box-side nodes are kept as well).  One block per node row.
__global__ void __launch_bounds__(kThreads)
k_unpack(Layout L, const uint16_t* __restrict__ code, const double* __restrict__ src,
         double* __restrict__ dst, int box) {
  const int n = L.n, j = blockIdx.x;
  const size_t row = L.idx(0, j);
  double* d = dst + (size_t)j * (n + 1);
  const bool edge_row = box && (j == 0 || j == n);
  for (int i0 = threadIdx.x; i0 <= n; i0 += kIoUnroll * blockDim.x) {
    bool keep[kIoUnroll];
#pragma unroll
    for (int k = 0; k < kIoUnroll; ++k) {
      const int i = i0 + k * (int)blockDim.x;
      keep[k] = i <= n && (code[row + i] || edge_row || (box && (i == 0 || i == n)));
    }
    double v[kIoUnroll];
#pragma unroll
    for (int k = 0; k < kIoUnroll; ++k) v[k] = keep[k] ? src[row + i0 + k * (int)blockDim.x] : 0.0;
#pragma unroll
    for (int k = 0; k < kIoUnroll; ++k) {
      const int i = i0 + k * (int)blockDim.x;
      if (i <= n) d[i] = v[k];
    }
  }
}

// k_unpack restricted to the listed tiles (64 x 32 nodes each, clipped to
// the grid): the nodes of tiles without DOFs are written by k_zero_inactive.
__global__ void k_unpack_tiles(Layout L, const uint16_t* __restrict__ code,
                               const int* __restrict__ tiles, const double* __restrict__ src,
                               double* __restrict__ dst, int box) {
  const int n = L.n, t = tiles[blockIdx.x];
  const int i0 = (t % L.ntx) * MG_TX, j0 = (t / L.ntx) * MG_TY;
  for (int q = threadIdx.x; q < MG_TX * MG_TY; q += blockDim.x) {
    const int i = i0 + (q % MG_TX), j = j0 + q / MG_TX;
    if (i > n || j > n) continue;
    const size_t g = L.idx(i, j);
    const bool keep = code[g] || (box && (i == 0 || j == 0 || i == n || j == n));
    dst[(size_t)j * (n + 1) + i] = keep ? src[g] : 0.0;
  }
}

// Zero in the user layout the nodes of every tile that holds no DOF; a few
// blocks stride over the tiles, so it can run beside the solve.
__global__ void k_zero_inactive(Layout L, const uint8_t* __restrict__ tile_active,
                                double* __restrict__ dst) {
  const int n = L.n, ntiles = L.ntx * L.nty;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    if (tile_active[t]) continue;
    const int i0 = (t % L.ntx) * MG_TX, j0 = (t / L.ntx) * MG_TY;
    for (int q = threadIdx.x; q < MG_TX * MG_TY; q += blockDim.x) {
      const int i = i0 + (q % MG_TX), j = j0 + q / MG_TX;
      if (i <= n && j <= n) dst[(size_t)j * (n + 1) + i] = 0.0;
    }
  }
}

// dst = (float)(src * scale) over the tiles (both padded layouts)
__global__ void k_scale_to_f32(Layout L, const int* __restrict__ tiles,
                               const double* __restrict__ src, float* __restrict__ dst,
                               double scale) {
  griddep_launch_next();
  griddep_wait();
  const int t = tiles[blockIdx.x];
  const int i0 = (t % L.ntx) * MG_TX, j0 = (t / L.ntx) * MG_TY;
  for (int rr = threadIdx.x >> 5; rr < MG_TY; rr += blockDim.x >> 5) {
    const size_t g = L.idx(i0, j0 + rr);
    const int ii = 2 * (threadIdx.x & 31);
    const double2 v = *reinterpret_cast<const double2*>(src + g + ii);
    float2 o;
    // scale is a power of two: exact in fp32 after the rounding
    o.x = (float)v.x * (float)scale;
    o.y = (float)v.y * (float)scale;
    *reinterpret_cast<float2*>(dst + g + ii) = o;
  }
}

__global__ void k_update(Layout L, const int* __restrict__ tiles, const uint16_t* __restrict__ code,
                         double* __restrict__ u, const float* __restrict__ e, double inv_scale) {
  griddep_launch_next();
  griddep_wait();
  const int t = tiles[blockIdx.x];
  const int i0 = (t % L.ntx) * MG_TX, j0 = (t / L.ntx) * MG_TY;
  for (int it = threadIdx.x; it < MG_TY * MG_TX; it += blockDim.x) {
    int rr = it / MG_TX, ii = it - rr * MG_TX;
    size_t g = L.idx(i0 + ii, j0 + rr);
    if (code[g]) u[g] += (double)e[g] * inv_scale;
  }
}

template <class T>
__global__ void k_export_stencil(OpArgs<T> op, double* __restrict__ out) {
  const int n = op.L.n;
  const size_t m = (size_t)(n + 1) * (n + 1);
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m;
       k += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(k % (n + 1)), j = (int)(k / (n + 1));
    uint16_t cd = op.code[op.L.idx(i, j)];
    double* o = out + k * 9;
    for (int s = 0; s < 9; ++s) o[s] = 0.0;
    if (cd == 1) {
      for (int s = 0; s < 9; ++s) o[s] = -1.0 / 3.0;
      o[4] = 8.0 / 3.0;
    } else if (cd >= 2) {
      const T* R = row_of(op, i, j, cd);
      for (int s = 0; s < 9; ++s) o[s] = (double)R[s];
    }
  }
}

inline int grid_for(size_t m, int threads = kThreads) {
  size_t b = (m + threads - 1) / threads;
  return (int)(b < 65536 * 8 ? (b ? b : 1) : 65536 * 8);
}

}  // namespace

// ------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------

template <class T>
size_t sweep_smem() { return 4 * SW_PLANE * (2 * sizeof(T) + sizeof(uint16_t)); }

template <class T>
size_t band_smem(int eta) {
  const int RB = band_region(eta), RS = tma_box_w(RB), EC = BandCap<T>::value;
  return kSmemSlack + band_a128((size_t)RS * RB * sizeof(T)) + (size_t)kBandNS * EC * sizeof(T) +
         (size_t)EC * sizeof(int);
}

int band_box_x(int eta) { return tma_box_w(band_region(eta)); }
int band_box_y(int eta) { return band_region(eta); }

template <class T>
cudaError_t configure_kernels(int eta) {
  cudaError_t e;
  e = cudaFuncSetAttribute(k_gs_sweep<T, kSweepPlain>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sweep_smem<T>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_gs_sweep<T, kSweepZero>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sweep_smem<T>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_gs_sweep<T, kSweepProlong>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sweep_smem<T>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_gs_sweep<T, kSweepPlain, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sweep_smem<T>());
  if (e != cudaSuccess) return e;
  // the largest eta allowed by the ABI, so handles with different eta coexist
  (void)eta;
  e = raise_smem_limit(k_band<T>, (int)band_smem<T>(8));
  if (e != cudaSuccess) return e;
  e = raise_smem_limit(k_band<T, true>, (int)band_smem<T>(8));
  return e;
}

template <class T>
void launch_gs_sweep(const OpArgs<T>& op, const int* tiles, int ntiles, const T* uin, T* uout,
                     const T* F, T* bval, bool zero_in, const Layout* Lc, const T* ec,
                     cudaStream_t st) {
  if (!ntiles) return;
  const Layout L0 = Lc ? *Lc : op.L;
  if (ec)
    launch_pdl(k_gs_sweep<T, kSweepProlong>, ntiles, kThreads, sweep_smem<T>(), st, op, tiles, uin,
               uout, F, bval, L0, ec);
  else if (zero_in)
    launch_pdl(k_gs_sweep<T, kSweepZero>, ntiles, kThreads, sweep_smem<T>(), st, op, tiles, uin,
               uout, F, bval, L0, ec);
  else
    launch_pdl(k_gs_sweep<T, kSweepPlain>, ntiles, kThreads, sweep_smem<T>(), st, op, tiles, uin,
               uout, F, bval, L0, ec);
}

template <class T>
void launch_gs_sweep_rev(const OpArgs<T>& op, const int* tiles, int ntiles, const T* uin,
                         T* uout, const T* F, T* bval, cudaStream_t st) {
  if (!ntiles) return;
  launch_pdl(k_gs_sweep<T, kSweepPlain, true>, ntiles, kThreads, sweep_smem<T>(), st, op, tiles,
             uin, uout, F, bval, op.L, (const T*)nullptr);
}

template <class T>
void launch_gather_bval(const Layout& L, const int* bnode, int nb, const T* u, T* bval,
                        cudaStream_t st) {
  if (!nb) return;
  launch_pdl(k_gather_bval<T>, (nb + kThreads - 1) / kThreads, kThreads, 0, st, L, bnode, nb, u,
             bval);
}

template <class T>
void launch_band_rev(const OpArgs<T>& op, const int* btiles, int nbt, int nbx, int eta, T* u,
                     const T* F, const T* bval, const int* boff, const int2* bent,
                     const BandMaps& maps, int umap, unsigned* err, unsigned wait_polls,
                     cudaStream_t st) {
  if (!nbt || eta <= 0) return;
  launch_pdl(k_band<T, true>, nbt, kBandThreads, band_smem<T>(eta), st, op, btiles, nbx, eta, u, F,
             bval, boff, bent, maps, umap, err, wait_polls);
}

template <class T>
void launch_band(const OpArgs<T>& op, const int* btiles, int nbt, int nbx, int eta, T* u,
                 const T* F, const T* bval, const int* boff, const int2* bent,
                 const BandMaps& maps, int umap, unsigned* err, unsigned wait_polls,
                 cudaStream_t st) {
  if (!nbt || eta <= 0) return;
  launch_pdl(k_band<T>, nbt, kBandThreads, band_smem<T>(eta), st, op, btiles, nbx, eta, u, F, bval,
             boff, bent, maps, umap, err, wait_polls);
}

template <class T>
void launch_resid_restrict(const OpArgs<T>& op, const T* u, const T* F, const Layout& Lc,
                           const int* ctiles, int nct, T* Fc, double* norms, cudaStream_t st,
                           const uint8_t* touch) {
  if (!nct) return;
  if constexpr (sizeof(T) == sizeof(float)) {
    launch_resid_restrict_f32(op, u, F, Lc, ctiles, nct, Fc, norms, st, touch);
    return;
  }
  if (norms)
    launch_pdl(k_resid_restrict<T, true>, nct * 4, kThreads, 0, st, op, u, F, Lc, ctiles, Fc, norms,
               touch);
  else
    launch_pdl(k_resid_restrict<T, false>, nct * 4, kThreads, 0, st, op, u, F, Lc, ctiles, Fc,
               norms, touch);
}

void launch_touch_flags(int mode, const Layout& L, const uint16_t* code, const int* tiles,
                        int tpr, int nblocks, uint8_t* flag, cudaStream_t st) {
  if (nblocks > 0) k_touch_flags<<<nblocks, kThreads, 0, st>>>(mode, L, code, tiles, tpr, flag);
}

template <class T, class TR>
void launch_residual(const OpArgs<T>& op, const int* tiles, int ntiles, const T* u, const T* F,
                     TR* rout, T scale, double* norms, cudaStream_t st, bool l2,
                     double* part) {
  if (!ntiles) return;
  if (!(norms && l2)) part = nullptr;
  launch_pdl(k_residual<T, TR>, ntiles, kThreads, 0, st, op, tiles, u, F, rout, scale, norms,
             (int)l2, part);
  if (part) launch_pdl(k_sum_partials, 1, kThreads, 0, st, (const double*)part, ntiles, norms);
}

template <class T>
void launch_prolong(const OpArgs<T>& op, const int* tiles, int ntiles, T* uf, const Layout& Lc,
                    const T* ec, cudaStream_t st) {
  if (!ntiles) return;
  launch_pdl(k_prolong<T>, ntiles, kThreads, 0, st, op, tiles, uf, Lc, ec);
}

template <class T>
void launch_coarse_solve(const Layout& Lc, const double* Ainv, const T* Fc, T* uc, cudaStream_t st) {
  int m = (Lc.n + 1) * (Lc.n + 1);
  launch_pdl(k_coarse_solve<T>, 1, kThreads, m * sizeof(double), st, Lc, Ainv, Fc, uc);
}

void launch_rhs(const RhsArgs& a, const int* tiles, int ntiles, const double* f, const double* g,
                double* F, double* norms, cudaStream_t st) {
  if (!ntiles) return;
  k_rhs<<<ntiles, kThreads, 0, st>>>(a, tiles, f, g, F, norms);
}

void launch_rhs_adj(const RhsArgs& a, const int* tiles, int ntiles, const double* w,
                    double* dLdf, double* dLdg, cudaStream_t st, double* dLdn) {
  if (!ntiles) return;
  k_rhs_adj<<<ntiles, kThreads, 0, st>>>(a, tiles, w, dLdf, dLdg, dLdn);
}

template <class T>
void launch_pack(const Layout& L, const uint16_t* code, const double* src, T* dst, unsigned* err,
                 cudaStream_t st, unsigned* nz) {
  k_pack<T><<<L.n + 1, kThreads, 0, st>>>(L, code, src, dst, err, nz);
}

void launch_unpack(const Layout& L, const uint16_t* code, const double* src, double* dst,
                   cudaStream_t st, int box) {
  k_unpack<<<L.n + 1, kThreads, 0, st>>>(L, code, src, dst, box);
}

void launch_unpack_tiles(const Layout& L, const uint16_t* code, const int* tiles, int ntiles,
                         const double* src, double* dst, cudaStream_t st, int box) {
  if (ntiles) k_unpack_tiles<<<ntiles, kThreads, 0, st>>>(L, code, tiles, src, dst, box);
}

void launch_zero_inactive(const Layout& L, const uint8_t* tile_active, double* dst, int blocks,
                          cudaStream_t st) {
  k_zero_inactive<<<blocks, kThreads, 0, st>>>(L, tile_active, dst);
}

void launch_update(const Layout& L, const int* tiles, int ntiles, const uint16_t* code, double* u,
                   const float* e, double inv_scale, cudaStream_t st) {
  if (!ntiles) return;
  launch_pdl(k_update, ntiles, kThreads, 0, st, L, tiles, code, u, e, inv_scale);
}

void launch_scale_to_f32(const Layout& L, const int* tiles, int ntiles, const double* src,
                         float* dst, double scale, cudaStream_t st) {
  if (!ntiles) return;
  launch_pdl(k_scale_to_f32, ntiles, kThreads, 0, st, L, tiles, src, dst, scale);
}

template <class T>
void launch_export_stencil(const OpArgs<T>& op, double* out, cudaStream_t st) {
  size_t m = (size_t)(op.L.n + 1) * (op.L.n + 1);
  k_export_stencil<T><<<grid_for(m), kThreads, 0, st>>>(op, out);
}

#define MG_INSTANTIATE(T)                                                                        \
  template size_t sweep_smem<T>();                                                               \
  template size_t band_smem<T>(int);                                                             \
  template cudaError_t configure_kernels<T>(int);                                                \
  template void launch_gs_sweep<T>(const OpArgs<T>&, const int*, int, const T*, T*, const T*, T*, \
                                   bool, const Layout*, const T*, cudaStream_t);                 \
  template void launch_band<T>(const OpArgs<T>&, const int*, int, int, int, T*, const T*,        \
                               const T*, const int*, const int2*, const BandMaps&, int,          \
                               unsigned*, unsigned, cudaStream_t);                               \
  template void launch_resid_restrict<T>(const OpArgs<T>&, const T*, const T*, const Layout&,    \
                                         const int*, int, T*, double*, cudaStream_t,             \
                                         const uint8_t*);                                        \
  template void launch_prolong<T>(const OpArgs<T>&, const int*, int, T*, const Layout&, const T*, \
                                  cudaStream_t);                                                 \
  template void launch_coarse_solve<T>(const Layout&, const double*, const T*, T*, cudaStream_t); \
  template void launch_pack<T>(const Layout&, const uint16_t*, const double*, T*, unsigned*,     \
                               cudaStream_t, unsigned*);                                         \
  template void launch_export_stencil<T>(const OpArgs<T>&, double*, cudaStream_t);

MG_INSTANTIATE(double)
MG_INSTANTIATE(float)
template void launch_gs_sweep_rev<double>(const OpArgs<double>&, const int*, int, const double*,
                                          double*, const double*, double*, cudaStream_t);
template void launch_gather_bval<double>(const Layout&, const int*, int, const double*, double*,
                                         cudaStream_t);
template void launch_band_rev<double>(const OpArgs<double>&, const int*, int, int, int, double*,
                                      const double*, const double*, const int*, const int2*,
                                      const BandMaps&, int, unsigned*, unsigned, cudaStream_t);
template void launch_residual<double, float>(const OpArgs<double>&, const int*, int, const double*,
                                             const double*, float*, double, double*, cudaStream_t,
                                             bool, double*);
template void launch_residual<double, double>(const OpArgs<double>&, const int*, int,
                                              const double*, const double*, double*, double,
                                              double*, cudaStream_t, bool, double*);

// binds the bounds-checked build's device error word (see common.cuh)
MG_BOUNDS_BINDER(bind_bounds_cycle)
