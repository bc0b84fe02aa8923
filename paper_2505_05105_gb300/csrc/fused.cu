// One whole smoothing step per kernel on the intermediate levels.
//
// Between the fine level (bandwidth bound, separate kernels) and the tail
// block (n <= 64) the levels are small enough that launch and phase latency
// dominate.  k_smooth_step does one smoothing step -- a 4-colour Gauss-Seidel
// sweep (Sec. 4.1) followed by eta colour sweeps over the cut-cell vertices
// (Sec. 5.3) -- for one 64 x 32 tile, redundantly on a halo of
// HS = 4 (eta + 2) >= 4 eta + 7 nodes: after 4 + 4 eta colour phases a stale
// halo value can have spread at most 4 + 4 eta nodes inwards, so the owned
// tile and two more rings are exact (the extra node keeps the region 16-byte
// aligned).  Optionally it
//   * starts from u = 0 (first smoothing step on a coarse level),
//   * adds the prolongated correction P e_2h while loading u (Sec. 5.1), and
//   * computes r = F - A u on the owned nodes plus one ring and restricts it,
//     F_2h = P^T r, for the 32 x 16 coarse block the tile covers.
// This replaces 8 launches per level (3 sweeps, 3 band sweeps, restriction,
// prolongation) by 3.
//
// The region is held as four parity planes, one per colour, so a colour's
// nodes and each class of their neighbours are contiguous: the full phases
// update two neighbouring nodes per thread with 8-byte shared loads and
// paired fp32 arithmetic (each lane an ordinary IEEE fp32 operation), and a
// band node's 9 stencil neighbours sit at offsets fixed per colour.  The
// region arrives with 16-byte loads straight into the planes (prolongation
// applied on the way); the boundary nodes (cut-cell vertices) of the region
// come from a list built at setup, grouped by colour, with their rows staged
// in shared memory before the wait for the previous kernel.
#include "fused.cuh"

namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr size_t kSlack = 128;        // the dynamic shared base is rounded up to 128 bytes

__host__ __device__ inline int halo_of(int eta) { return 4 * (eta + 2); }
__host__ __device__ inline int region_x(int eta) { return MG_TX + 2 * halo_of(eta); }
__host__ __device__ inline int region_y(int eta) { return MG_TY + 2 * halo_of(eta); }
__host__ __device__ inline size_t a128(size_t b) { return (b + 127) & ~(size_t)127; }

// elements of the shared area used for the coarse correction (prolongation)
// and later for the restriction staging (owned tile plus one ring)
__host__ __device__ inline int e_size(int RX, int RY) {
  int a = (RX / 2 + 3) * (RY / 2 + 3), b = (MG_TX + 2) * (MG_TY + 2);
  return a > b ? a : b;
}

// listed boundary nodes whose rows are staged in shared memory (stride kRS)
constexpr int kRC = 1024;
constexpr int kRS = MG_ROW + 1;       // odd stride: conflict-free row reads
// tiles around the owned one whose boundary-row bases a region can need:
// x offsets -1..1 (HS < MG_TX), y offsets -2..2 (HS < 2 MG_TY)
constexpr int kTBX = 3, kTBY = 5;

struct Carve {
  float *sU, *sF, *sE, *sS;
  uint16_t* sC;
  int* sP;
};

__host__ __device__ inline size_t carve(unsigned char* base, int eta, Carve* c) {
  const int n4 = region_x(eta) * region_y(eta);          // 4 planes
  size_t off = 0;
  auto take = [&](size_t bytes) { unsigned char* p = base + off; off += a128(bytes); return p; };
  unsigned char* u = take((size_t)n4 * sizeof(float));
  unsigned char* f = take((size_t)n4 * sizeof(float));
  unsigned char* cd = take((size_t)n4 * sizeof(uint16_t));
  unsigned char* e = take((size_t)e_size(region_x(eta), region_y(eta)) * sizeof(float));
  unsigned char* s = take((size_t)kRC * kRS * sizeof(float));
  unsigned char* pp = take((size_t)kRC * sizeof(int));
  if (c) {
    c->sU = reinterpret_cast<float*>(u);
    c->sF = reinterpret_cast<float*>(f);
    c->sC = reinterpret_cast<uint16_t*>(cd);
    c->sE = reinterpret_cast<float*>(e);
    c->sS = reinterpret_cast<float*>(s);
    c->sP = reinterpret_cast<int*>(pp);
  }
  return off;
}

__device__ __forceinline__ unsigned long long as_u64(float2 v) {
  return *reinterpret_cast<unsigned long long*>(&v);
}
__device__ __forceinline__ float2 as_f2(unsigned long long v) {
  return *reinterpret_cast<float2*>(&v);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(as_u64(a)), "l"(as_u64(b)));
  return as_f2(r);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(as_u64(a)), "l"(as_u64(b)));
  return as_f2(r);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(as_u64(a)), "l"(as_u64(b)), "l"(as_u64(c)));
  return as_f2(r);
}

// boundary-row update u_p + (F_p - sum_s w_s u_s) w_9 of a node whose 9
// stencil values are U[off[s]]
__device__ __forceinline__ float row_update(const float* w, const float* U, const int* off,
                                            float f) {
  float acc = w[0] * U[off[0]] + w[1] * U[off[1]] + w[2] * U[off[2]] + w[3] * U[off[3]] +
              w[4] * U[off[4]] + w[5] * U[off[5]] + w[6] * U[off[6]] + w[7] * U[off[7]] +
              w[8] * U[off[8]];
  return U[off[4]] + (f - acc) * w[9];
}

template <bool ZERO_IN, bool PROLONG, bool RESTRICT>
__global__ void __launch_bounds__(kThreads)
k_smooth_step(FusedArgs<float> a) {
  griddep_launch_next();
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  unsigned char* smem_raw =
      smem_dyn + ((128u - ((uint32_t)__cvta_generic_to_shared(smem_dyn) & 127u)) & 127u);
  const int HS = halo_of(a.eta);
  const int RX = region_x(a.eta), RY = region_y(a.eta);
  const int PX = RX / 2, PY = RY / 2, PL = PX * PY;
  Carve cv;
  carve(smem_raw, a.eta, &cv);
  float* sU = cv.sU;
  float* sF = cv.sF;
  uint16_t* sC = cv.sC;
  float* sE = cv.sE;
  float* sS = cv.sS;
  int* sP = cv.sP;
  __shared__ int sTB[kTBX * kTBY];
  __shared__ int gs[6];
  const Layout& L = a.L;
  const int n = L.n;
  const int t = a.tiles[blockIdx.x];
  const int tx = t % L.ntx, ty = t / L.ntx;
  const int i0 = tx * MG_TX, j0 = ty * MG_TY;
  const int ri0 = i0 - HS, rj0 = j0 - HS;          // multiples of 4
  const int warp = threadIdx.x >> 5;
  auto row_base = [&](int gi, int gj) {
    int k = ((gj / MG_TY) - ty + 2) * kTBX + (gi / MG_TX) - tx + 1;
    if (!MG_CHECKED(k >= 0 && k < kTBX * kTBY)) k = 0;
    return sTB[k];
  };

  // static data first (row bases, lists, rows, offsets): it may overlap the
  // end of the previous kernel
  if (threadIdx.x < kTBX * kTBY) {
    int ux = tx + threadIdx.x % kTBX - 1, uy = ty + threadIdx.x / kTBX - 2;
    sTB[threadIdx.x] =
        (ux >= 0 && uy >= 0 && ux < L.ntx && uy < L.nty) ? a.tile_base[uy * L.ntx + ux] : 0;
  }
  const int e0 = a.loff[5 * t];
  if (threadIdx.x < 6) gs[threadIdx.x] = a.loff[5 * t + threadIdx.x] - e0;
  const int m = a.loff[5 * t + 4] - e0;        // colour groups only: the rim is never updated
  for (int e = threadIdx.x; e < m && e < kRC; e += blockDim.x) {
    const int2 en = a.lent[e0 + e];
    const int2 xy = region_pos(en, true, RX, RY);
    const int x = xy.x, y = xy.y;
    const float* R = a.rows + (size_t)checked_row(en.y, a.n_rows) * MG_ROW;
    float v[MG_ROW];
#pragma unroll
    for (int k = 0; k < MG_ROW; ++k) v[k] = R[k];
#pragma unroll
    for (int k = 0; k < MG_ROW; ++k) sS[e * kRS + k] = v[k];
    sP[e] = (y >> 1) * PX + (x >> 1);
  }

  // then the data of the previous kernels: u, F (and codes) of the region,
  // 4 nodes per 16-byte load straight into the planes, the coarse correction
  // added on the way.  A group of 4 nodes starts at a multiple of 4, so it
  // lies either wholly left of column 0 or starts inside the row (the
  // padded row holds zeros past n).
  griddep_wait();
  {
    const int QX = RX / 4, NI = RY * QX;
    constexpr int B = 5;
    for (int it0 = threadIdx.x; it0 < NI; it0 += B * kThreads) {
      float4 f4[B], u4[B];
      uint2 c4[B];
      float e0v[B], e1v[B], e2v[B], g0v[B], g1v[B], g2v[B];
#pragma unroll
      for (int k = 0; k < B; ++k) {
        const int it = it0 + k * kThreads;
        const int y = it / QX, q = it - y * QX;
        const int gi = ri0 + 4 * q, gj = rj0 + y;
        const bool in = it < NI && gi >= 0 && gj >= 0 && gi <= n && gj <= n;
        const size_t g = in ? L.idx(gi, gj) : 0;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        f4[k] = in ? *reinterpret_cast<const float4*>(a.F + g) : z;
        u4[k] = (in && !ZERO_IN) ? *reinterpret_cast<const float4*>(a.uin + g) : z;
        c4[k] = in ? *reinterpret_cast<const uint2*>(a.code + g) : make_uint2(0u, 0u);
        if (PROLONG) {
          // coarse nodes I .. I+2 of row J (and J+1 for odd j), I = gi / 2
          const float* E = a.ec + (in ? a.Lc.idx(gi >> 1, gj >> 1) : a.Lc.idx(0, 0));
          e0v[k] = E[0];
          e1v[k] = E[1];
          e2v[k] = E[2];
          const bool odd = gj & 1;
          g0v[k] = odd ? E[a.Lc.pitch] : 0.f;
          g1v[k] = odd ? E[a.Lc.pitch + 1] : 0.f;
          g2v[k] = odd ? E[a.Lc.pitch + 2] : 0.f;
        }
      }
#pragma unroll
      for (int k = 0; k < B; ++k) {
        const int it = it0 + k * kThreads;
        if (it >= NI) continue;
        const int y = it / QX, q = it - y * QX;
        const uint32_t c0 = c4[k].x & 0xffffu, c1 = c4[k].x >> 16;
        const uint32_t c2 = c4[k].y & 0xffffu, c3 = c4[k].y >> 16;
        float u0 = u4[k].x, u1 = u4[k].y, u2 = u4[k].z, u3 = u4[k].w;
        if (PROLONG) {
          // same association as k_prolong
          if ((rj0 + y) & 1) {
            if (c0) u0 = u0 + 0.5f * (e0v[k] + g0v[k]);
            if (c1) u1 = u1 + 0.25f * ((e0v[k] + e1v[k]) + (g0v[k] + g1v[k]));
            if (c2) u2 = u2 + 0.5f * (e1v[k] + g1v[k]);
            if (c3) u3 = u3 + 0.25f * ((e1v[k] + e2v[k]) + (g1v[k] + g2v[k]));
          } else {
            if (c0) u0 = u0 + e0v[k];
            if (c1) u1 = u1 + 0.5f * (e0v[k] + e1v[k]);
            if (c2) u2 = u2 + e1v[k];
            if (c3) u3 = u3 + 0.5f * (e1v[k] + e2v[k]);
          }
        }
        const int pe = (y & 1) * 2 * PL + (y >> 1) * PX + 2 * q;   // even-x plane
        const int po = pe + PL;                                     // odd-x plane
        *reinterpret_cast<float2*>(sU + pe) = make_float2(u0, u2);
        *reinterpret_cast<float2*>(sU + po) = make_float2(u1, u3);
        *reinterpret_cast<float2*>(sF + pe) = make_float2(f4[k].x, f4[k].z);
        *reinterpret_cast<float2*>(sF + po) = make_float2(f4[k].y, f4[k].w);
        *reinterpret_cast<uint32_t*>(sC + pe) = c0 | (c2 << 16);
        *reinterpret_cast<uint32_t*>(sC + po) = c1 | (c3 << 16);
      }
    }
  }
  __syncthreads();

  // one listed node (entry e, colour c), from shared memory when staged
  auto listed = [&](int c, int e) {
    // neighbour (dx, dy) of a node of colour c = px + 2 py: plane
    // ((py + dy) & 1) * 2 + ((px + dx) & 1), row shift (py + dy) >> 1,
    // column shift (px + dx) >> 1 (floor); s = (dx + 1) + 3 (dy + 1)
    int off[9];
#pragma unroll
    for (int s = 0; s < 9; ++s) {
      const int nx = (c & 1) + (s % 3) - 1, ny = (c >> 1) + (s / 3) - 1;
      off[s] = ((ny & 1) * 2 + (nx & 1)) * PL + (ny >> 1) * PX + (nx >> 1);
    }
    int q;
    float w[MG_ROW];
    if (e < kRC) {
      q = sP[e];
#pragma unroll
      for (int k = 0; k < MG_ROW; ++k) w[k] = sS[e * kRS + k];
    } else {
      const int2 en = a.lent[e0 + e];
      const int2 xy = region_pos(en, true, RX, RY);
      q = (xy.y >> 1) * PX + (xy.x >> 1);
      const float* R = a.rows + (size_t)checked_row(en.y, a.n_rows) * MG_ROW;
#pragma unroll
      for (int k = 0; k < MG_ROW; ++k) w[k] = R[k];
    }
    float* U = sU + q;
    U[off[4]] = row_update(w, U, off, sF[c * PL + q]);
  };

  // 4 full colour phases; a thread updates plane nodes (a, b) and (a + 1, b)
  // of the colour's plane: interior nodes by the constant stencil, the
  // colour's listed boundary nodes from their rows (same-colour nodes never
  // interact).  Every node off the region's rim is updated in every phase:
  // a node near the rim computed from stale neighbours is itself stale, and
  // staleness moves inward by one node per phase.
  {
    const int pairs = PX / 2;
    const int step = kThreads / pairs;
    const int tb = threadIdx.x / pairs, ta = 2 * (threadIdx.x - tb * pairs);
    const bool on = tb < step;
    for (int c = 0; c < 4; ++c) {
      const int ci = c & 1, cj = c >> 1;
      float* P = sU + c * PL;
      const float* PXn = sU + (c ^ 1) * PL;
      const float* PYn = sU + (c ^ 2) * PL;
      const float* PDn = sU + (c ^ 3) * PL;
      const float* PF = sF + c * PL;
      const uint16_t* PC = sC + c * PL;
      const int b0 = cj ? 0 : 1, b1 = cj ? PY - 2 : PY - 1;
      const uint32_t mask = (ta == 0 && ci == 0) ? 0xffff0000u
                            : (ta == PX - 2 && ci == 1) ? 0x0000ffffu : 0xffffffffu;
      for (int b = b0 + tb; on && b <= b1; b += step) {
        const int a2 = ta;
        const uint32_t cc = *reinterpret_cast<const uint32_t*>(PC + b * PX + a2) & mask;
        const bool in0 = (cc & 0xffffu) == 1u, in1 = (cc >> 16) == 1u;
        if (!in0 && !in1) continue;
        const int ym = b + cj - 1, yp = b + cj;
        float2 W, E, SW, SE, NW, NE;
        if (ci) {
          const float2 mm = *reinterpret_cast<const float2*>(PXn + b * PX + a2);
          const float r = PXn[b * PX + a2 + 2];
          W = mm;
          E = make_float2(mm.y, r);
          const float2 dm = *reinterpret_cast<const float2*>(PDn + ym * PX + a2);
          const float dr = PDn[ym * PX + a2 + 2];
          SW = dm;
          SE = make_float2(dm.y, dr);
          const float2 um = *reinterpret_cast<const float2*>(PDn + yp * PX + a2);
          const float ur = PDn[yp * PX + a2 + 2];
          NW = um;
          NE = make_float2(um.y, ur);
        } else {
          const float l = PXn[b * PX + a2 - 1];
          const float2 mm = *reinterpret_cast<const float2*>(PXn + b * PX + a2);
          W = make_float2(l, mm.x);
          E = mm;
          const float dl = PDn[ym * PX + a2 - 1];
          const float2 dm = *reinterpret_cast<const float2*>(PDn + ym * PX + a2);
          SW = make_float2(dl, dm.x);
          SE = dm;
          const float ul = PDn[yp * PX + a2 - 1];
          const float2 um = *reinterpret_cast<const float2*>(PDn + yp * PX + a2);
          NW = make_float2(ul, um.x);
          NE = um;
        }
        const float2 S = *reinterpret_cast<const float2*>(PYn + ym * PX + a2);
        const float2 N = *reinterpret_cast<const float2*>(PYn + yp * PX + a2);
        const float2 f = *reinterpret_cast<const float2*>(PF + b * PX + a2);
        // u_p = (3 F_p + sum of the 8 neighbours) / 8, the sum as
        // ((W + E) + (S + N)) + ((SW + SE) + (NW + NE))
        const float2 s8 = add2(add2(add2(W, E), add2(S, N)), add2(add2(SW, SE), add2(NW, NE)));
        const float2 v = mul2(fma2(make_float2(3.f, 3.f), f, s8), make_float2(0.125f, 0.125f));
        if (in0 && in1) *reinterpret_cast<float2*>(P + b * PX + a2) = v;
        else if (in0) P[b * PX + a2] = v.x;
        else P[b * PX + a2 + 1] = v.y;
      }
      // the colour's boundary nodes from the last threads, which make one
      // pass of the pairs fewer than the first ones
      for (int e = gs[c] + (int)(blockDim.x - 1 - threadIdx.x); e < gs[c + 1]; e += blockDim.x)
        listed(c, e);
      __syncthreads();
    }
  }

  // 4 eta phases on the cut-cell vertices only, on nw warps; each thread's
  // node of every colour (position, F and its row) stays in registers, and
  // the stencil offsets of a colour are computed, not loaded
  if (a.eta > 0) {
    int g[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) g[c] = gs[c];
    int mc = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) mc = max(mc, g[c + 1] - g[c]);
    const int nw = min(kWarps, max(1, (mc + 31) / 32));
    if (warp < nw) {
      const int nt = 32 * nw;
      int q[4];
      float w[4][MG_ROW], fv[4];
      bool more = false;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int e = g[c] + threadIdx.x;
        q[c] = -1;
        fv[c] = 0.f;
#pragma unroll
        for (int k = 0; k < MG_ROW; ++k) w[c][k] = 0.f;
        if (e < g[c + 1] && e < kRC) {
          q[c] = sP[e];
#pragma unroll
          for (int k = 0; k < MG_ROW; ++k) w[c][k] = sS[e * kRS + k];
          fv[c] = sF[c * PL + q[c]];
        }
        more |= g[c + 1] - g[c] > nt || g[c + 1] > kRC;
      }
      for (int it = 0; it < a.eta; ++it) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (q[c] >= 0) {
            // neighbour (dx, dy) of colour c, as in listed()
            int off[9];
#pragma unroll
            for (int s = 0; s < 9; ++s) {
              const int nx = (c & 1) + (s % 3) - 1, ny = (c >> 1) + (s / 3) - 1;
              off[s] = ((ny & 1) * 2 + (nx & 1)) * PL + (ny >> 1) * PX + (nx >> 1);
            }
            float* U = sU + q[c];
            U[off[4]] = row_update(w[c], U, off, fv[c]);
          }
          if (more)
            for (int e = g[c] + threadIdx.x; e < g[c + 1]; e += nt)
              if (e - g[c] >= nt || e >= kRC) listed(c, e);
          if (nt == 32) __syncwarp();
          else asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
        }
      }
    }
    __syncthreads();
  }

  // owned tile out: 4 nodes per 16-byte store
  for (int it = threadIdx.x; it < MG_TY * (MG_TX / 4); it += blockDim.x) {
    const int rr = it / (MG_TX / 4), q4 = it - rr * (MG_TX / 4);
    const int y = HS + rr;
    const int pe = (y & 1) * 2 * PL + (y >> 1) * PX + HS / 2 + 2 * q4, po = pe + PL;
    const float2 ve = *reinterpret_cast<const float2*>(sU + pe);
    const float2 vo = *reinterpret_cast<const float2*>(sU + po);
    *reinterpret_cast<float4*>(a.uout + L.idx(i0 + 4 * q4, j0 + rr)) =
        make_float4(ve.x, vo.x, ve.y, vo.y);
  }

  if (RESTRICT) {
    // residual on the owned nodes plus one ring, staged in sE (natural layout)
    constexpr int SX = MG_TX + 2;
    for (int it = threadIdx.x; it < (MG_TX + 2) * (MG_TY + 2); it += blockDim.x) {
      const int rr = it / SX, ii = it - rr * SX;
      const int x = HS - 1 + ii, y = HS - 1 + rr;
      const int c = (x & 1) + 2 * (y & 1);
      const int q = (y >> 1) * PX + (x >> 1);
      const uint16_t cd = sC[c * PL + q];
      float r = 0.f;
      if (cd) {
        int off[9];
#pragma unroll
        for (int s = 0; s < 9; ++s) {
          const int nx = (c & 1) + (s % 3) - 1, ny = (c >> 1) + (s / 3) - 1;
          off[s] = ((ny & 1) * 2 + (nx & 1)) * PL + (ny >> 1) * PX + (nx >> 1);
        }
        const float* U = sU + q;
        const float f = sF[c * PL + q];
        if (cd == 1) {
          float s8 = ((U[off[3]] + U[off[5]]) + (U[off[1]] + U[off[7]])) +
                     ((U[off[0]] + U[off[2]]) + (U[off[6]] + U[off[8]]));
          r = f - (8.f * U[off[4]] - s8) * (1.f / 3.f);
        } else {
          const float* R =
              a.rows + (size_t)checked_row(row_base(ri0 + x, rj0 + y) + cd - 2, a.n_rows) * MG_ROW;
          float acc = R[0] * U[off[0]] + R[1] * U[off[1]] + R[2] * U[off[2]] +
                      R[3] * U[off[3]] + R[4] * U[off[4]] + R[5] * U[off[5]] +
                      R[6] * U[off[6]] + R[7] * U[off[7]] + R[8] * U[off[8]];
          r = f - acc;
        }
      }
      sE[it] = r;
    }
    __syncthreads();
    const Layout& Lc = a.Lc;
    const int I0 = i0 / 2, J0 = j0 / 2;
    for (int it = threadIdx.x; it < (MG_TX / 2) * (MG_TY / 2); it += blockDim.x) {
      const int cy = it / (MG_TX / 2), cx = it - cy * (MG_TX / 2);
      const int I = I0 + cx, J = J0 + cy;
      if (I > Lc.n || J > Lc.n) continue;
      const float* R = sE + (2 * cy + 1) * SX + (2 * cx + 1);
      float rc = R[0] + 0.5f * ((R[-1] + R[1]) + (R[-SX] + R[SX])) +
                 0.25f * ((R[-SX - 1] + R[-SX + 1]) + (R[SX - 1] + R[SX + 1]));
      a.Fc[Lc.idx(I, J)] = rc;
    }
  }
}

}  // namespace

int fused_halo(int eta) { return halo_of(eta); }

// fp32 only (the fp64 cycle uses the separate kernels)
size_t fused_smem_bytes(int eta, size_t elem) {
  return elem == sizeof(float) ? kSlack + carve(nullptr, eta, nullptr) : ~(size_t)0;
}

template <class T>
cudaError_t configure_fused(size_t smem) {
  if (sizeof(T) != sizeof(float)) return cudaSuccess;
  cudaError_t e;
#define MG_CFG(Z, P, R)                                                                     \
  e = raise_smem_limit(k_smooth_step<Z, P, R>, smem);                                       \
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
  if constexpr (sizeof(T) != sizeof(float)) {
    (void)a; (void)ntiles; (void)zero_in; (void)prolong; (void)restrict_; (void)smem; (void)st;
  } else {
    if (!ntiles) return;
    if (zero_in && !prolong && !restrict_)
      launch_pdl(k_smooth_step<true, false, false>, ntiles, kThreads, smem, st, a);
    else if (zero_in && !prolong && restrict_)
      launch_pdl(k_smooth_step<true, false, true>, ntiles, kThreads, smem, st, a);
    else if (!zero_in && !prolong && !restrict_)
      launch_pdl(k_smooth_step<false, false, false>, ntiles, kThreads, smem, st, a);
    else if (!zero_in && !prolong && restrict_)
      launch_pdl(k_smooth_step<false, false, true>, ntiles, kThreads, smem, st, a);
    else if (!zero_in && prolong && !restrict_)
      launch_pdl(k_smooth_step<false, true, false>, ntiles, kThreads, smem, st, a);
    else
      launch_pdl(k_smooth_step<false, true, true>, ntiles, kThreads, smem, st, a);
  }
}

template cudaError_t configure_fused<float>(size_t);
template cudaError_t configure_fused<double>(size_t);
template void launch_smooth_step<float>(const FusedArgs<float>&, int, bool, bool, bool, size_t,
                                        cudaStream_t);
template void launch_smooth_step<double>(const FusedArgs<double>&, int, bool, bool, bool, size_t,
                                         cudaStream_t);

// binds the bounds-checked build's device error word (see common.cuh)
MG_BOUNDS_BINDER(bind_bounds_fused)
