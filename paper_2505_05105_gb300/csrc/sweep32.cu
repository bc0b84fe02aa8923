// The fp32 Gauss-Seidel sweep of the levels above the fused ones, written
// for instruction economy.
//
// One 4-colour sweep (Sec. 4.1, colours (i mod 2, j mod 2) in the order
// (0,0), (1,0), (0,1), (1,1)) of a 64 x 32 tile, recomputed on a 4-node halo
// (one node per colour phase) so that the owned nodes are exact.  The region
// is held as four parity planes (one per colour), so the nodes of a colour
// and each of their neighbour classes are contiguous in shared memory.  This
// kernel is the same computation as k_gs_sweep<float> with:
//   * 16-byte global loads (4 nodes of u and F, 8 bytes of codes per load)
//     and 16-byte global stores,
//   * two neighbouring nodes of a colour per thread: 8-byte shared loads
//     and paired fp32 arithmetic (add/fma/mul .f32x2, each lane an ordinary
//     IEEE fp32 operation, so results are bit for bit those of the scalar
//     code), 384 threads so that each colour phase (19 rows of 18 pairs) is
//     one pass of the block,
//   * the region's boundary rows (cut-cell vertices) staged in shared memory
//     from a setup-time list before the wait for the previous kernel, so the
//     colour phases read no global memory: the list entry of each boundary
//     node replaces its code in the code plane, and
//   * the prolongation P e_2h (Sec. 5.1) added while loading, when asked.
#include "cycle.cuh"

namespace {

constexpr int kT = 384;
constexpr int H = 4;                       // halo: one node per colour phase
constexpr int RX = MG_TX + 2 * H;          // 72
constexpr int RY = MG_TY + 2 * H;          // 40
constexpr int PX = RX / 2, PY = RY / 2;    // parity plane 36 x 20
constexpr int PL = PX * PY;
constexpr int QX = RX / 4;                 // 16-byte groups per region row (18)
constexpr int kLoadIt = (RY * QX + kT - 1) / kT;                  // 2
constexpr int kRC = 384;                   // boundary rows staged in shared memory
constexpr int kRS = MG_ROW + 1;            // odd stride: conflict-free row reads
constexpr int kStoreIt = (MG_TY * (MG_TX / 4) + kT - 1) / kT;    // 2

enum : int { kPlain = 0, kZero = 1, kProlong = 2 };

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

// Row of list entry e of the region (code 2 + e in the code plane): staged
// in shared memory for e < kRC, else from global memory.
struct RowSrc {
  const float* sRow;                       // kRC staged rows, stride kRS
  const float* rows;                       // the level's boundary rows
  const int2* ent;                         // the tile's list entries
  int n_rows;
};
__device__ __forceinline__ const float* row_ptr(const RowSrc& rs, int e) {
  return e < kRC ? rs.sRow + e * kRS
                 : rs.rows + (size_t)checked_row(rs.ent[e].y, rs.n_rows) * MG_ROW;
}

// boundary-row update of a node whose code is cd >= 2, same arithmetic as
// k_gs_sweep
__device__ __forceinline__ float boundary_update(const RowSrc& rs, int cd, float uc, float f,
                                                 float w, float e, float s, float n, float sw,
                                                 float se, float nw, float ne) {
  const float* R = row_ptr(rs, cd - 2);
  float acc = R[0] * sw + R[1] * s + R[2] * se + R[3] * w + R[4] * uc + R[5] * e +
              R[6] * nw + R[7] * n + R[8] * ne;
  return uc + (f - acc) * R[9];
}

// One colour phase (CI, CJ) = (i mod 2, j mod 2) over the parity planes: a
// thread updates plane nodes (a, b) and (a + 1, b) of row b = b0 + tb (the
// block covers all of the colour's rows in one pass).  Every node off the
// region's rim is updated in every phase: a node near the rim computed from
// stale neighbours is itself stale, and staleness still moves inward by one
// node per phase, so the owned tile is exact after the 4 phases.  The colour
// is a template argument, so plane bases and neighbour offsets are constants.
template <int CI, int CJ>
__device__ __forceinline__ void colour_phase(const RowSrc& rs, float* sU, const float* sF,
                                             const uint16_t* sC, int tb, int ta, bool lane_on) {
  float* P = sU + (CJ * 2 + CI) * PL;
  const float* PXn = sU + (CJ * 2 + (CI ^ 1)) * PL;
  const float* PYn = sU + ((CJ ^ 1) * 2 + CI) * PL;
  const float* PDn = sU + ((CJ ^ 1) * 2 + (CI ^ 1)) * PL;
  const float* PF = sF + (CJ * 2 + CI) * PL;
  const uint16_t* PC = sC + (CJ * 2 + CI) * PL;
  // rows with 1 <= 2b + cj <= RY - 2; columns: the rim node of the first or
  // last pair is masked
  constexpr int b0 = CJ ? 0 : 1, b1 = CJ ? PY - 2 : PY - 1;
  const int b = b0 + tb;
  if (!lane_on || b > b1) return;
  const int a = ta;
  const uint32_t mask = (CI == 0 && ta == 0) ? 0xffff0000u
                        : (CI == 1 && ta == PX - 2) ? 0x0000ffffu : 0xffffffffu;
  const int q = b * PX + a;                          // (a, b) in the plane
  constexpr int dm = (CJ - 1) * PX, dp = CJ * PX;    // rows ym = b + cj - 1, yp = b + cj
  const uint32_t cc = *reinterpret_cast<const uint32_t*>(PC + q) & mask;
  if (cc == 0u) return;
  // x neighbours: columns a + ci - 1 .. a + ci + 1 of the neighbour planes
  float2 W, E, SW, SE, NW, NE;
  if (CI) {
    const float2 m = *reinterpret_cast<const float2*>(PXn + q);
    const float r = PXn[q + 2];
    W = m;
    E = make_float2(m.y, r);
    const float2 dmv = *reinterpret_cast<const float2*>(PDn + q + dm);
    const float dr = PDn[q + dm + 2];
    SW = dmv;
    SE = make_float2(dmv.y, dr);
    const float2 um = *reinterpret_cast<const float2*>(PDn + q + dp);
    const float ur = PDn[q + dp + 2];
    NW = um;
    NE = make_float2(um.y, ur);
  } else {
    const float l = PXn[q - 1];
    const float2 m = *reinterpret_cast<const float2*>(PXn + q);
    W = make_float2(l, m.x);
    E = m;
    const float dl = PDn[q + dm - 1];
    const float2 dmv = *reinterpret_cast<const float2*>(PDn + q + dm);
    SW = make_float2(dl, dmv.x);
    SE = dmv;
    const float ul = PDn[q + dp - 1];
    const float2 um = *reinterpret_cast<const float2*>(PDn + q + dp);
    NW = make_float2(ul, um.x);
    NE = um;
  }
  const float2 S = *reinterpret_cast<const float2*>(PYn + q + dm);
  const float2 N = *reinterpret_cast<const float2*>(PYn + q + dp);
  const float2 f = *reinterpret_cast<const float2*>(PF + q);
  // interior rows: 8/3 u_p - 1/3 (sum of 8 neighbours) = F_p, i.e.
  // u_p = (3 F_p + sum) / 8 with the association of k_gs_sweep
  const float2 A = add2(add2(W, E), add2(S, N));
  const float2 Bd = add2(add2(SW, SE), add2(NW, NE));
  const float2 in = mul2(add2(fma2(make_float2(3.f, 3.f), f, A), Bd),
                         make_float2(0.125f, 0.125f));
  if (cc == 0x00010001u) {       // both interior: the common case
    *reinterpret_cast<float2*>(P + q) = in;
    return;
  }
  const uint32_t c0 = cc & 0xffffu, c1 = cc >> 16;
  const float2 uc = *reinterpret_cast<const float2*>(P + q);
  float r0 = uc.x, r1 = uc.y;
  if (c0 == 1u) r0 = in.x;
  else if (c0 >= 2u)
    r0 = boundary_update(rs, (int)c0, uc.x, f.x, W.x, E.x, S.x, N.x, SW.x, SE.x, NW.x, NE.x);
  if (c1 == 1u) r1 = in.y;
  else if (c1 >= 2u)
    r1 = boundary_update(rs, (int)c1, uc.y, f.y, W.y, E.y, S.y, N.y, SW.y, SE.y, NW.y, NE.y);
  *reinterpret_cast<float2*>(P + q) = make_float2(r0, r1);
}

template <int MODE>
__global__ void __launch_bounds__(kT)
k_gs_sweep_f32(OpArgs<float> op, const int* __restrict__ tiles, const float* __restrict__ uin,
               float* __restrict__ uout, const float* __restrict__ F, float* __restrict__ bval,
               Layout Lc, const float* __restrict__ ec, const int* __restrict__ loff,
               const int2* __restrict__ lent, const uint8_t* __restrict__ touch) {
  griddep_launch_next();
  __shared__ __align__(16) float sU[4 * PL];       // plane 2 (y parity) + (x parity)
  __shared__ __align__(16) float sF[4 * PL];
  __shared__ __align__(16) uint16_t sC[4 * PL];
  __shared__ float sRow[kRC * kRS];
  __shared__ int sGrow[kRC];                       // the staged entries' global rows
  const int t = tiles[blockIdx.x];
  const int i0 = (t % op.L.ntx) * MG_TX, j0 = (t / op.L.ntx) * MG_TY;
  const int ri0 = i0 - H, rj0 = j0 - H;            // both even
  const int n = op.L.n;
  // 0. static data first (it may overlap the end of the previous kernel):
  //    the region's boundary nodes (colour groups, not the rim) and their rows
  const int e0 = loff[5 * blockIdx.x];
  const int m = loff[5 * blockIdx.x + 4] - e0;
  const RowSrc rs{sRow, op.rows, lent + e0, op.n_rows};
  for (int e = threadIdx.x; e < m && e < kRC; e += kT) {
    const int2 en = lent[e0 + e];
    const float* R = op.rows + (size_t)checked_row(en.y, op.n_rows) * MG_ROW;
    float v[MG_ROW];
#pragma unroll
    for (int k = 0; k < MG_ROW; ++k) v[k] = R[k];
#pragma unroll
    for (int k = 0; k < MG_ROW; ++k) sRow[e * kRS + k] = v[k];
    sGrow[e] = checked_row(en.y, op.n_rows);
  }
  if (!band_independent(touch)) griddep_wait();

  // 1. region -> parity planes; item (rj, q) = nodes ri0 + 4q .. + 3 of row rj
  {
    float4 f4[kLoadIt], u4[kLoadIt];
    uint2 c4[kLoadIt];
    float e0[kLoadIt], e1[kLoadIt], e2[kLoadIt], g0[kLoadIt], g1[kLoadIt], g2[kLoadIt];
#pragma unroll
    for (int k = 0; k < kLoadIt; ++k) {
      const int it = threadIdx.x + k * kT;
      const bool ok = it < RY * QX;
      const int rj = it / QX, q = it - rj * QX;
      const size_t g = ok ? op.L.idx(ri0 + 4 * q, rj0 + rj) : op.L.idx(0, 0);
      f4[k] = __ldcg(reinterpret_cast<const float4*>(F + g));
      u4[k] = MODE == kZero ? make_float4(0.f, 0.f, 0.f, 0.f)
                            : __ldcg(reinterpret_cast<const float4*>(uin + g));
      c4[k] = *reinterpret_cast<const uint2*>(op.code + g);
      if (MODE == kProlong) {
        // coarse nodes I .. I+2 of row J (and J+1 for odd j), I = gi / 2
        const int gi = ri0 + 4 * q, gj = rj0 + rj;
        const bool in = ok && gi >= 0 && gj >= 0 && gi <= n && gj <= n;
        const float* E = ec + (in ? Lc.idx(gi >> 1, gj >> 1) : Lc.idx(0, 0));
        e0[k] = __ldcg(E);
        e1[k] = __ldcg(E + 1);
        e2[k] = __ldcg(E + 2);
        const bool odd = gj & 1;
        g0[k] = odd ? __ldcg(E + Lc.pitch) : 0.f;
        g1[k] = odd ? __ldcg(E + Lc.pitch + 1) : 0.f;
        g2[k] = odd ? __ldcg(E + Lc.pitch + 2) : 0.f;
      }
    }
#pragma unroll
    for (int k = 0; k < kLoadIt; ++k) {
      const int it = threadIdx.x + k * kT;
      if (it >= RY * QX) continue;
      const int rj = it / QX, q = it - rj * QX;
      const uint32_t c0 = c4[k].x & 0xffffu, c1 = c4[k].x >> 16;
      const uint32_t c2 = c4[k].y & 0xffffu, c3 = c4[k].y >> 16;
      float u0 = u4[k].x, u1 = u4[k].y, u2 = u4[k].z, u3 = u4[k].w;
      if (MODE == kProlong) {
        // same association as k_prolong
        if ((rj0 + rj) & 1) {
          if (c0) u0 = u0 + 0.5f * (e0[k] + g0[k]);
          if (c1) u1 = u1 + 0.25f * ((e0[k] + e1[k]) + (g0[k] + g1[k]));
          if (c2) u2 = u2 + 0.5f * (e1[k] + g1[k]);
          if (c3) u3 = u3 + 0.25f * ((e1[k] + e2[k]) + (g1[k] + g2[k]));
        } else {
          if (c0) u0 = u0 + e0[k];
          if (c1) u1 = u1 + 0.5f * (e0[k] + e1[k]);
          if (c2) u2 = u2 + e1[k];
          if (c3) u3 = u3 + 0.5f * (e1[k] + e2[k]);
        }
      }
      const int pe = (rj & 1) * 2 * PL + (rj >> 1) * PX + 2 * q;   // even-x plane
      const int po = pe + PL;                                       // odd-x plane
      *reinterpret_cast<float2*>(sU + pe) = make_float2(u0, u2);
      *reinterpret_cast<float2*>(sU + po) = make_float2(u1, u3);
      *reinterpret_cast<float2*>(sF + pe) = make_float2(f4[k].x, f4[k].z);
      *reinterpret_cast<float2*>(sF + po) = make_float2(f4[k].y, f4[k].w);
      *reinterpret_cast<uint32_t*>(sC + pe) = c0 | (c2 << 16);
      *reinterpret_cast<uint32_t*>(sC + po) = c1 | (c3 << 16);
    }
  }
  __syncthreads();
  // each listed boundary node's code becomes 2 + its list entry
  for (int e = threadIdx.x; e < m; e += kT) {
    const int2 xy = region_pos(lent[e0 + e], true, RX, RY);
    const int x = xy.x, y = xy.y;
    sC[(y & 1) * 2 * PL + (x & 1) * PL + (y >> 1) * PX + (x >> 1)] = (uint16_t)(2 + e);
  }
  __syncthreads();

  // 2. the four colour phases, (0,0), (1,0), (0,1), (1,1)
  constexpr int kPairCols = PX / 2;                 // 18
  constexpr int kRowStep = kT / kPairCols;          // 21 rows per pass
  static_assert(kRowStep >= PY - 1, "a colour phase must be one pass of the block");
  const int tb = threadIdx.x / kPairCols;
  const int ta = 2 * (threadIdx.x - tb * kPairCols);
  const bool lane_on = tb < kRowStep;
  colour_phase<0, 0>(rs, sU, sF, sC, tb, ta, lane_on);
  __syncthreads();
  colour_phase<1, 0>(rs, sU, sF, sC, tb, ta, lane_on);
  __syncthreads();
  colour_phase<0, 1>(rs, sU, sF, sC, tb, ta, lane_on);
  __syncthreads();
  colour_phase<1, 1>(rs, sU, sF, sC, tb, ta, lane_on);
  __syncthreads();

  // 3. owned tile out (16-byte stores), boundary values to bval (the global
  //    row of the node's list entry)
#pragma unroll
  for (int k = 0; k < kStoreIt; ++k) {
    const int it = threadIdx.x + k * kT;
    if (it >= MG_TY * (MG_TX / 4)) break;
    const int rr = it / (MG_TX / 4), q = it - rr * (MG_TX / 4);
    const int rj = H + rr;
    const int pe = (rj & 1) * 2 * PL + (rj >> 1) * PX + H / 2 + 2 * q, po = pe + PL;
    const float2 ve = *reinterpret_cast<const float2*>(sU + pe);
    const float2 vo = *reinterpret_cast<const float2*>(sU + po);
    *reinterpret_cast<float4*>(uout + op.L.idx(i0 + 4 * q, j0 + rr)) =
        make_float4(ve.x, vo.x, ve.y, vo.y);
    if (bval && m > 0) {          // m = 0: no boundary node in the tile
      const uint32_t ce = *reinterpret_cast<const uint32_t*>(sC + pe);
      const uint32_t co = *reinterpret_cast<const uint32_t*>(sC + po);
      const uint32_t c[4] = {ce & 0xffffu, co & 0xffffu, ce >> 16, co >> 16};
      const float v[4] = {ve.x, vo.x, ve.y, vo.y};
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2)
        if (c[k2] >= 2u) {
          const int e = (int)c[k2] - 2;
          bval[e < kRC ? sGrow[e] : checked_row(lent[e0 + e].y, op.n_rows)] = v[k2];
        }
    }
  }
}

}  // namespace

void launch_gs_sweep_f32(const OpArgs<float>& op, const int* tiles, int ntiles, const float* uin,
                         float* uout, const float* F, float* bval, bool zero_in,
                         const Layout* Lc, const float* ec, const int* loff, const int2* lent,
                         const uint8_t* touch, cudaStream_t st) {
  if (!ntiles) return;
  const Layout L0 = Lc ? *Lc : op.L;
  if (ec)
    launch_pdl(k_gs_sweep_f32<kProlong>, ntiles, kT, 0, st, op, tiles, uin, uout, F, bval, L0, ec,
               loff, lent, touch);
  else if (zero_in)
    launch_pdl(k_gs_sweep_f32<kZero>, ntiles, kT, 0, st, op, tiles, uin, uout, F, bval, L0, ec,
               loff, lent, (const uint8_t*)nullptr);
  else
    launch_pdl(k_gs_sweep_f32<kPlain>, ntiles, kT, 0, st, op, tiles, uin, uout, F, bval, L0, ec,
               loff, lent, touch);
}

// binds the bounds-checked build's device error word (see common.cuh)
MG_BOUNDS_BINDER(bind_bounds_sweep32)
