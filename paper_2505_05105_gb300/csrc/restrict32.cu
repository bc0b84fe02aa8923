// The fp32 residual + restriction of the levels that run the separate
// kernels, written for instruction economy (the generic k_resid_restrict
// spends most of its time issuing instructions).
//
// For a 32 x 16 block of coarse nodes (I0 .. I0+31, J0 .. J0+15) it computes
// r = F - A u (Sec. 4.1) on the fine nodes the restriction reads, 2 I - 1 ..
// 2 I + 1 around each coarse node, and F_2h = P^T r with the bilinear weights
// (1, 1/2, 1/4) of Sec. 5.1.  Compared with the generic kernel:
//   * u, F and the codes of the fine region arrive with 16-byte loads (the
//     region starts 4 nodes left of 2 I0, a multiple of 4),
//   * two neighbouring fine nodes per thread: 8-byte shared loads and paired
//     fp32 arithmetic (add/fma .f32x2, each lane an ordinary IEEE fp32
//     operation), boundary rows (cut-cell vertices) node by node,
//   * r replaces F in shared memory, and a thread walks fixed columns of the
//     region (no division per node).
#include "cycle.cuh"

namespace {

constexpr int kT = 256;
constexpr int RX = 72;                   // fine columns 2 I0 - 4 .. 2 I0 + 67
constexpr int RY = 36;                   // fine rows    2 J0 - 2 .. 2 J0 + 33
constexpr int QX = RX / 4;               // 16-byte groups per row
constexpr int kLoadIt = (RY * QX + kT - 1) / kT;
constexpr int kPairs = 33;               // pairs per row: columns 2 .. 67
constexpr int kRowLanes = kT / kPairs;   // 7 rows of pairs per pass

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
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(as_u64(a)), "l"(as_u64(b)), "l"(as_u64(c)));
  return as_f2(r);
}
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// residual of a boundary node (code cd >= 2) from its 9 stencil values
__device__ __forceinline__ float boundary_residual(const OpArgs<float>& op, int gi, int gj, int cd,
                                                   float f, float sw, float s, float se, float w,
                                                   float uc, float e, float nw, float n,
                                                   float ne) {
  int t = op.L.tile_of(gi, gj);
  if (!MG_CHECKED(t >= 0 && t < op.L.ntx * op.L.nty)) t = 0;
  const float* R = op.rows + (size_t)checked_row(op.tile_base[t] + cd - 2, op.n_rows) * MG_ROW;
  const float acc = R[0] * sw + R[1] * s + R[2] * se + R[3] * w + R[4] * uc + R[5] * e +
                    R[6] * nw + R[7] * n + R[8] * ne;
  return f - acc;
}

template <bool NORM>
__global__ void __launch_bounds__(kT)
k_resid_restrict_f32(OpArgs<float> op, const float* __restrict__ u, const float* __restrict__ F,
                     Layout Lc, const int* __restrict__ ctiles, float* __restrict__ Fc,
                     double* __restrict__ norms, const uint8_t* __restrict__ touch) {
  griddep_launch_next();
  if (!band_independent(touch)) griddep_wait();
  __shared__ __align__(16) float sU[RY * RX];
  __shared__ __align__(16) float sF[RY * RX];        // F, then r in place
  __shared__ __align__(16) uint16_t sC[RY * RX];
  const int t = ctiles[blockIdx.x >> 2], sub = blockIdx.x & 3;
  const int I0 = (t % Lc.ntx) * MG_TX + (sub & 1) * 32;
  const int J0 = (t / Lc.ntx) * MG_TY + (sub >> 1) * 16;
  if (I0 > Lc.n || J0 > Lc.n) return;
  const int x0 = 2 * I0 - 4, y0 = 2 * J0 - 2;
  // 1. the region, 4 nodes per 16-byte load
  {
    float4 u4[kLoadIt], f4[kLoadIt];
    uint2 c4[kLoadIt];
#pragma unroll
    for (int k = 0; k < kLoadIt; ++k) {
      const int it = threadIdx.x + k * kT;
      const int ry = it / QX, q = it - ry * QX;
      const size_t g = it < RY * QX ? op.L.idx(x0 + 4 * q, y0 + ry) : op.L.idx(0, 0);
      u4[k] = __ldcg(reinterpret_cast<const float4*>(u + g));
      f4[k] = __ldcg(reinterpret_cast<const float4*>(F + g));
      c4[k] = *reinterpret_cast<const uint2*>(op.code + g);
    }
#pragma unroll
    for (int k = 0; k < kLoadIt; ++k) {
      const int it = threadIdx.x + k * kT;
      if (it >= RY * QX) continue;
      const int ry = it / QX, q = it - ry * QX;
      *reinterpret_cast<float4*>(sU + ry * RX + 4 * q) = u4[k];
      *reinterpret_cast<float4*>(sF + ry * RX + 4 * q) = f4[k];
      *reinterpret_cast<uint2*>(sC + ry * RX + 4 * q) = c4[k];
    }
  }
  __syncthreads();
  // 2. r on fine rows 2 J0 - 1 .. 2 J0 + 31 (region rows 1 .. 33), columns
  //    2 I0 - 2 .. 2 I0 + 63 (region columns 2 .. 67) in pairs
  unsigned long long vmax = 0ull;
  double vsum = 0.0;
  const int tc = threadIdx.x % kPairs, tr = threadIdx.x / kPairs;
  if (tr < kRowLanes) {
    const int c = 2 + 2 * tc;
    for (int ry = 1 + tr; ry <= 33; ry += kRowLanes) {
      const float* up = sU + (ry - 1) * RX;
      const float* md = sU + ry * RX;
      const float* dn = sU + (ry + 1) * RX;
      const uint32_t cc = *reinterpret_cast<const uint32_t*>(sC + ry * RX + c);
      float2* fr = reinterpret_cast<float2*>(sF + ry * RX + c);
      const float2 f = *fr;
      if (cc == 0u) {
        *fr = make_float2(0.f, 0.f);
        continue;
      }
      const float2 m = *reinterpret_cast<const float2*>(md + c);
      const float2 sm = *reinterpret_cast<const float2*>(up + c);
      const float2 nm = *reinterpret_cast<const float2*>(dn + c);
      const float ml = md[c - 1], mr = md[c + 2];
      const float sl = up[c - 1], sr = up[c + 2];
      const float nl = dn[c - 1], nr = dn[c + 2];
      const float2 W = make_float2(ml, m.x), E = make_float2(m.y, mr);
      const float2 SW = make_float2(sl, sm.x), SE = make_float2(sm.y, sr);
      const float2 NW = make_float2(nl, nm.x), NE = make_float2(nm.y, nr);
      // interior rows: r = F - (8 u - s8) / 3, s8 the 8 neighbours summed as
      // ((W + E) + (S + N)) + ((SW + SE) + (NW + NE))
      const float2 s8 = add2(add2(add2(W, E), add2(sm, nm)), add2(add2(SW, SE), add2(NW, NE)));
      const float2 d = fma2(make_float2(8.f, 8.f), m, neg2(s8));
      const float2 ri = fma2(neg2(d), make_float2(1.f / 3.f, 1.f / 3.f), f);
      const uint32_t c0 = cc & 0xffffu, c1 = cc >> 16;
      const int gj = y0 + ry, gi = x0 + c;
      float r0 = 0.f, r1 = 0.f;
      if (c0 == 1u) r0 = ri.x;
      else if (c0 >= 2u)
        r0 = boundary_residual(op, gi, gj, (int)c0, f.x, SW.x, sm.x, SE.x, W.x, m.x, E.x, NW.x,
                               nm.x, NE.x);
      if (c1 == 1u) r1 = ri.y;
      else if (c1 >= 2u)
        r1 = boundary_residual(op, gi + 1, gj, (int)c1, f.y, SW.y, sm.y, SE.y, W.y, m.y, E.y,
                               NW.y, nm.y, NE.y);
      *fr = make_float2(r0, r1);
      // owned fine nodes: columns 4 .. 67, rows 2 .. 33
      if (NORM && c >= 4 && ry >= 2) {
        max_abs(vmax, (double)r0);
        max_abs(vmax, (double)r1);
        vsum += (double)r0 * (double)r0 + (double)r1 * (double)r1;
      }
    }
  }
  __syncthreads();
  // 3. F_2h = P^T r for the 32 x 16 coarse nodes
  for (int it = threadIdx.x; it < 32 * 16; it += kT) {
    const int cy = it >> 5, cx = it & 31;
    const int I = I0 + cx, J = J0 + cy;
    if (I > Lc.n || J > Lc.n) continue;
    const float* R = sF + (2 * cy + 2) * RX + (2 * cx + 4);
    const float rc = R[0] + 0.5f * ((R[-1] + R[1]) + (R[-RX] + R[RX])) +
                     0.25f * ((R[-RX - 1] + R[-RX + 1]) + (R[RX - 1] + R[RX + 1]));
    Fc[Lc.idx(I, J)] = rc;
  }
  if (NORM) block_norms_to_global(vmax, vsum, norms);
}

}  // namespace

void launch_resid_restrict_f32(const OpArgs<float>& op, const float* u, const float* F,
                               const Layout& Lc, const int* ctiles, int nct, float* Fc,
                               double* norms, cudaStream_t st, const uint8_t* touch) {
  if (!nct) return;
  if (norms)
    launch_pdl(k_resid_restrict_f32<true>, nct * 4, kT, 0, st, op, u, F, Lc, ctiles, Fc, norms,
               touch);
  else
    launch_pdl(k_resid_restrict_f32<false>, nct * 4, kT, 0, st, op, u, F, Lc, ctiles, Fc, norms,
               touch);
}

// binds the bounds-checked build's device error word (see common.cuh)
MG_BOUNDS_BINDER(bind_bounds_restrict32)
