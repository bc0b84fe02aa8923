// F = M f + G g on one 64 x 32 node tile (Eq. disc_rhs with Q1
// interpolants), shared by the single-problem and the batched kernels.
#pragma once

#include "cycle.cuh"

namespace {

// F = M f + G g on one active tile (64 x 32 nodes).  Interior nodes (all
// four cells inside) take the whole-cell Q1 mass, whose sum over the four
// cells is the separable 9-point stencil h^2/36 [1 4 1] x [1 4 1]: a row pass
// and a column pass over f staged in shared memory (5 fp64 operations per
// node instead of 16).  Vertices of cut cells sum the cells one by one, with
// the cut cells' Mk and Gk (Eq. disc_rhs with Q1 interpolants).
constexpr int RHS_X = MG_TX + 2, RHS_Y = MG_TY + 2;
// Block-wide over tile t, one tile per block (any block size that is a
// multiple of 32); returns the thread's max |F| over the nodes it wrote (as
// the bit pattern of |F|, see abs_bits).
__device__ __forceinline__ unsigned long long rhs_tile(const RhsArgs& a, int t, const double* __restrict__ f,
                                           const double* __restrict__ g, double* __restrict__ F) {
  __shared__ double sf[RHS_Y * RHS_X];       // f on the tile plus one ring
  __shared__ double st[RHS_Y * MG_TX];       // row pass f(i-1) + 4 f(i) + f(i+1)
  const int n = a.L.n;
  const size_t W = (size_t)n + 1;
  const int i0 = (t % a.L.ntx) * MG_TX, j0 = (t / a.L.ntx) * MG_TY;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int y = warp; y < RHS_Y; y += nw) {
    const int j = j0 - 1 + y;
    double v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int x = lane + 32 * k, i = i0 - 1 + x;
      const bool in = x < RHS_X && i >= 0 && j >= 0 && i <= n && j <= n;
      v[k] = in ? f[(size_t)j * W + i] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int x = lane + 32 * k;
      if (x < RHS_X) sf[y * RHS_X + x] = v[k];
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < RHS_Y * MG_TX; q += blockDim.x) {
    const int y = q / MG_TX, x = q - y * MG_TX;
    const double* r = sf + y * RHS_X + x;
    st[q] = fma(4.0, r[1], r[0] + r[2]);
  }
  __syncthreads();
  const double h2 = a.h * a.h / 36.0;
  unsigned long long vmax = 0ull;
  // interior nodes here; vertices of cut cells (and, with box sides, nodes
  // next to the box) go to a list and are done after, a thread each, so that
  // their long fp64 path does not hold up whole warps of interior nodes
  __shared__ uint16_t s_list[MG_TX * MG_TY];
  __shared__ int s_nl;
  if (threadIdx.x == 0) s_nl = 0;
  __syncthreads();
  auto finish = [&](size_t gk, double s) {
    F[gk] = s;
    // every f, g (and g_N) value that enters F_p is in s with a weight:
    // a NaN or Inf among them (0 * Inf included) leaves s not finite
    if (a.err != nullptr && !finite_bits(s)) atomicOr(a.err, DEV_ERR_NAN);
    max_abs(vmax, s);
  };
  for (int q = threadIdx.x; q < MG_TY * MG_TX; q += blockDim.x) {
    const int y = q / MG_TX, x = q - y * MG_TX;
    const int i = i0 + x, j = j0 + y;
    const size_t gk = a.L.idx(i, j);
    const uint16_t cd = a.code[gk];
    if (cd >= 2 || (a.box && cd && (i == 1 || j == 1 || i == n - 1 || j == n - 1))) {
      s_list[atomicAdd(&s_nl, 1)] = (uint16_t)q;
      continue;
    }
    double s = 0.0;
    if (cd == 1) {
      const double* c = st + y * MG_TX + x;
      s = h2 * fma(4.0, c[MG_TX], c[0] + c[2 * MG_TX]);
    }
    finish(gk, s);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < s_nl; e += blockDim.x) {
    const int q = s_list[e];
    const int y = q / MG_TX, x = q - y * MG_TX;
    const int i = i0 + x, j = j0 + y;
    const size_t gk = a.L.idx(i, j);
    const uint16_t cd = a.code[gk];
    double s = 0.0;
    if (cd == 1) {
      const double* c = st + y * MG_TX + x;
      s = h2 * fma(4.0, c[MG_TX], c[0] + c[2 * MG_TX]);
    } else {
      // the four cells' classes, then the cut cells' indices, each as one
      // batch of independent loads (three round trips to memory, not twelve)
      uint8_t cl4[4];
      int cut4[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int ic = i - 1 + (k & 1), jc = j - 1 + (k >> 1);
        const bool in = ic >= 0 && jc >= 0 && ic < n && jc < n;
        cl4[k] = in ? a.cls[(size_t)jc * n + ic] : (uint8_t)CELL_EXT;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int ic = i - 1 + (k & 1), jc = j - 1 + (k >> 1);
        cut4[k] = cl4[k] == CELL_CUT ? a.cell_cut[(size_t)jc * n + ic] : 0;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int dx = k & 1, dy = k >> 1;
        const int ic = i - 1 + dx, jc = j - 1 + dy;
        const uint8_t cl = cl4[k];
        if (cl == CELL_EXT) continue;
        const int av = (1 - dx) + 2 * (1 - dy);
        // the cell's vertices (0,0),(1,0),(0,1),(1,1) in sf
        const double* fv = sf + (y + dy) * RHS_X + (x + dx);
        const double fb[4] = {fv[0], fv[1], fv[RHS_X], fv[RHS_X + 1]};
        if (cl == CELL_INT) {
          // whole-cell Q1 mass h^2/36 [[4,2,2,1],...]: 4 on the diagonal,
          // 2 along edges, 1 across the diagonal
          for (int b = 0; b < 4; ++b) {
            int wgt = (b == av) ? 4 : ((b ^ av) == 3 ? 1 : 2);
            s += h2 * wgt * fb[b];
          }
        } else {
          const double* Mk = a.Mk + (size_t)cut4[k] * 16 + av * 4;
          const double* Gk = a.Gk + (size_t)cut4[k] * 16 + av * 4;
          const size_t k0 = (size_t)jc * W + ic;
          const size_t vk[4] = {k0, k0 + 1, k0 + W, k0 + W + 1};
          for (int b = 0; b < 4; ++b) s += Mk[b] * fb[b] + Gk[b] * g[vk[b]];
          if (a.gN != nullptr && a.Nk != nullptr) {
            // Neumann load of the cell (zero on Dirichlet cells)
            const double* Nk = a.Nk + (size_t)cut4[k] * 16 + av * 4;
            for (int b = 0; b < 4; ++b) s += Nk[b] * a.gN[vk[b]];
          }
        }
      }
    }
    if (a.box && cd && (i == 1 || j == 1 || i == n - 1 || j == n - 1)) {
      // strong Dirichlet values of the box nodes moved to the right-hand
      // side: - sum over the adjacent cells of A_K(p, q) g_q, q on the box
      for (int k = 0; k < 4; ++k) {
        const int dx = k & 1, dy = k >> 1;
        const int ic = i - 1 + dx, jc = j - 1 + dy;
        if (ic < 0 || jc < 0 || ic >= n || jc >= n) continue;
        const size_t c = (size_t)jc * n + ic;
        const uint8_t cl = a.cls[c];
        if (cl == CELL_EXT) continue;
        const int av = (1 - dx) + 2 * (1 - dy);
        for (int b = 0; b < 4; ++b) {
          const int bi = ic + (b & 1), bj = jc + (b >> 1);
          if (!(bi == 0 || bj == 0 || bi == n || bj == n)) continue;
          double e;
          if (cl == CELL_INT) {
            // whole-cell Q1 stiffness: 4/6 diagonal, -1/6 along edges,
            // -2/6 across the diagonal
            e = (b == av) ? 4.0 / 6.0 : ((b ^ av) == 3 ? -2.0 / 6.0 : -1.0 / 6.0);
          } else {
            e = a.Ke[(size_t)a.cell_cut[c] * 16 + av * 4 + b];
          }
          s -= e * g[(size_t)bj * W + bi];
        }
      }
    }
    finish(gk, s);
  }
  return vmax;
}

}  // namespace
