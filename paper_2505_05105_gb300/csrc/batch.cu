// Batched solves: one persistent kernel V-cycles many independent geometries.
//
// Each block takes a whole problem from a work queue (largest first) and
// runs its entire mixed-precision solve without leaving the kernel: the fp64
// residual r = F - A u of the fine level, its l_inf norm and the stop test
// ||r|| / ||F|| <= tol; groups of fp32 V(nu1, nu2)-cycles on A e = sigma r
// (the group size predicted from the contraction seen so far, as in the
// single-problem solver); u += e / sigma in fp64.  The problems are
// independent, so blocks never wait for one another.  Per V-cycle, the
// levels above 64 x 64 cells are smoothed block-wide in global memory (a
// 4-colour Gauss-Seidel sweep over the level's active tiles with the colour's
// cut-cell vertices from a list, then eta sweeps over those vertices,
// Sec. 4.1 and Sec. 5.3), restricted (R = P^T) and prolongated (P) as in
// Sec. 5.1; the levels from 64 x 64 down run in shared memory by the tail
// code (tail_impl.cuh).  The arithmetic is that of the single-problem
// kernels.
#include "batch.cuh"
#include "ghostmg.h"
#include "rhs_impl.cuh"
#include "tail_impl.cuh"

namespace {

__device__ __forceinline__ double block_max(double v) {
  __shared__ double s[32];
  __syncthreads();
  v = warp_max(v);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0.0;
    v = warp_max(v);
    if (threadIdx.x == 0) s[0] = v;
  }
  __syncthreads();
  return s[0];
}

// node q of the active tiles: q >> 11 selects the tile, the rest the node
__device__ __forceinline__ bool tile_node(const Layout& L, const int* active, int q, int& i,
                                          int& j) {
  const int t = active[q >> 11], w = q & 2047;
  i = (t % L.ntx) * MG_TX + (w & (MG_TX - 1));
  j = (t / L.ntx) * MG_TY + (w >> 6);
  return i <= L.n && j <= L.n;
}

// node q of colour (ci, cj) of the active tiles (512 per tile)
__device__ __forceinline__ bool colour_node(const Layout& L, const int* active, int q, int ci,
                                            int cj, int& i, int& j) {
  const int t = active[q >> 9], w = q & 511;
  i = (t % L.ntx) * MG_TX + 2 * (w & 31) + ci;
  j = (t / L.ntx) * MG_TY + 2 * (w >> 5) + cj;
  return i <= L.n && j <= L.n;
}

template <class T>
__device__ __forceinline__ T row_apply(const T* R, const T* U, int P) {
  return R[0] * U[-P - 1] + R[1] * U[-P] + R[2] * U[-P + 1] + R[3] * U[-1] + R[4] * U[0] +
         R[5] * U[1] + R[6] * U[P - 1] + R[7] * U[P] + R[8] * U[P + 1];
}

__device__ __forceinline__ void listed_update(const BatchLevel& v, int e) {
  const int2 en = v.blist[e];
  const float* R = v.rows + (size_t)en.y * MG_ROW;
  float* U = v.u + v.L.idx(en.x & 0xffff, en.x >> 16);
  const float f = v.F[U - v.u];
  const float acc = row_apply(R, U, v.L.pitch);
  *U = U[0] + (f - acc) * R[9];
}

// one smoothing step of a level in global memory: 4 colour phases (interior
// nodes by the constant stencil, the colour's boundary nodes from the list),
// then eta phases per colour over the boundary nodes only
__device__ void smooth_level(const BatchLevel& v, int eta) {
  const int P = v.L.pitch;
  for (int c = 0; c < 4; ++c) {
    const int ci = c & 1, cj = c >> 1;
    for (int q = threadIdx.x; q < v.n_active * 512; q += blockDim.x) {
      int i, j;
      if (!colour_node(v.L, v.active, q, ci, cj, i, j)) continue;
      const size_t g = v.L.idx(i, j);
      if (v.code[g] != 1) continue;
      const float* U = v.u + g;
      const float s8 = ((U[-1] + U[1]) + (U[-P] + U[P])) + ((U[-P - 1] + U[-P + 1]) +
                                                            (U[P - 1] + U[P + 1]));
      v.u[g] = (3.f * v.F[g] + s8) * 0.125f;
    }
    for (int e = v.boff[c] + threadIdx.x; e < v.boff[c + 1]; e += blockDim.x) listed_update(v, e);
    __syncthreads();
  }
  for (int it = 0; it < eta; ++it)
    for (int c = 0; c < 4; ++c) {
      for (int e = v.boff[c] + threadIdx.x; e < v.boff[c + 1]; e += blockDim.x)
        listed_update(v, e);
      __syncthreads();
    }
}

__device__ void zero_level(const BatchLevel& v) {
  for (int q = threadIdx.x; q < v.n_active * 2048; q += blockDim.x) {
    int i, j;
    if (tile_node(v.L, v.active, q, i, j)) v.u[v.L.idx(i, j)] = 0.f;
  }
  __syncthreads();
}

// F_2h = P^T (F - A u): the residual of the active tiles into scr, then the
// 9-point restriction (weights 1, 1/2, 1/4) for every node of the coarse
// level's active tiles
__device__ void resid_restrict_level(const BatchLevel& v, const Layout& Lc, const int* cact,
                                     int nc_act, float* Fc) {
  const int P = v.L.pitch;
  for (int q = threadIdx.x; q < v.n_active * 2048; q += blockDim.x) {
    int i, j;
    if (!tile_node(v.L, v.active, q, i, j)) continue;
    const size_t g = v.L.idx(i, j);
    const uint16_t cd = v.code[g];
    float r = 0.f;
    if (cd == 1) {
      const float* U = v.u + g;
      const float s8 = ((U[-1] + U[1]) + (U[-P] + U[P])) + ((U[-P - 1] + U[-P + 1]) +
                                                            (U[P - 1] + U[P + 1]));
      r = v.F[g] - (8.f * U[0] - s8) * (1.f / 3.f);
    } else if (cd >= 2) {
      const float* R = v.rows + (size_t)(v.tile_base[v.L.tile_of(i, j)] + cd - 2) * MG_ROW;
      r = v.F[g] - row_apply(R, v.u + g, P);
    }
    v.scr[g] = r;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nc_act * 2048; q += blockDim.x) {
    int I, J;
    if (!tile_node(Lc, cact, q, I, J)) continue;
    const float* R = v.scr + v.L.idx(2 * I, 2 * J);
    const float rc = R[0] + 0.5f * ((R[-1] + R[1]) + (R[-P] + R[P])) +
                     0.25f * ((R[-P - 1] + R[-P + 1]) + (R[P - 1] + R[P + 1]));
    Fc[Lc.idx(I, J)] = rc;
  }
  __syncthreads();
}

// u += P e_2h on the DOFs of the active tiles (same association as k_prolong)
__device__ void prolong_level(const BatchLevel& v, const Layout& Lc, const float* ec) {
  for (int q = threadIdx.x; q < v.n_active * 2048; q += blockDim.x) {
    int i, j;
    if (!tile_node(v.L, v.active, q, i, j)) continue;
    const size_t g = v.L.idx(i, j);
    if (!v.code[g]) continue;
    const float* E = ec + Lc.idx(i >> 1, j >> 1);
    float e;
    if (!(i & 1) && !(j & 1)) e = E[0];
    else if (!(j & 1)) e = 0.5f * (E[0] + E[1]);
    else if (!(i & 1)) e = 0.5f * (E[0] + E[Lc.pitch]);
    else e = 0.25f * ((E[0] + E[1]) + (E[Lc.pitch] + E[Lc.pitch + 1]));
    v.u[g] = v.u[g] + e;
  }
  __syncthreads();
}

// one fp32 V-cycle of problem p on the correction equation; load_image: the
// tail's static image is not yet in shared memory
__device__ void vcycle(const BatchProblem& p, bool zero_init, unsigned char* smem,
                       bool load_image) {
  for (int l = 0; l < p.n_top; ++l) {
    const BatchLevel& v = p.lev[l];
    if (l > 0 || zero_init) zero_level(v);
    for (int s = 0; s < p.nu1; ++s) smooth_level(v, p.eta);
    const bool next_top = l + 1 < p.n_top;
    const Layout& Lc = next_top ? p.lev[l + 1].L : p.tail.L0;
    const int* cact = next_top ? p.lev[l + 1].active : nullptr;
    if (next_top) {
      resid_restrict_level(v, Lc, cact, p.lev[l + 1].n_active, p.lev[l + 1].F);
    } else {
      // the tail's top level (its active tiles; the tail ignores F off the DOFs)
      resid_restrict_level(v, Lc, p.tail_active, p.tail_n_active, p.tail_F);
    }
  }
  tail_vcycle<float>(p.tail, smem, p.n_top == 0 && !zero_init, load_image);
  __syncthreads();
  for (int l = p.n_top - 1; l >= 0; --l) {
    const BatchLevel& v = p.lev[l];
    const bool next_top = l + 1 < p.n_top;
    prolong_level(v, next_top ? p.lev[l + 1].L : p.tail.L0,
                  next_top ? p.lev[l + 1].u : p.tail.u0);
    for (int s = 0; s < p.nu2; ++s) smooth_level(v, p.eta);
  }
}

// fp64 residual of the fine level: F32 = sigma r on the DOFs, returns ||r||_inf
__device__ double residual64(const BatchProblem& p, double sigma) {
  const Layout& L = p.L0;
  const int P = L.pitch;
  double vmax = 0.0;
  for (int q = threadIdx.x; q < p.n_active0 * 2048; q += blockDim.x) {
    int i, j;
    if (!tile_node(L, p.active0, q, i, j)) continue;
    const size_t g = L.idx(i, j);
    const uint16_t cd = p.code0[g];
    double r = 0.0;
    if (cd == 1) {
      const double* U = p.u64 + g;
      const double s8 = ((U[-1] + U[1]) + (U[-P] + U[P])) + ((U[-P - 1] + U[-P + 1]) +
                                                             (U[P - 1] + U[P + 1]));
      r = p.F64[g] - (8.0 * U[0] - s8) * (1.0 / 3.0);
    } else if (cd >= 2) {
      const double* R = p.rows64 + (size_t)(p.tile_base0[L.tile_of(i, j)] + cd - 2) * MG_ROW;
      r = p.F64[g] - row_apply(R, p.u64 + g, P);
    }
    vmax = fmax(vmax, fabs(r));
    p.F32[g] = (float)(r * sigma);
  }
  return block_max(vmax);
}

__device__ double pow2_near_inverse(double x) {
  if (!(x > 0.0) || !isfinite(x)) return 1.0;
  int e;
  frexp(x, &e);
  return ldexp(1.0, -e);
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1)
k_batch(const BatchProblem* __restrict__ probs, const int* __restrict__ order, int count,
        int* next, const unsigned* __restrict__ bad, const double* __restrict__ params,
        int first_group, BatchResult* res) {
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  unsigned char* smem = smem_align128(smem_dyn);
  __shared__ int cur;
  const double tol = params[0];
  const int max_cycles = (int)params[1];
  const int fixed = (int)params[2];           // > 0: fixed group size
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) cur = atomicAdd(next, 1);
    __syncthreads();
    const int k = cur;
    if (k >= count) break;
    const int pi = order[k];
    const BatchProblem& p = probs[pi];
    const Layout& L = p.L0;
    const bool invalid = bad[pi] != 0;
    // u = 0 and ||F||_inf
    double fmax_ = 0.0;
    for (int q = threadIdx.x; q < p.n_active0 * 2048; q += blockDim.x) {
      int i, j;
      if (!tile_node(L, p.active0, q, i, j)) continue;
      const size_t g = L.idx(i, j);
      p.u64[g] = 0.0;
      if (!invalid) fmax_ = fmax(fmax_, fabs(p.F64[g]));
    }
    const double Fn = block_max(fmax_);
    int cycles = 0, checks = 0, status = invalid ? MG_ERR_INVALID_ARG : MG_OK;
    double rel = 0.0;
    if (!invalid && Fn > 0.0) {
      double sigma = pow2_near_inverse(Fn), rmax = Fn, best = 1.0, rho = 0.1;
      // u = 0: the first refinement residual is F itself
      for (int q = threadIdx.x; q < p.n_active0 * 2048; q += blockDim.x) {
        int i, j;
        if (!tile_node(L, p.active0, q, i, j)) continue;
        const size_t g = L.idx(i, j);
        p.F32[g] = (float)(p.F64[g] * sigma);
      }
      __syncthreads();
      rel = 1.0;
      int kk = fixed > 0 ? fixed : first_group;
      while (rel > tol) {
        if (cycles >= max_cycles) { status = MG_ERR_NOT_CONVERGED; break; }
        kk = min(kk, max_cycles - cycles);
        for (int s = 0; s < kk; ++s) {
          vcycle(p, s == 0, smem, cycles + s == 0);
        }
        cycles += kk;
        // u += e / sigma on the DOFs (same arithmetic as k_update)
        const double inv = 1.0 / sigma;
        for (int q = threadIdx.x; q < p.n_active0 * 2048; q += blockDim.x) {
          int i, j;
          if (!tile_node(L, p.active0, q, i, j)) continue;
          const size_t g = L.idx(i, j);
          if (p.code0[g]) p.u64[g] += (double)p.e32[g] * inv;
        }
        __syncthreads();
        sigma = pow2_near_inverse(rmax * pow(rho, kk));
        const double rnew = residual64(p, sigma);
        ++checks;
        rel = rnew / Fn;
        if (!isfinite(rel) || rel > 1e3 * best) { status = MG_ERR_DIVERGED; break; }
        best = fmin(best, rel);
        rho = fmin(0.9, fmax(0.01, pow(rnew / rmax, 1.0 / kk)));
        rmax = rnew;
        if (fixed <= 0 && rel > tol) {
          const double need = log(tol / rel) / log(rho);
          kk = max(1, min(8, (int)ceil(need + 0.5)));
        }
      }
    }
    if (threadIdx.x == 0) {
      BatchResult r;
      r.cycles = cycles;
      r.checks = checks;
      r.status = status;
      r.pad = 0;
      r.rel_res = rel;
      res[pi] = r;
    }
  }
}

// member p of the flattened range: off[p] <= x < off[p + 1]
template <class I>
__device__ __forceinline__ int member_of(const I* off, int count, I x) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

constexpr int kFlatThreads = 256;

__global__ void __launch_bounds__(kFlatThreads)
k_batch_check(const BatchProblem* __restrict__ probs, const size_t* __restrict__ node_off,
              int count, size_t total, unsigned* __restrict__ bad) {
  const size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (x >= total) return;
  const int p = member_of(node_off, count, x);
  const size_t k = x - node_off[p];
  if (!isfinite(probs[p].f[k]) || !isfinite(probs[p].g[k])) atomicOr(&bad[p], 1u);
}

__global__ void __launch_bounds__(kFlatThreads)
k_batch_rhs(const BatchProblem* __restrict__ probs, const int* __restrict__ tile_off,
            int count) {
  const int p = member_of(tile_off, count, (int)blockIdx.x);
  const BatchProblem& b = probs[p];
  rhs_tile(b.rhs, b.active0[blockIdx.x - tile_off[p]], b.f, b.g, b.F64);
}

__global__ void __launch_bounds__(kFlatThreads)
k_batch_unpack(const BatchProblem* __restrict__ probs, const size_t* __restrict__ node_off,
               int count, size_t total) {
  const size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (x >= total) return;
  const int p = member_of(node_off, count, x);
  const BatchProblem& b = probs[p];
  const int k = (int)(x - node_off[p]), W = b.L0.n + 1;
  const int j = k / W, i = k - j * W;
  const size_t g = b.L0.idx(i, j);
  b.u_out[k] = b.code0[g] ? b.u64[g] : 0.0;
}

// colour-sorted boundary-node list of one level (one block)
__global__ void k_batch_lists(Layout L, const uint16_t* __restrict__ code,
                              const int* __restrict__ tile_base, int2* __restrict__ blist,
                              int* __restrict__ boff) {
  __shared__ int cnt[4], cur[4];
  if (threadIdx.x < 4) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int W = L.n + 1;
  for (int q = threadIdx.x; q < W * W; q += blockDim.x) {
    const int j = q / W, i = q - j * W;
    if (code[L.idx(i, j)] >= 2) atomicAdd(&cnt[(i & 1) + 2 * (j & 1)], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int c = 0; c < 4; ++c) {
      boff[c] = acc;
      cur[c] = acc;
      acc += cnt[c];
    }
    boff[4] = acc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < W * W; q += blockDim.x) {
    const int j = q / W, i = q - j * W;
    const uint16_t cd = code[L.idx(i, j)];
    if (cd < 2) continue;
    const int pos = atomicAdd(&cur[(i & 1) + 2 * (j & 1)], 1);
    blist[pos] = make_int2(i | (j << 16), tile_base[L.tile_of(i, j)] + cd - 2);
  }
}

}  // namespace

cudaError_t configure_batch(size_t smem) {
  cudaError_t e;
  e = cudaFuncSetAttribute(k_batch<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_batch<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_batch<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

void launch_batch(const BatchProblem* probs, const int* order, int count, int* next,
                  const unsigned* bad, const double* params, BatchTune tune, int grid,
                  size_t smem, BatchResult* res, cudaStream_t st) {
  if (tune.threads >= 1024)
    k_batch<1024><<<grid, 1024, smem, st>>>(probs, order, count, next, bad, params,
                                            tune.first_group, res);
  else if (tune.threads >= 512)
    k_batch<512><<<grid, 512, smem, st>>>(probs, order, count, next, bad, params,
                                          tune.first_group, res);
  else
    k_batch<256><<<grid, 256, smem, st>>>(probs, order, count, next, bad, params,
                                          tune.first_group, res);
}

static unsigned flat_grid(size_t total) {
  return (unsigned)((total + kFlatThreads - 1) / kFlatThreads);
}

void launch_batch_check(const BatchProblem* probs, const size_t* node_off, int count,
                        size_t total_nodes, unsigned* bad, cudaStream_t st) {
  if (total_nodes == 0) return;
  k_batch_check<<<flat_grid(total_nodes), kFlatThreads, 0, st>>>(probs, node_off, count,
                                                                 total_nodes, bad);
}

void launch_batch_rhs(const BatchProblem* probs, const int* tile_off, int count, int total_tiles,
                      cudaStream_t st) {
  if (total_tiles == 0) return;
  k_batch_rhs<<<total_tiles, kFlatThreads, 0, st>>>(probs, tile_off, count);
}

void launch_batch_unpack(const BatchProblem* probs, const size_t* node_off, int count,
                         size_t total_nodes, cudaStream_t st) {
  if (total_nodes == 0) return;
  k_batch_unpack<<<flat_grid(total_nodes), kFlatThreads, 0, st>>>(probs, node_off, count,
                                                                  total_nodes);
}

void launch_batch_lists(const Layout& L, const uint16_t* code, const int* tile_base,
                        int2* blist, int* boff, cudaStream_t st) {
  k_batch_lists<<<1, 1024, 0, st>>>(L, code, tile_base, blist, boff);
}
