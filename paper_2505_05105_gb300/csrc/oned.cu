// The one-dimensional ghost-FEM multigrid of Sec. 4, for the convergence
// studies of Sec. 4.5: Omega_art = [0, 1] with n cells, Omega = (a, b),
// a = (1 - theta_1) h, b = 1 - (1 - theta_2) h, P1 hats phi_0..phi_n, the
// Dirichlet value at a imposed by Nitsche's terms with penalty lambda and
// Neumann data at b (Eq. ls1dA).  Lexicographic Gauss-Seidel (P = L_h,
// Sec. 4.1), restriction Eq. resop and its transpose, Galerkin coarse
// operators (Eq. galerkin), coarsest grid of 8 cells solved exactly; the
// two-grid correction scheme of Alg. 1 or gamma* = 1, 2 cycles (Sec. 3.2).
//
// One thread block per problem; every level's tridiagonal operator and
// vectors live in shared memory.  Lexicographic Gauss-Seidel is a chain of
// dependent updates in 1D, so one thread runs each sweep and the exact
// tridiagonal solves; the residual, restriction, prolongation and norms use
// the whole block.
#include "ghostmg.h"

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace {

constexpr int kT = 128;
constexpr int kCoarsest = 8;
constexpr int kMaxLevels = 12;

struct Lev {
  int n;
  double *lo, *di, *up, *u, *F;
};

struct Hier {
  int nl;
  Lev L[kMaxLevels];
  double *cp, *dp;        // forward-elimination scratch of the exact solves
};

__host__ __device__ inline int levels_of(int n) {
  int nl = 1;
  while (n > kCoarsest) { n >>= 1; ++nl; }
  return nl;
}

__host__ __device__ inline size_t smem_doubles(int n) {
  size_t s = 0;
  for (int m = n; ; m >>= 1) {
    s += 5 * (size_t)(m + 1);
    if (m <= kCoarsest) break;
  }
  return s + 2 * (size_t)(n / 2 + 1);
}

__device__ void carve(Hier& H, double* base, int n) {
  H.nl = levels_of(n);
  double* p = base;
  for (int l = 0, m = n; l < H.nl; ++l, m >>= 1) {
    Lev& L = H.L[l];
    L.n = m;
    L.lo = p; p += m + 1;
    L.di = p; p += m + 1;
    L.up = p; p += m + 1;
    L.u = p; p += m + 1;
    L.F = p; p += m + 1;
  }
  H.cp = p; p += n / 2 + 1;
  H.dp = p;
}

// Eq. ls1dA from the element integrals: the stiffness of each cell's part in
// Omega (length len, slopes -1/h, 1/h) and Nitsche's terms at a,
// lambda u v + u' v + v' u (outward normal -1).
__device__ void assemble_fine(const Lev& L, double t1, double t2, double lam) {
  const int n = L.n;
  const double h = 1.0 / n;
  const double a = (1.0 - t1) * h, b = 1.0 - (1.0 - t2) * h;
  for (int i = threadIdx.x; i <= n; i += blockDim.x) {
    double di = 0.0, lo = 0.0, up = 0.0;
    for (int k = i - 1; k <= i; ++k) {
      if (k < 0 || k >= n) continue;
      const double len = fmin((k + 1) * h, b) - fmax(k * h, a);
      if (!(len > 0.0)) continue;
      const double s = len / (h * h);
      di += s;
      if (k == i - 1) lo -= s;
      else up -= s;
    }
    // the cell [x_0, x_1] holds a for theta_1 in (0, 1]
    const double va0 = 1.0 - a / h, va1 = a / h, d0 = -1.0 / h, d1 = 1.0 / h;
    if (i == 0) {
      di += lam * va0 * va0 + 2.0 * va0 * d0;
      up += lam * va0 * va1 + va0 * d1 + d0 * va1;
    } else if (i == 1) {
      di += lam * va1 * va1 + 2.0 * va1 * d1;
      lo += lam * va1 * va0 + va1 * d0 + d1 * va0;
    }
    L.di[i] = di;
    L.lo[i] = lo;
    L.up[i] = up;
  }
}

__device__ __forceinline__ double a_entry(const Lev& L, int p, int q) {
  if (q == p) return L.di[p];
  if (q == p - 1) return L.lo[p];
  if (q == p + 1) return L.up[p];
  return 0.0;
}

// A_2h = R A_h R^T (Eq. galerkin, Eq. resop): row I couples to I-1, I, I+1.
__device__ void galerkin(const Lev& F, const Lev& C) {
  const double w[3] = {0.5, 1.0, 0.5};
  for (int I = threadIdx.x; I <= C.n; I += blockDim.x) {
    double v[3] = {0.0, 0.0, 0.0};
    for (int d = -1; d <= 1; ++d) {
      const int J = I + d;
      if (J < 0 || J > C.n) continue;
      double s = 0.0;
      for (int a = -1; a <= 1; ++a) {
        const int p = 2 * I + a;
        if (p < 0 || p > F.n) continue;
        for (int b = -1; b <= 1; ++b) {
          const int q = 2 * J + b;
          if (q < 0 || q > F.n) continue;
          s += w[a + 1] * a_entry(F, p, q) * w[b + 1];
        }
      }
      v[d + 1] = s;
    }
    C.lo[I] = v[0];
    C.di[I] = v[1];
    C.up[I] = v[2];
  }
}

__device__ __forceinline__ double residual_at(const Lev& L, int i) {
  double s = L.di[i] * L.u[i];
  if (i > 0) s += L.lo[i] * L.u[i - 1];
  if (i < L.n) s += L.up[i] * L.u[i + 1];
  return L.F[i] - s;
}

// one lexicographic sweep, u_i += (F_i - (A u)_i) / A_ii, on thread 0
__device__ void gs_lex(const Lev& L) {
  if (threadIdx.x == 0) {
    const int n = L.n;
    double um = 0.0, uc = L.u[0];
    for (int i = 0; i <= n; ++i) {
      const double un = i < n ? L.u[i + 1] : 0.0;
      double s = L.di[i] * uc;
      if (i > 0) s += L.lo[i] * um;
      if (i < n) s += L.up[i] * un;
      const double v = uc + (L.F[i] - s) / L.di[i];
      L.u[i] = v;
      um = v;
      uc = un;
    }
  }
  __syncthreads();
}

// F_c = R (F - A u), u_c = 0
__device__ void restrict_residual(const Lev& F, const Lev& C) {
  for (int I = threadIdx.x; I <= C.n; I += blockDim.x) {
    double s = residual_at(F, 2 * I);
    if (2 * I - 1 >= 0) s += 0.5 * residual_at(F, 2 * I - 1);
    if (2 * I + 1 <= F.n) s += 0.5 * residual_at(F, 2 * I + 1);
    C.F[I] = s;
    C.u[I] = 0.0;
  }
  __syncthreads();
}

// u += R^T e_c (linear interpolation)
__device__ void prolong(const Lev& F, const Lev& C) {
  for (int i = threadIdx.x; i <= F.n; i += blockDim.x) {
    const double e = (i & 1) ? 0.5 * C.u[i >> 1] + 0.5 * C.u[(i >> 1) + 1] : C.u[i >> 1];
    F.u[i] += e;
  }
  __syncthreads();
}

// exact solve of the tridiagonal A u = F (forward elimination, back
// substitution; A is symmetric positive definite, so no pivoting)
__device__ void exact(const Hier& H, const Lev& L, unsigned* err) {
  if (threadIdx.x == 0) {
    const int n = L.n;
    double m = L.di[0];
    if (!(m > 0.0)) *err |= DEV_ERR_NOT_SPD;
    H.cp[0] = L.up[0] / m;
    H.dp[0] = L.F[0] / m;
    for (int i = 1; i <= n; ++i) {
      m = L.di[i] - L.lo[i] * H.cp[i - 1];
      if (!(m > 0.0)) *err |= DEV_ERR_NOT_SPD;
      H.cp[i] = i < n ? L.up[i] / m : 0.0;
      H.dp[i] = (L.F[i] - L.lo[i] * H.dp[i - 1]) / m;
    }
    L.u[n] = H.dp[n];
    for (int i = n - 1; i >= 0; --i) L.u[i] = H.dp[i] - H.cp[i] * L.u[i + 1];
  }
  __syncthreads();
}

__device__ double res_norm(const Lev& L, double* red) {
  double m = 0.0;
  for (int i = threadIdx.x; i <= L.n; i += blockDim.x) m = fmax(m, fabs(residual_at(L, i)));
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  double r = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
  __syncthreads();
  return r;
}

// One cycle of Alg. 1 from level 0, without recursion: cnt[l] counts the
// visits of level l still due from its parent (gamma* per parent visit).
__device__ void one_cycle(const Hier& H, int nu1, int nu2, int gam, bool two_grid,
                          unsigned* err) {
  int cnt[kMaxLevels];
  const int last = H.nl - 1;
  int l = 0;
  for (;;) {
    if (l == last) {
      exact(H, H.L[l], err);
      --l;
      bool done = false;
      for (;;) {
        if (--cnt[l + 1] > 0) { ++l; break; }       // visit the child again
        prolong(H.L[l], H.L[l + 1]);
        for (int k = 0; k < nu2; ++k) gs_lex(H.L[l]);
        if (l == 0) { done = true; break; }
        --l;
      }
      if (done) return;
      continue;
    }
    for (int k = 0; k < nu1; ++k) gs_lex(H.L[l]);
    restrict_residual(H.L[l], H.L[l + 1]);
    if (two_grid) {
      exact(H, H.L[1], err);
      prolong(H.L[0], H.L[1]);
      for (int k = 0; k < nu2; ++k) gs_lex(H.L[0]);
      return;
    }
    cnt[l + 1] = gam;
    ++l;
  }
}

struct Prob {
  int n;
  double t1, t2, lam;
  long long off;          // first node in the packed arrays
};

__global__ void __launch_bounds__(kT)
k_mg1d(const Prob* __restrict__ probs, const double* __restrict__ F, double* __restrict__ u,
       double* __restrict__ res, int cycles, int nu1, int nu2, int gam, int two_grid,
       unsigned* __restrict__ err_out) {
  extern __shared__ __align__(16) double sm[];
  __shared__ double red[kT / 32];
  __shared__ unsigned err;
  const Prob P = probs[blockIdx.x];
  Hier H;
  carve(H, sm, P.n);
  if (threadIdx.x == 0) err = 0u;
  assemble_fine(H.L[0], P.t1, P.t2, P.lam);
  for (int i = threadIdx.x; i <= P.n; i += blockDim.x) {
    H.L[0].u[i] = u[P.off + i];
    H.L[0].F[i] = F ? F[P.off + i] : 0.0;
  }
  __syncthreads();
  for (int l = 1; l < H.nl; ++l) {
    galerkin(H.L[l - 1], H.L[l]);
    __syncthreads();
  }
  double* rh = res + (size_t)blockIdx.x * (cycles + 1);
  double r = res_norm(H.L[0], red);
  if (threadIdx.x == 0) rh[0] = r;
  for (int m = 1; m <= cycles; ++m) {
    one_cycle(H, nu1, nu2, gam, two_grid != 0, &err);
    r = res_norm(H.L[0], red);
    if (threadIdx.x == 0) rh[m] = r;
  }
  for (int i = threadIdx.x; i <= P.n; i += blockDim.x) u[P.off + i] = H.L[0].u[i];
  __syncthreads();
  if (threadIdx.x == 0 && err) atomicOr(err_out, err);
}

bool device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int mg1d_cycles(int count, const mg1d_problem* problems, int cycle, int nu1, int nu2,
                           int cycles, const double* F, double* u, double* res,
                           void* cuda_stream) {
  if (count < 1 || !problems || !u || !res) return MG_ERR_INVALID_ARG;
  if (cycle < 0 || cycle > 2 || nu1 < 0 || nu1 > 8 || nu2 < 0 || nu2 > 8 || nu1 + nu2 == 0 ||
      cycles < 0 || cycles > 1000)
    return MG_ERR_INVALID_ARG;
  if (!device_ptr(u) || (F && !device_ptr(F)) || device_ptr(res)) return MG_ERR_INVALID_ARG;
  std::vector<Prob> P(count);
  long long off = 0;
  int nmax = 0;
  for (int k = 0; k < count; ++k) {
    const mg1d_problem& q = problems[k];
    const int n = q.n_cells;
    if (n < 2 * kCoarsest || n > MG1D_MAX_CELLS || (n & (n - 1)) != 0)
      return MG_ERR_INVALID_ARG;
    if (!(q.theta1 > 0.0 && q.theta1 <= 1.0) || !(q.theta2 > 0.0 && q.theta2 <= 1.0) ||
        !(q.lambda > 0.0) || !std::isfinite(q.lambda))
      return MG_ERR_INVALID_ARG;
    P[k] = Prob{n, q.theta1, q.theta2, q.lambda, off};
    off += n + 1;
    nmax = std::max(nmax, n);
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t smem = smem_doubles(nmax) * sizeof(double);
  MG_CUDA_TRY(raise_smem_limit(k_mg1d, smem));
  Prob* dP = nullptr;
  double* dres = nullptr;
  unsigned* derr = nullptr;
  const size_t nres = (size_t)count * (cycles + 1);
  MG_CUDA_TRY(cudaMallocAsync(&dP, sizeof(Prob) * count, st));
  cudaError_t e = cudaMallocAsync(&dres, sizeof(double) * nres, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&derr, sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dP, P.data(), sizeof(Prob) * count,
                                            cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) {
    k_mg1d<<<count, kT, smem, st>>>(dP, F, u, dres, cycles, nu1, nu2, cycle == 2 ? 2 : 1,
                                     cycle == 0 ? 1 : 0, derr);
    e = cudaGetLastError();
  }
  unsigned herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(res, dres, sizeof(double) * nres,
                                            cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(unsigned),
                                            cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(dP, st);
  if (dres) cudaFreeAsync(dres, st);
  if (derr) cudaFreeAsync(derr, st);
  if (e != cudaSuccess) return mg_cuda_fail(e);
  if (herr & DEV_ERR_NOT_SPD) return MG_ERR_NOT_SPD;
  return MG_OK;
}

// binds the bounds-checked build's device error word (see common.cuh)
MG_BOUNDS_BINDER(bind_bounds_oned)
