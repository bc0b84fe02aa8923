// The global stabilisation constant of Sec. 5.2 on the GPU.
//
// C_global is the largest generalized eigenvalue of the global pencil
//     K v = Lambda M v,   K_ij = int_{Gamma_D} (n . grad phi_i)(n . grad phi_j) dS,
//                         M_ij = int_{Omega_h} grad phi_i . grad phi_j dx,
// over the whole FE space (the DOFs of the fine level).  Both matrices
// annihilate the constants; the pencil is taken modulo constants (the
// rank-based definition of Sec. 4.4): with w = 1 / sqrt(#DOFs) on the DOFs,
// M' = M + w w^T is positive definite (connected active region) and every
// v = c 1 + v' (w . v' = 0) has the Rayleigh quotient of v', so
// Lambda_max(K, M') is the value.
//
// Steps:
//   k_cut_pencil   per cut cell: the volume stiffness S and the normal-
//                  derivative matrix Kn (zero on Neumann cells), from the
//                  same exact quadrature as the element matrices;
//   k_pencil_rows  9-point rows of M (internal cells: the Q1 stiffness; cut
//                  cells: S) and K (cut cells: Kn), summed over each node's
//                  four cells;
//   k_lanczos      Lanczos on T = M'^{-1} K, which is self-adjoint in the M'
//                  inner product, with full M'-reorthogonalisation; each
//                  application of M'^{-1} is a Jacobi-preconditioned conjugate
//                  gradient solve.  The largest Ritz value of the Lanczos
//                  tridiagonal (Sturm bisection) is Lambda_max.  One
//                  cooperative launch: blocks meet at grid-wide barriers, and
//                  every reduction is summed in a fixed order, so the result
//                  is deterministic.
// Everything is in cell units (h = 1): S is h-independent in 2D and
// Kn_phys = Kn / h, so C_global = Lambda / h.
#include <cooperative_groups.h>

#include "cutcell.cuh"
#include "global.cuh"

namespace cg = cooperative_groups;

namespace {

__device__ __constant__ double kS1[16] = {
    4.0 / 6.0,  -1.0 / 6.0, -1.0 / 6.0, -2.0 / 6.0,
    -1.0 / 6.0, 4.0 / 6.0,  -2.0 / 6.0, -1.0 / 6.0,
    -1.0 / 6.0, -2.0 / 6.0, 4.0 / 6.0,  -1.0 / 6.0,
    -2.0 / 6.0, -1.0 / 6.0, -1.0 / 6.0, 4.0 / 6.0};

__global__ void k_cut_pencil(const double* __restrict__ psi_s, int n, const int* __restrict__ list,
                             int ncut, const uint8_t* __restrict__ nmask, double* __restrict__ S,
                             double* __restrict__ Kn) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncut) return;
  const int c = list[t];
  const int ic = c % n, jc = c / n;
  const size_t k0 = (size_t)jc * (n + 1) + ic;
  const double psi[4] = {psi_s[k0], psi_s[k0 + 1], psi_s[k0 + n + 1], psi_s[k0 + n + 2]};
  cutcell::CellOut o;
  cutcell::cut_cell_matrices(psi, 1.0, 1.0, o, nmask != nullptr && nmask[c] != 0);
  for (int k = 0; k < 16; ++k) {
    S[(size_t)t * 16 + k] = o.S[k];
    Kn[(size_t)t * 16 + k] = o.Kn[k];
  }
}

// rows of node (i, j): s = (di + 1) + 3 (dj + 1); dof[k] = 1 for a vertex of
// an active cell
__global__ void k_pencil_rows(int n, const uint8_t* __restrict__ cls,
                              const int* __restrict__ cell_cut, const double* __restrict__ S,
                              const double* __restrict__ Kn, double* __restrict__ Mr,
                              double* __restrict__ Kr, uint8_t* __restrict__ dof) {
  const int m = (n + 1) * (n + 1);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const int i = k % (n + 1), j = k / (n + 1);
  double mr[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, kr[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  int active = 0;
  for (int q = 0; q < 4; ++q) {
    const int ic = i - 1 + (q & 1), jc = j - 1 + (q >> 1);
    if (ic < 0 || jc < 0 || ic >= n || jc >= n) continue;
    const size_t c = (size_t)jc * n + ic;
    const uint8_t v = cls[c];
    if (v == CELL_EXT) continue;
    active = 1;
    const double* E = v == CELL_INT ? kS1 : S + (size_t)cell_cut[c] * 16;
    const double* B = v == CELL_INT ? nullptr : Kn + (size_t)cell_cut[c] * 16;
    const int a = (i - ic) + 2 * (j - jc);          // local vertex of (i, j)
    for (int b = 0; b < 4; ++b) {
      const int di = ic + (b & 1) - i, dj = jc + (b >> 1) - j;
      const int s = (di + 1) + 3 * (dj + 1);
      mr[s] += E[a * 4 + b];
      if (B) kr[s] += B[a * 4 + b];
    }
  }
  for (int s = 0; s < 9; ++s) {
    Mr[(size_t)k * 9 + s] = mr[s];
    Kr[(size_t)k * 9 + s] = kr[s];
  }
  dof[k] = (uint8_t)active;
}

// ---------------------------------------------------------------------------
// Lanczos with inner conjugate-gradient solves, one cooperative launch
// ---------------------------------------------------------------------------

constexpr int kThreads = 512;
constexpr int kRed = 4;                 // values per block partial

struct Work {
  int n, m;                             // cells per side, nodes
  const double* Mr;                     // 9 per node
  const double* Kr;
  const uint8_t* dof;
  double wgt;                           // 1 / sqrt(#DOFs)
  double* Q;                            // (kmax + 1) x m Lanczos vectors
  double* MQ;                           // M' Q
  double *x, *r, *z, *p, *q, *u;        // m each
  double* part;                         // 3 x gridDim x kRed partials
  double* out;                          // [0] Lambda, [1] steps, [2] CG iterations, [3] last beta
  int kmax;
  int cg_max;
  double cg_tol;
};

// y = A x for the 9-point rows R (zero rows off the DOFs)
__device__ __forceinline__ double row_apply(const double* R, const double* x, int k, int n) {
  const int i = k % (n + 1), j = k / (n + 1);
  double s = 0.0;
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    const double a = R[(size_t)k * 9 + t];
    if (a != 0.0) {
      const int ii = i + t % 3 - 1, jj = j + t / 3 - 1;
      s += a * x[(size_t)jj * (n + 1) + ii];
    }
  }
  return s;
}

// Sums `cnt` per-thread values over the grid in a fixed order; every block
// gets the same totals.  `slot` rotates through three partial buffers, so
// that a buffer is rewritten only after every block has read it (two grid
// barriers later).
template <int CNT>
__device__ void grid_sum(const Work& w, cg::grid_group& g, double* v, int& slot) {
  __shared__ double sred[kThreads / 32][kRed];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < CNT; ++c) {
    double a = v[c];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) sred[warp][c] = a;
  }
  __syncthreads();
  double* P = w.part + (size_t)slot * gridDim.x * kRed;
  if (threadIdx.x < CNT) {
    double a = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) a += sred[q][threadIdx.x];
    P[(size_t)blockIdx.x * kRed + threadIdx.x] = a;
  }
  g.sync();
  __shared__ double stot[kRed];
  if (threadIdx.x < CNT) {
    double a = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) a += P[(size_t)b * kRed + threadIdx.x];
    stot[threadIdx.x] = a;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < CNT; ++c) v[c] = stot[c];
  __syncthreads();
  slot = (slot + 1) % 3;
}

// Largest eigenvalue of the symmetric tridiagonal (a[0..k-1], b[0..k-2]) by
// Sturm-sequence bisection.
__device__ double tridiag_max(const double* a, const double* b, int k) {
  double lo = a[0], hi = a[0];
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < k ? fabs(b[i]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    // eigenvalues greater than mid = sign changes counted on T - mid
    int above = 0;
    double d = 1.0;
    for (int i = 0; i < k; ++i) {
      const double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
      d = (a[i] - mid) - (i > 0 ? bb / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d > 0.0) ++above;
    }
    if (above > 0) lo = mid;
    else hi = mid;
  }
  return 0.5 * (lo + hi);
}

// deterministic start vector entry (splitmix64 of the node index), in [-1, 1)
__device__ __forceinline__ double start_value(int k) {
  unsigned long long x = (unsigned long long)k + 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// x = M'^{-1} b by Jacobi-preconditioned CG from x = 0 (b = w.r: the
// caller's vector in w.r); returns the iterations
__device__ int cg_solve(const Work& w, cg::grid_group& g, int& slot) {
  const int m = w.m, n = w.n;
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  // x = 0, z = D^{-1} r, p = z; r.r, r.z, w.z
  double v[3] = {0.0, 0.0, 0.0};
  for (size_t k = tid; k < (size_t)m; k += stride) {
    w.x[k] = 0.0;
    double zk = 0.0;
    if (w.dof[k]) {
      const double dg = w.Mr[k * 9 + 4] + w.wgt * w.wgt;
      zk = w.r[k] / dg;
      v[0] += w.r[k] * w.r[k];
      v[1] += w.r[k] * zk;
      v[2] += w.wgt * zk;
    }
    w.z[k] = zk;
    w.p[k] = zk;
  }
  grid_sum<3>(w, g, v, slot);
  const double bb = v[0];
  double rz = v[1], wp = v[2];
  if (!(bb > 0.0)) return 0;
  int it = 0;
  for (; it < w.cg_max; ++it) {
    // q = M' p = M p + w (w . p); p . q
    double pq[1] = {0.0};
    for (size_t k = tid; k < (size_t)m; k += stride) {
      double qk = 0.0;
      if (w.dof[k]) qk = row_apply(w.Mr, w.p, (int)k, n) + w.wgt * wp;
      w.q[k] = qk;
      pq[0] += w.p[k] * qk;
    }
    grid_sum<1>(w, g, pq, slot);
    const double alpha = rz / pq[0];
    double v2[3] = {0.0, 0.0, 0.0};
    for (size_t k = tid; k < (size_t)m; k += stride) {
      if (!w.dof[k]) continue;
      w.x[k] += alpha * w.p[k];
      const double rk = w.r[k] - alpha * w.q[k];
      w.r[k] = rk;
      const double zk = rk / (w.Mr[k * 9 + 4] + w.wgt * w.wgt);
      w.z[k] = zk;
      v2[0] += rk * rk;
      v2[1] += rk * zk;
      v2[2] += w.wgt * zk;
    }
    grid_sum<3>(w, g, v2, slot);
    if (v2[0] <= w.cg_tol * w.cg_tol * bb) { ++it; break; }
    const double beta = v2[1] / rz;
    rz = v2[1];
    wp = v2[2] + beta * wp;
    for (size_t k = tid; k < (size_t)m; k += stride)
      if (w.dof[k]) w.p[k] = w.z[k] + beta * w.p[k];
    g.sync();
  }
  return it;
}

__global__ void __launch_bounds__(kThreads) k_lanczos(Work w) {
  cg::grid_group g = cg::this_grid();
  const int m = w.m, n = w.n;
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  __shared__ double sa[128], sb[128];
  int slot = 0;
  long long cg_total = 0;
  // start: q0 = T s for a pseudo-random s on the DOFs (lands in range(T))
  for (size_t k = tid; k < (size_t)m; k += stride) w.u[k] = w.dof[k] ? start_value((int)k) : 0.0;
  g.sync();
  for (size_t k = tid; k < (size_t)m; k += stride)
    w.r[k] = w.dof[k] ? row_apply(w.Kr, w.u, (int)k, n) : 0.0;
  g.sync();
  cg_total += cg_solve(w, g, slot);
  // normalise in M': q0 = x / sqrt(x . M' x)
  double* Q = w.Q;
  double* MQ = w.MQ;
  {
    double v[2] = {0.0, 0.0};
    for (size_t k = tid; k < (size_t)m; k += stride)
      if (w.dof[k]) v[0] += w.wgt * w.x[k];
    grid_sum<1>(w, g, v, slot);
    const double wx = v[0];
    double xm[1] = {0.0};
    for (size_t k = tid; k < (size_t)m; k += stride) {
      double mq = 0.0;
      if (w.dof[k]) mq = row_apply(w.Mr, w.x, (int)k, n) + w.wgt * wx;
      MQ[k] = mq;
      xm[0] += w.x[k] * mq;
    }
    grid_sum<1>(w, g, xm, slot);
    const double s = 1.0 / sqrt(xm[0]);
    for (size_t k = tid; k < (size_t)m; k += stride) {
      Q[k] = w.x[k] * s;
      MQ[k] *= s;
    }
    g.sync();
  }
  double theta = 0.0, prev = -1.0;
  int steps = 0, stable = 0;
  double beta_last = 0.0;
  for (int j = 0; j < w.kmax; ++j) {
    double* qj = Q + (size_t)j * m;
    // r = K q_j, alpha = q_j . K q_j
    double al[1] = {0.0};
    for (size_t k = tid; k < (size_t)m; k += stride) {
      const double rk = w.dof[k] ? row_apply(w.Kr, qj, (int)k, n) : 0.0;
      w.r[k] = rk;
      al[0] += rk * qj[k];
    }
    grid_sum<1>(w, g, al, slot);
    if (threadIdx.x == 0) sa[j] = al[0];
    // x = T q_j
    cg_total += cg_solve(w, g, slot);
    // u = x - alpha q_j - beta q_{j-1}, then M'-orthogonalise against all q_i
    for (size_t k = tid; k < (size_t)m; k += stride) {
      double uk = w.x[k] - al[0] * qj[k];
      if (j > 0) uk -= sb[j - 1] * Q[(size_t)(j - 1) * m + k];
      w.u[k] = uk;
    }
    g.sync();
    for (int pass = 0; pass < 2; ++pass)
      for (int i = 0; i <= j; ++i) {
        double c[1] = {0.0};
        for (size_t k = tid; k < (size_t)m; k += stride) c[0] += MQ[(size_t)i * m + k] * w.u[k];
        grid_sum<1>(w, g, c, slot);
        for (size_t k = tid; k < (size_t)m; k += stride) w.u[k] -= c[0] * Q[(size_t)i * m + k];
        g.sync();
      }
    // beta = sqrt(u . M' u)
    double wu[1] = {0.0};
    for (size_t k = tid; k < (size_t)m; k += stride)
      if (w.dof[k]) wu[0] += w.wgt * w.u[k];
    grid_sum<1>(w, g, wu, slot);
    double um[1] = {0.0};
    double* qn = Q + (size_t)(j + 1) * m;
    double* mqn = MQ + (size_t)(j + 1) * m;
    for (size_t k = tid; k < (size_t)m; k += stride) {
      double mu = 0.0;
      if (w.dof[k]) mu = row_apply(w.Mr, w.u, (int)k, n) + w.wgt * wu[0];
      mqn[k] = mu;
      um[0] += w.u[k] * mu;
    }
    grid_sum<1>(w, g, um, slot);
    const double beta = sqrt(fmax(um[0], 0.0));
    if (threadIdx.x == 0) sb[j] = beta;
    __syncthreads();
    steps = j + 1;
    beta_last = beta;
    theta = tridiag_max(sa, sb, j + 1);
    // converged: the largest Ritz value stable to 1e-14 over 3 steps, or an
    // invariant subspace
    stable = fabs(theta - prev) <= 1e-14 * fabs(theta) ? stable + 1 : 0;
    prev = theta;
    if (stable >= 3 || !(beta > 1e-13 * fabs(theta))) break;
    const double s = 1.0 / beta;
    for (size_t k = tid; k < (size_t)m; k += stride) {
      qn[k] = w.u[k] * s;
      mqn[k] *= s;
    }
    g.sync();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    w.out[0] = theta;
    w.out[1] = steps;
    w.out[2] = (double)cg_total;
    w.out[3] = beta_last;
  }
}

}  // namespace

void launch_cut_pencil(const double* psi_s, int n, const int* list, int ncut,
                       const uint8_t* nmask, double* S, double* Kn, cudaStream_t st) {
  if (ncut)
    k_cut_pencil<<<(ncut + 127) / 128, 128, 0, st>>>(psi_s, n, list, ncut, nmask, S, Kn);
}

void launch_pencil_rows(int n, const uint8_t* cls, const int* cell_cut, const double* S,
                        const double* Kn, double* Mr, double* Kr, uint8_t* dof, cudaStream_t st) {
  const int m = (n + 1) * (n + 1);
  k_pencil_rows<<<(m + 255) / 256, 256, 0, st>>>(n, cls, cell_cut, S, Kn, Mr, Kr, dof);
}

size_t lanczos_doubles(int n, int kmax, int blocks) {
  const size_t m = (size_t)(n + 1) * (n + 1);
  return (size_t)(2 * (kmax + 2) + 6) * m + (size_t)3 * blocks * kRed + 4;
}

cudaError_t lanczos_blocks(int n, int* blocks) {
  int dev = 0, nsm = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_lanczos, kThreads, 0);
  if (e != cudaSuccess) return e;
  const int m = (n + 1) * (n + 1);
  int want = (m + kThreads - 1) / kThreads;
  const int cap = nsm * (per > 0 ? per : 1);
  *blocks = want < 1 ? 1 : want > cap ? cap : want;
  return cudaSuccess;
}

cudaError_t launch_lanczos(int n, const double* Mr, const double* Kr, const uint8_t* dof,
                           int ndof, double* work, int kmax, int cg_max, double cg_tol,
                           int blocks, double* out, cudaStream_t st) {
  const size_t m = (size_t)(n + 1) * (n + 1);
  Work w;
  w.n = n;
  w.m = (int)m;
  w.Mr = Mr;
  w.Kr = Kr;
  w.dof = dof;
  w.wgt = 1.0 / sqrt((double)ndof);
  w.Q = work;
  w.MQ = w.Q + (size_t)(kmax + 2) * m;
  w.x = w.MQ + (size_t)(kmax + 2) * m;
  w.r = w.x + m;
  w.z = w.r + m;
  w.p = w.z + m;
  w.q = w.p + m;
  w.u = w.q + m;
  w.part = w.u + m;
  w.out = out;
  w.kmax = kmax;
  w.cg_max = cg_max;
  w.cg_tol = cg_tol;
  void* args[] = {&w};
  return cudaLaunchCooperativeKernel((const void*)k_lanczos, dim3(blocks), dim3(kThreads), args,
                                     0, st);
}

// binds the bounds-checked build's device error word (see common.cuh)
MG_BOUNDS_BINDER(bind_bounds_global)
