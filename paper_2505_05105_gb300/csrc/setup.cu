// Setup kernels: snapping and classification (Sec. 2), cut-cell element
// matrices and local stabilisation (Sec. 5.2), per-node operator rows,
// Galerkin coarse levels (Eq. galerkin read as R A P with R = P^T, Sec. 5.1)
// and the coarsest-level inverse.
#include "setup.cuh"
#include "cutcell.cuh"

namespace {

// Q1 stiffness of a whole cell (h-independent in 2D), local order
// v0 (0,0), v1 (1,0), v2 (0,1), v3 (1,1).
__device__ __constant__ double kQ1[16] = {
    4.0 / 6, -1.0 / 6, -1.0 / 6, -2.0 / 6,
   -1.0 / 6,  4.0 / 6, -2.0 / 6, -1.0 / 6,
   -1.0 / 6, -2.0 / 6,  4.0 / 6, -1.0 / 6,
   -2.0 / 6, -1.0 / 6, -1.0 / 6,  4.0 / 6};

__global__ void k_snap(const double* __restrict__ psi, double* __restrict__ psi_s, int n,
                       double thr, unsigned* err, int box) {
  size_t m = (size_t)(n + 1) * (n + 1);
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m;
       k += (size_t)gridDim.x * blockDim.x) {
    double p = psi[k];
    if (!isfinite(p)) atomicOr(err, DEV_ERR_NAN);
    if (p < 0.0 && p > -thr) p = 0.0;          // snapping back to grid
    psi_s[k] = p;
    int i = (int)(k % (n + 1)), j = (int)(k / (n + 1));
    if (!box && (i == 0 || j == 0 || i == n || j == n) && p < 0.0) atomicOr(err, DEV_ERR_EDGE);
  }
}

__global__ void k_cell_class(const double* __restrict__ psi_s, int n, uint8_t* __restrict__ cls,
                             uint8_t* __restrict__ cut_flag) {
  size_t m = (size_t)n * n;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < m;
       c += (size_t)gridDim.x * blockDim.x) {
    int ic = (int)(c % n), jc = (int)(c / n);
    size_t k0 = (size_t)jc * (n + 1) + ic;
    int nin = (psi_s[k0] < 0.0) + (psi_s[k0 + 1] < 0.0) + (psi_s[k0 + n + 1] < 0.0) +
              (psi_s[k0 + n + 2] < 0.0);
    uint8_t v = nin == 4 ? CELL_INT : (nin == 0 ? CELL_EXT : CELL_CUT);
    cls[c] = v;
    cut_flag[c] = v == CELL_CUT;
  }
}

__global__ void k_fill_int(int* p, size_t m, int v) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m;
       k += (size_t)gridDim.x * blockDim.x)
    p[k] = v;
}

__global__ void k_scatter_cut_id(const int* __restrict__ list, int ncut, int* __restrict__ cell_cut) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < ncut) cell_cut[list[t]] = t;
}

__global__ void k_cut_cells(const double* __restrict__ psi_s, int n, double h, double gamma,
                            const int* __restrict__ list, int ncut, double* __restrict__ Ke,
                            double* __restrict__ Mk, double* __restrict__ Gk, double* __restrict__ Cl,
                            int* __restrict__ cfg, const uint8_t* __restrict__ nmask,
                            double* __restrict__ Nk, double ch_global) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncut) return;
  int c = list[t];
  int ic = c % n, jc = c / n;
  size_t k0 = (size_t)jc * (n + 1) + ic;
  double psi[4] = {psi_s[k0], psi_s[k0 + 1], psi_s[k0 + n + 1], psi_s[k0 + n + 2]};
  cutcell::CellOut o;
  cutcell::cut_cell_matrices(psi, h, gamma, o, nmask != nullptr && nmask[c] != 0, ch_global);
  for (int k = 0; k < 16; ++k) {
    Ke[(size_t)t * 16 + k] = o.Ke[k];
    Mk[(size_t)t * 16 + k] = o.Mk[k];
    Gk[(size_t)t * 16 + k] = o.Gk[k];
    if (Nk) Nk[(size_t)t * 16 + k] = o.Nk[k];
  }
  Cl[(size_t)t * 4 + 0] = o.C;
  Cl[(size_t)t * 4 + 1] = o.lam;
  Cl[(size_t)t * 4 + 2] = o.area;
  Cl[(size_t)t * 4 + 3] = o.length;
  cfg[t] = o.config;
}

// Element matrix of cell (ic, jc) of a level, or nullptr-equivalent (false).
__device__ __forceinline__ bool cell_matrix(const CellData& cd, int ic, int jc, const double** E) {
  if (ic < 0 || jc < 0 || ic >= cd.n || jc >= cd.n) return false;
  size_t c = (size_t)jc * cd.n + ic;
  uint8_t v = cd.cls[c];
  if (v == CELL_EXT) return false;
  if (v == CELL_INT) { *E = kQ1; return true; }
  *E = cd.Ke + (size_t)cd.cell_cut[c] * 16;
  return true;
}

// DOF / interior / boundary status of node (i, j) from its adjacent cells.
__device__ __forceinline__ int node_kind(const CellData& cd, int i, int j) {
  if (i < 0 || j < 0 || i > cd.n || j > cd.n) return 0;
  if (cd.box && (i == 0 || j == 0 || i == cd.n || j == cd.n)) return 0;   // strong Dirichlet
  int nact = 0, nint = 0;
  for (int q = 0; q < 4; ++q) {
    int ic = i - 1 + (q & 1), jc = j - 1 + (q >> 1);
    if (ic < 0 || jc < 0 || ic >= cd.n || jc >= cd.n) continue;
    uint8_t v = cd.cls[(size_t)jc * cd.n + ic];
    nact += v != CELL_EXT;
    nint += v == CELL_INT;
  }
  if (nact == 0) return 0;       // not a DOF
  if (nint == 4) return 1;       // interior: constant stencil
  return 2;                      // boundary: vertex of a cut cell
}

constexpr int kTileThreads = 256;
constexpr int kPerThread = MG_TX * MG_TY / kTileThreads;   // 8

// Pass 1: per tile, count boundary nodes, flag tiles with DOFs.
__global__ void k_tile_counts(CellData cd, Layout L, int* __restrict__ tile_cnt,
                              uint8_t* __restrict__ tile_active, int* __restrict__ ndof) {
  int t = blockIdx.x;
  int ti = t % L.ntx, tj = t / L.ntx;
  int nb = 0, nd = 0;
  for (int k = 0; k < kPerThread; ++k) {
    int l = threadIdx.x * kPerThread + k;
    int i = ti * MG_TX + (l % MG_TX), j = tj * MG_TY + (l / MG_TX);
    int kind = node_kind(cd, i, j);
    nb += kind == 2;
    nd += kind != 0;
  }
  __shared__ int s_b[kTileThreads / 32], s_d[kTileThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    nb += __shfl_xor_sync(0xffffffffu, nb, o);
    nd += __shfl_xor_sync(0xffffffffu, nd, o);
  }
  if ((threadIdx.x & 31) == 0) { s_b[threadIdx.x >> 5] = nb; s_d[threadIdx.x >> 5] = nd; }
  __syncthreads();
  if (threadIdx.x == 0) {
    int B = 0, D = 0;
    for (int w = 0; w < kTileThreads / 32; ++w) { B += s_b[w]; D += s_d[w]; }
    tile_cnt[t] = B;
    tile_active[t] = D > 0;
    if (D) atomicAdd(ndof, D);
  }
}

// Pass 2: codes, boundary rows (fp64) and boundary node positions.
__global__ void k_tile_assemble(CellData cd, Layout L, const int* __restrict__ tile_base,
                                uint16_t* __restrict__ code, double* __restrict__ rows,
                                int* __restrict__ bnode, unsigned* err) {
  int t = blockIdx.x;
  int ti = t % L.ntx, tj = t / L.ntx;
  int kinds[kPerThread];
  int nb = 0;
  for (int k = 0; k < kPerThread; ++k) {
    int l = threadIdx.x * kPerThread + k;
    int i = ti * MG_TX + (l % MG_TX), j = tj * MG_TY + (l / MG_TX);
    kinds[k] = node_kind(cd, i, j);
    nb += kinds[k] == 2;
  }
  // exclusive scan of nb over the block (raster order within the tile)
  __shared__ int s_w[kTileThreads / 32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = nb;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  int off = 0;
  for (int q = 0; q < w; ++q) off += s_w[q];
  int rank = off + x - nb;
  int base = tile_base[t];
  for (int k = 0; k < kPerThread; ++k) {
    int l = threadIdx.x * kPerThread + k;
    int i = ti * MG_TX + (l % MG_TX), j = tj * MG_TY + (l / MG_TX);
    uint16_t cv = 0;
    if (kinds[k] == 1) cv = 1;
    if (kinds[k] == 2) {
      if (rank + 2 > 65535) { atomicOr(err, DEV_ERR_TILE); rank++; continue; }
      cv = (uint16_t)(2 + rank);
      int r = base + rank;
      double row[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      // adjacent cells in a fixed order; node is vertex (1-dx) + 2 (1-dy)
      for (int q = 0; q < 4; ++q) {
        int dx = q & 1, dy = q >> 1;
        int ic = i - 1 + dx, jc = j - 1 + dy;
        const double* E;
        if (!cell_matrix(cd, ic, jc, &E)) continue;
        int a = (1 - dx) + 2 * (1 - dy);
        for (int b = 0; b < 4; ++b) {
          int bi = ic + (b & 1) - i, bj = jc + (b >> 1) - j;   // in {-1,0,1}
          row[(bi + 1) + 3 * (bj + 1)] += E[a * 4 + b];
        }
      }
      for (int s = 0; s < 9; ++s) rows[(size_t)r * MG_ROW + s] = row[s];
      rows[(size_t)r * MG_ROW + 9] = 1.0 / row[4];
      bnode[r] = i | (j << 16);
      ++rank;
    }
    if (i <= L.n + MG_TX && j <= L.n + MG_TY) code[L.idx(i, j)] = cv;
  }
}

// Flag the fine tiles whose 32 x 16 block of coarse nodes holds a coarse DOF
// (a superset of the active fine tiles: a fine DOF at (i, j) makes the coarse
// node (i/2, j/2) a DOF); the fused restriction runs on these tiles so that
// every coarse DOF receives its restricted residual.
__global__ void k_restrict_tile_flags(Layout Lf, Layout Lc, const uint16_t* __restrict__ code_c,
                                      uint8_t* __restrict__ flag) {
  int t = blockIdx.x;
  int tx = t % Lf.ntx, ty = t / Lf.ntx;
  int any = 0;
  for (int k = threadIdx.x; k < (MG_TX / 2) * (MG_TY / 2); k += blockDim.x) {
    int I = tx * (MG_TX / 2) + k % (MG_TX / 2), J = ty * (MG_TY / 2) + k / (MG_TX / 2);
    if (I <= Lc.n && J <= Lc.n && code_c[Lc.idx(I, J)] != 0) any = 1;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) flag[t] = any ? 1 : 0;
}

// Flag the 32 x 32 band tiles containing boundary nodes.
__global__ void k_band_flags(const int* __restrict__ bnode, int nb, int nbx, uint8_t* __restrict__ flag) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nb) return;
  int p = bnode[r];
  int i = p & 0xffff, j = p >> 16;
  flag[(j >> 5) * nbx + (i >> 5)] = 1;
}

// Boundary-node lists of tile regions.  For tile b (tw x th nodes, tpr tiles
// per row; tiles[b] or, if tiles is null, b itself) and its region of halo
// H, every vertex of a cut cell in the region is listed once, grouped: the
// four colours (i mod 2) + 2 (j mod 2) off the region's rim, then the rim
// nodes (read by the sweeps, never updated).  Entry: {x | y << 16 (region
// coordinates), boundary row index}.  First pass (ent == nullptr): counts
// per group into cnt[5 b ..]; second pass: fills from the offsets
// off[5 b ..] (exclusive scan of the counts).  The order inside a group is
// immaterial: nodes of one colour never interact.
__global__ void k_region_list(Layout L, const uint16_t* __restrict__ code,
                              const int* __restrict__ tile_base, const int* __restrict__ tiles,
                              int tpr, int tw, int th, int H, int* __restrict__ cnt,
                              const int* __restrict__ off, int2* __restrict__ ent) {
  __shared__ int c5[5];
  const int b = blockIdx.x, t = tiles ? tiles[b] : b;
  const int ri0 = (t % tpr) * tw - H, rj0 = (t / tpr) * th - H;
  const int RX = tw + 2 * H, RY = th + 2 * H;
  if (threadIdx.x < 5) c5[threadIdx.x] = ent ? off[5 * b + threadIdx.x] : 0;
  __syncthreads();
  for (int p = threadIdx.x; p < RX * RY; p += blockDim.x) {
    const int y = p / RX, x = p - y * RX;
    const int gi = ri0 + x, gj = rj0 + y;
    if (gi < 0 || gj < 0 || gi > L.n || gj > L.n) continue;
    const uint16_t cd = code[L.idx(gi, gj)];
    if (cd < 2) continue;
    const bool rim = x == 0 || y == 0 || x == RX - 1 || y == RY - 1;
    const int g = rim ? 4 : (gi & 1) + 2 * (gj & 1);
    const int pos = atomicAdd(&c5[g], 1);
    if (ent) ent[pos] = make_int2(x | (y << 16), tile_base[L.tile_of(gi, gj)] + cd - 2);
  }
  __syncthreads();
  if (!ent && threadIdx.x < 5) cnt[5 * b + threadIdx.x] = c5[threadIdx.x];
}

// Coarse cell classes from the four children (Sec. 5.1 hierarchy).
__global__ void k_coarse_class(const uint8_t* __restrict__ fcls, int nf, uint8_t* __restrict__ ccls,
                               uint8_t* __restrict__ cut_flag) {
  int nc = nf / 2;
  size_t m = (size_t)nc * nc;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < m;
       c += (size_t)gridDim.x * blockDim.x) {
    int I = (int)(c % nc), J = (int)(c / nc);
    int nint = 0, next = 0;
    for (int q = 0; q < 4; ++q) {
      uint8_t v = fcls[(size_t)(2 * J + (q >> 1)) * nf + 2 * I + (q & 1)];
      nint += v == CELL_INT;
      next += v == CELL_EXT;
    }
    uint8_t v = nint == 4 ? CELL_INT : (next == 4 ? CELL_EXT : CELL_CUT);
    ccls[c] = v;
    cut_flag[c] = v == CELL_CUT;
  }
}

// Element-wise Galerkin product for coarse cut cells:
// Ke_C = P_C^T (sum of the children's element matrices on the 3x3 fine
// nodes of C) P_C, P_C the bilinear weights (1, 1/2, 1/4) of Sec. 5.1.
__global__ void k_coarse_cut(CellData fine, const int* __restrict__ clist, int ncut, int nc,
                             double* __restrict__ Ke) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncut) return;
  int c = clist[t];
  int I = c % nc, J = c / nc;
  double K9[9][9];
  for (int a = 0; a < 9; ++a)
    for (int b = 0; b < 9; ++b) K9[a][b] = 0.0;
  for (int q = 0; q < 4; ++q) {
    int cx = q & 1, cy = q >> 1;
    const double* E;
    if (!cell_matrix(fine, 2 * I + cx, 2 * J + cy, &E)) continue;
    for (int a = 0; a < 4; ++a) {
      int fa = (cx + (a & 1)) + 3 * (cy + (a >> 1));
      for (int b = 0; b < 4; ++b) {
        int fb = (cx + (b & 1)) + 3 * (cy + (b >> 1));
        K9[fa][fb] += E[a * 4 + b];
      }
    }
  }
  // w(f, X): weight of coarse vertex coordinate X in {0,1} at fine coordinate f in {0,1,2}
  double Pw[9][4];
  for (int f = 0; f < 9; ++f) {
    int fx = f % 3, fy = f / 3;
    for (int A = 0; A < 4; ++A) {
      int X = A & 1, Y = A >> 1;
      double wx = X ? 0.5 * fx : 1.0 - 0.5 * fx;
      double wy = Y ? 0.5 * fy : 1.0 - 0.5 * fy;
      Pw[f][A] = wx * wy;
    }
  }
  double T9[9][4];
  for (int f = 0; f < 9; ++f)
    for (int B = 0; B < 4; ++B) {
      double s = 0.0;
      for (int g = 0; g < 9; ++g) s += K9[f][g] * Pw[g][B];
      T9[f][B] = s;
    }
  for (int A = 0; A < 4; ++A)
    for (int B = 0; B < 4; ++B) {
      double s = 0.0;
      for (int f = 0; f < 9; ++f) s += Pw[f][A] * T9[f][B];
      Ke[(size_t)t * 16 + A * 4 + B] = s;
    }
  for (int A = 0; A < 4; ++A)
    for (int B = A + 1; B < 4; ++B) {
      double v = 0.5 * (Ke[(size_t)t * 16 + A * 4 + B] + Ke[(size_t)t * 16 + B * 4 + A]);
      Ke[(size_t)t * 16 + A * 4 + B] = Ke[(size_t)t * 16 + B * 4 + A] = v;
    }
}

// Dense coarsest matrix (non-DOF rows/columns replaced by identity),
// Cholesky factorisation and explicit inverse; one block.
__global__ void k_coarsest(CellData cd, double* __restrict__ A, double* __restrict__ Ainv,
                           unsigned* err) {
  int n = cd.n, m = (n + 1) * (n + 1);
  for (int p = threadIdx.x; p < m * m; p += blockDim.x) A[p] = 0.0;
  __syncthreads();
  for (int p = threadIdx.x; p < m; p += blockDim.x) {
    int i = p % (n + 1), j = p / (n + 1);
    int kind = node_kind(cd, i, j);
    if (kind == 0) { A[(size_t)p * m + p] = 1.0; continue; }
    for (int q = 0; q < 4; ++q) {
      int dx = q & 1, dy = q >> 1;
      int ic = i - 1 + dx, jc = j - 1 + dy;
      const double* E;
      if (!cell_matrix(cd, ic, jc, &E)) continue;
      int a = (1 - dx) + 2 * (1 - dy);
      for (int b = 0; b < 4; ++b) {
        const int bi = ic + (b & 1), bj = jc + (b >> 1);
        // couplings to strong Dirichlet box nodes are not part of A
        if (cd.box && node_kind(cd, bi, bj) == 0) continue;
        int col = bi + bj * (n + 1);
        A[(size_t)p * m + col] += E[a * 4 + b];
      }
    }
  }
  __syncthreads();
  // right-looking Cholesky, lower triangle
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) {
      double d = A[(size_t)k * m + k];
      if (!(d > 0.0)) { bad = 1; d = 1.0; }
      A[(size_t)k * m + k] = sqrt(d);
    }
    __syncthreads();
    double dk = A[(size_t)k * m + k];
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) A[(size_t)i * m + k] /= dk;
    __syncthreads();
    int rem = m - k - 1;
    for (int p = threadIdx.x; p < rem * rem; p += blockDim.x) {
      int i = k + 1 + p / rem, j = k + 1 + p % rem;
      if (j <= i) A[(size_t)i * m + j] -= A[(size_t)i * m + k] * A[(size_t)j * m + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && bad) atomicOr(err, DEV_ERR_NOT_SPD);
  // inverse: column c solves L L^T x = e_c
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    double* x = Ainv + (size_t)c * m;     // column c stored contiguously (A^-1 symmetric)
    for (int i = 0; i < m; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= A[(size_t)i * m + k] * x[k];
      x[i] = s / A[(size_t)i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) {
      double s = x[i];
      for (int k = i + 1; k < m; ++k) s -= A[(size_t)k * m + i] * x[k];
      x[i] = s / A[(size_t)i * m + i];
    }
    // a node that is not a DOF gets u = 0 whatever F holds there (the unit
    // diagonal above only keeps the factorisation regular); F off the DOFs
    // can be nonzero when a coarse level is not the Galerkin one
    if (node_kind(cd, c % (n + 1), c / (n + 1)) == 0)
      for (int i = 0; i < m; ++i) x[i] = 0.0;
  }
}

__global__ void k_rows_to_f32(const double* __restrict__ r64, float* __restrict__ r32, size_t m) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m;
       k += (size_t)gridDim.x * blockDim.x)
    r32[k] = (float)r64[k];
}

inline int grid_for(size_t m, int threads = 256) {
  size_t b = (m + threads - 1) / threads;
  return (int)(b < 65536 * 8 ? (b ? b : 1) : 65536 * 8);
}

}  // namespace

// ------------------------------------------------------------------------------
// host launchers
// ------------------------------------------------------------------------------

// out[(J, I)] = in[(step J, step I)]: a coarse grid's nodal values of a
// level set given on the (n_in + 1)^2 fine nodes
__global__ void k_subsample(const double* __restrict__ in, int n_in, int step,
                            double* __restrict__ out, int n_out) {
  const size_t m = (size_t)(n_out + 1) * (n_out + 1);
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < m;
       k += (size_t)gridDim.x * blockDim.x) {
    const int I = (int)(k % (n_out + 1)), J = (int)(k / (n_out + 1));
    out[k] = in[(size_t)J * step * (n_in + 1) + (size_t)I * step];
  }
}

void launch_subsample(const double* in, int n_in, int step, double* out, int n_out,
                      cudaStream_t st) {
  k_subsample<<<grid_for((size_t)(n_out + 1) * (n_out + 1)), 256, 0, st>>>(in, n_in, step, out,
                                                                            n_out);
}

void launch_snap(const double* psi, double* psi_s, int n, double thr, unsigned* err,
                 cudaStream_t st, int box) {
  k_snap<<<grid_for((size_t)(n + 1) * (n + 1)), 256, 0, st>>>(psi, psi_s, n, thr, err, box);
}

void launch_cell_class(const double* psi_s, int n, uint8_t* cls, uint8_t* cut_flag,
                       cudaStream_t st) {
  k_cell_class<<<grid_for((size_t)n * n), 256, 0, st>>>(psi_s, n, cls, cut_flag);
}

void launch_fill_int(int* p, size_t m, int v, cudaStream_t st) {
  k_fill_int<<<grid_for(m), 256, 0, st>>>(p, m, v);
}

void launch_scatter_cut_id(const int* list, int ncut, int* cell_cut, cudaStream_t st) {
  if (ncut) k_scatter_cut_id<<<(ncut + 255) / 256, 256, 0, st>>>(list, ncut, cell_cut);
}

void launch_cut_cells(const double* psi_s, int n, double h, double gamma, const int* list,
                      int ncut, double* Ke, double* Mk, double* Gk, double* Cl, int* cfg,
                      const uint8_t* nmask, double* Nk, cudaStream_t st, double ch_global) {
  if (ncut)
    k_cut_cells<<<(ncut + 127) / 128, 128, 0, st>>>(psi_s, n, h, gamma, list, ncut, Ke, Mk, Gk,
                                                    Cl, cfg, nmask, Nk, ch_global);
}

void launch_tile_counts(const CellData& cd, const Layout& L, int* tile_cnt, uint8_t* tile_active,
                        int* ndof, cudaStream_t st) {
  k_tile_counts<<<L.ntx * L.nty, kTileThreads, 0, st>>>(cd, L, tile_cnt, tile_active, ndof);
}

void launch_tile_assemble(const CellData& cd, const Layout& L, const int* tile_base,
                          uint16_t* code, double* rows, int* bnode, unsigned* err,
                          cudaStream_t st) {
  k_tile_assemble<<<L.ntx * L.nty, kTileThreads, 0, st>>>(cd, L, tile_base, code, rows, bnode,
                                                         err);
}

void launch_band_flags(const int* bnode, int nb, int nbx, uint8_t* flag, cudaStream_t st) {
  if (nb) k_band_flags<<<(nb + 255) / 256, 256, 0, st>>>(bnode, nb, nbx, flag);
}

void launch_region_list(const Layout& L, const uint16_t* code, const int* tile_base,
                        const int* tiles, int ntl, int tpr, int tw, int th, int H, int* cnt,
                        const int* off, int2* ent, cudaStream_t st) {
  if (ntl)
    k_region_list<<<ntl, 256, 0, st>>>(L, code, tile_base, tiles, tpr, tw, th, H, cnt, off, ent);
}

void launch_restrict_tile_flags(const Layout& Lf, const Layout& Lc, const uint16_t* code_c,
                                uint8_t* flag, cudaStream_t st) {
  k_restrict_tile_flags<<<Lf.ntx * Lf.nty, 256, 0, st>>>(Lf, Lc, code_c, flag);
}

void launch_coarse_class(const uint8_t* fcls, int nf, uint8_t* ccls, uint8_t* cut_flag,
                         cudaStream_t st) {
  k_coarse_class<<<grid_for((size_t)(nf / 2) * (nf / 2)), 256, 0, st>>>(fcls, nf, ccls, cut_flag);
}

void launch_coarse_cut(const CellData& fine, const int* clist, int ncut, int nc, double* Ke,
                       cudaStream_t st) {
  if (ncut) k_coarse_cut<<<(ncut + 127) / 128, 128, 0, st>>>(fine, clist, ncut, nc, Ke);
}

void launch_coarsest(const CellData& cd, double* A, double* Ainv, unsigned* err, cudaStream_t st) {
  k_coarsest<<<1, 256, 0, st>>>(cd, A, Ainv, err);
}

void launch_rows_to_f32(const double* r64, float* r32, size_t m, cudaStream_t st) {
  if (m) k_rows_to_f32<<<grid_for(m), 256, 0, st>>>(r64, r32, m);
}

// binds the bounds-checked build's device error word (see common.cuh)
MG_BOUNDS_BINDER(bind_bounds_setup)
