// V-cycle kernel launchers (see cycle.cu).
#pragma once

#include "tma.cuh"

// Operator of one level for kernels in arithmetic type T.
template <class T> struct OpArgs {
  Layout L;
  const uint16_t* code;      // per node, padded layout
  const int* tile_base;      // per tile: first boundary row
  const T* rows;             // boundary rows, MG_ROW values each
  int n_rows;                // rows in the table
};

// Level-0 data for the right-hand side F = M f + G g.
struct RhsArgs {
  Layout L;
  double h;
  const uint16_t* code;
  const uint8_t* cls;        // n x n cell classes
  const int* cell_cut;       // n x n, index into the cut list or -1
  const double* Mk;          // 16 per cut cell, mass on K cap Omega_h
  const double* Gk;          // 16 per cut cell, Dirichlet load (0 on Neumann cells)
  const double* Nk = nullptr;  // 16 per cut cell, Neumann load (null: no Neumann cells)
  const double* gN = nullptr;  // nodal Neumann data, user layout (null: g_N = 0)
  const double* Ke = nullptr;  // 16 per cut cell, element matrices (strong box sides)
  int box = 0;                 // box nodes are strong Dirichlet nodes: F -= A_pq g_q
  unsigned* err = nullptr;     // gets DEV_ERR_NAN where an F value is not finite
};

// TMA descriptors of a level's two u buffers in one precision (band kernel box)
struct BandMaps {
  CUtensorMap u[2];
};
int band_box_x(int eta);
int band_box_y(int eta);

template <class T> size_t sweep_smem();
template <class T> size_t band_smem(int eta);
template <class T> cudaError_t configure_kernels(int eta);

// load modes of a sweep: u as stored, u = 0, u + P e_2h (Sec. 5.1)
enum SweepMode : int { kSweepPlain = 0, kSweepZero = 1, kSweepProlong = 2 };

template <class T>
// One 4-colour sweep; ec != nullptr adds the prolongated coarse correction
// P ec (coarse layout *Lc) to uin while loading.  (The fp32 sweep is
// launch_gs_sweep_f32.)
void launch_gs_sweep(const OpArgs<T>& op, const int* tiles, int ntiles, const T* uin, T* uout,
                     const T* F, T* bval, bool zero_in, const Layout* Lc, const T* ec,
                     cudaStream_t st);

// The fp32 sweep (sweep32.cu): launch_gs_sweep's arguments plus the tiles'
// region lists of boundary nodes (5 group offsets per listed tile, entries
// {x | y << 16, row} in region coordinates of a 64 x 32 tile with a 4-node
// halo; see build_region_lists).  touch (or nullptr): per tile of the list,
// whether its region holds a node the directly preceding band kernel writes
// (launch_touch_flags, TOUCH_SWEEP; TOUCH_PROLONG when ec is given); blocks
// of untouched tiles skip the wait for that kernel.
void launch_gs_sweep_f32(const OpArgs<float>& op, const int* tiles, int ntiles, const float* uin,
                         float* uout, const float* F, float* bval, bool zero_in,
                         const Layout* Lc, const float* ec, const int* loff, const int2* lent,
                         const uint8_t* touch, cudaStream_t st);
template <class T>
void launch_band(const OpArgs<T>& op, const int* btiles, int nbt, int nbx, int eta, T* u,
                 const T* F, const T* bval, const int* boff, const int2* bent,
                 const BandMaps& maps, int umap, unsigned* err, unsigned wait_polls,
                 cudaStream_t st);
// The transposed smoothing step's kernels (fp64; the transposed V-cycle of
// the adjoint): a sweep with the colours in the reverse order, the snapshot
// of the boundary values the band kernel reads (bnode[r] = i | j << 16), and
// the band sweeps with the colours in the reverse order.
template <class T>
void launch_gs_sweep_rev(const OpArgs<T>& op, const int* tiles, int ntiles, const T* uin,
                         T* uout, const T* F, T* bval, cudaStream_t st);
template <class T>
void launch_gather_bval(const Layout& L, const int* bnode, int nb, const T* u, T* bval,
                        cudaStream_t st);
template <class T>
void launch_band_rev(const OpArgs<T>& op, const int* btiles, int nbt, int nbx, int eta, T* u,
                     const T* F, const T* bval, const int* boff, const int2* bent,
                     const BandMaps& maps, int umap, unsigned* err, unsigned wait_polls,
                     cudaStream_t st);
// touch (or nullptr): per block (4 per coarse tile), whether its fine
// region holds a node the directly preceding band kernel writes
// (launch_touch_flags, TOUCH_RESTRICT).
template <class T>
void launch_resid_restrict(const OpArgs<T>& op, const T* u, const T* F, const Layout& Lc,
                           const int* ctiles, int nct, T* Fc, double* norms, cudaStream_t st,
                           const uint8_t* touch = nullptr);
// Which blocks of a later launch read a boundary node (code >= 2) of the
// level with layout L and codes `code`, one flag per block:
//   TOUCH_SWEEP    tiles of L (ntx tpr), the fp32 sweep's region (4-node halo);
//   TOUCH_PROLONG  tiles of the next finer level (tpr its ntx), the coarse
//                  nodes of L that the prolongating sweep's region reads;
//   TOUCH_RESTRICT 4 blocks per coarse tile (tpr the coarse ntx), the fine
//                  region of L that a residual + restriction block reads.
// The fp32 version (restrict32.cu), which launch_resid_restrict<float> runs.
void launch_resid_restrict_f32(const OpArgs<float>& op, const float* u, const float* F,
                               const Layout& Lc, const int* ctiles, int nct, float* Fc,
                               double* norms, cudaStream_t st, const uint8_t* touch);
enum TouchMode : int { TOUCH_SWEEP = 0, TOUCH_PROLONG = 1, TOUCH_RESTRICT = 2 };
void launch_touch_flags(int mode, const Layout& L, const uint16_t* code, const int* tiles,
                        int tpr, int nblocks, uint8_t* flag, cudaStream_t st);
template <class T, class TR>
// norms[0] gets max |r| (atomic max); with l2 norms[1] gets sum r^2; rout
// (if given) gets scale r -- for an fp32 rout, scale must be a power of two
// (it is applied after the rounding to fp32).  part (ntiles doubles, or
// nullptr): the l2 sum is taken through per-block partial sums added in a
// fixed order, the same bits on every run (else by atomic adds).
void launch_residual(const OpArgs<T>& op, const int* tiles, int ntiles, const T* u, const T* F,
                     TR* rout, T scale, double* norms, cudaStream_t st, bool l2 = true,
                     double* part = nullptr);
template <class T>
void launch_prolong(const OpArgs<T>& op, const int* tiles, int ntiles, T* uf, const Layout& Lc,
                    const T* ec, cudaStream_t st);
template <class T>
void launch_coarse_solve(const Layout& Lc, const double* Ainv, const T* Fc, T* uc, cudaStream_t st);
void launch_rhs(const RhsArgs& a, const int* tiles, int ntiles, const double* f, const double* g,
                double* F, double* norms, cudaStream_t st);
// dLdf = M^T w, dLdg = G^T w, dLdn = N^T w (a.Nk) for w in the padded
// layout (any output may be null): the adjoint of launch_rhs
void launch_rhs_adj(const RhsArgs& a, const int* tiles, int ntiles, const double* w,
                    double* dLdf, double* dLdg, cudaStream_t st, double* dLdn = nullptr);
template <class T>
void launch_pack(const Layout& L, const uint16_t* code, const double* src, T* dst, unsigned* err,
                 cudaStream_t st, unsigned* nz = nullptr);
// box != 0: the box-side nodes are copied too (gradients on strong box nodes)
void launch_unpack(const Layout& L, const uint16_t* code, const double* src, double* dst,
                   cudaStream_t st, int box = 0);
// launch_unpack split in two: the listed (active) tiles, and zeros on the
// tiles without DOFs (`blocks` blocks striding over all tiles)
void launch_unpack_tiles(const Layout& L, const uint16_t* code, const int* tiles, int ntiles,
                         const double* src, double* dst, cudaStream_t st, int box = 0);
void launch_zero_inactive(const Layout& L, const uint8_t* tile_active, double* dst, int blocks,
                          cudaStream_t st);
// dst = (float)(src * scale) on the DOFs of the tiles (the refinement
// residual when u = 0: r = F); scale a power of two
void launch_scale_to_f32(const Layout& L, const int* tiles, int ntiles, const double* src,
                         float* dst, double scale, cudaStream_t st);
void launch_update(const Layout& L, const int* tiles, int ntiles, const uint16_t* code, double* u,
                   const float* e, double inv_scale, cudaStream_t st);
template <class T>
void launch_export_stencil(const OpArgs<T>& op, double* out, cudaStream_t st);
