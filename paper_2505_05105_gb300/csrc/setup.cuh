// Setup-kernel launchers (see setup.cu).
#pragma once

#include "common.cuh"

// Cells of one level: class per cell (n x n, row-major [jc][ic]), the index of
// each cut cell in the compacted cut list (-1 otherwise) and the cut cells'
// 4x4 element matrices (16 doubles each, local order v0..v3).
struct CellData {
  int n;
  const uint8_t* cls;
  const int* cell_cut;
  const double* Ke;
  int box = 0;       // nodes on the box sides are strong Dirichlet nodes (not DOFs)
};

// out: the nodal values at every step-th node (n_out = n_in / step cells)
void launch_subsample(const double* in, int n_in, int step, double* out, int n_out,
                      cudaStream_t st);
// box != 0: the domain may reach the box sides (strong Dirichlet there)
void launch_snap(const double* psi, double* psi_s, int n, double thr, unsigned* err,
                 cudaStream_t st, int box = 0);
void launch_cell_class(const double* psi_s, int n, uint8_t* cls, uint8_t* cut_flag,
                       cudaStream_t st);
void launch_fill_int(int* p, size_t m, int v, cudaStream_t st);
void launch_scatter_cut_id(const int* list, int ncut, int* cell_cut, cudaStream_t st);
// nmask (n x n cells, may be null): nonzero marks a cut cell whose boundary
// piece is Neumann; Nk (16 per cut cell, may be null) gets its Neumann load;
// ch_global >= 0 sets lambda = gamma ch_global / h on every cut cell
void launch_cut_cells(const double* psi_s, int n, double h, double gamma, const int* list,
                      int ncut, double* Ke, double* Mk, double* Gk, double* Cl, int* cfg,
                      const uint8_t* nmask, double* Nk, cudaStream_t st,
                      double ch_global = -1.0);
void launch_tile_counts(const CellData& cd, const Layout& L, int* tile_cnt, uint8_t* tile_active,
                        int* ndof, cudaStream_t st);
void launch_tile_assemble(const CellData& cd, const Layout& L, const int* tile_base,
                          uint16_t* code, double* rows, int* bnode, unsigned* err,
                          cudaStream_t st);
void launch_band_flags(const int* bnode, int nb, int nbx, uint8_t* flag, cudaStream_t st);
// Boundary-node lists of tile regions (see k_region_list): 5 groups per
// tile (colours 0..3 off the rim, then the rim), entries {x | y << 16, row}.
void launch_region_list(const Layout& L, const uint16_t* code, const int* tile_base,
                        const int* tiles, int ntl, int tpr, int tw, int th, int H, int* cnt,
                        const int* off, int2* ent, cudaStream_t st);
void launch_restrict_tile_flags(const Layout& Lf, const Layout& Lc, const uint16_t* code_c,
                                uint8_t* flag, cudaStream_t st);
void launch_coarse_class(const uint8_t* fcls, int nf, uint8_t* ccls, uint8_t* cut_flag,
                         cudaStream_t st);
void launch_coarse_cut(const CellData& fine, const int* clist, int ncut, int nc, double* Ke,
                       cudaStream_t st);
void launch_coarsest(const CellData& cd, double* A, double* Ainv, unsigned* err, cudaStream_t st);
void launch_rows_to_f32(const double* r64, float* r32, size_t m, cudaStream_t st);
