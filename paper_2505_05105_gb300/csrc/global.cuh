// The global stabilisation constant of Sec. 5.2 (see global.cu).
#pragma once

#include "common.cuh"

// per cut cell of a level with n cells per side (cell units, h = 1): the
// volume stiffness S and the normal-derivative matrix Kn (zero on cells
// nmask marks Neumann), 16 doubles each
void launch_cut_pencil(const double* psi_s, int n, const int* list, int ncut,
                       const uint8_t* nmask, double* S, double* Kn, cudaStream_t st);
// 9-point rows of the global pencil's M and K over the (n+1)^2 nodes and the
// DOF mask (vertices of active cells)
void launch_pencil_rows(int n, const uint8_t* cls, const int* cell_cut, const double* S,
                        const double* Kn, double* Mr, double* Kr, uint8_t* dof, cudaStream_t st);
// cooperative grid size for the Lanczos kernel
cudaError_t lanczos_blocks(int n, int* blocks);
// doubles of work space the Lanczos kernel needs
size_t lanczos_doubles(int n, int kmax, int blocks);
// Lambda_max(K, M + w w^T) (cell units) into out[0]; out[1] Lanczos steps,
// out[2] conjugate-gradient iterations in total, out[3] the last beta;
// kmax <= 100 Lanczos steps
cudaError_t launch_lanczos(int n, const double* Mr, const double* Kr, const uint8_t* dof,
                           int ndof, double* work, int kmax, int cg_max, double cg_tol,
                           int blocks, double* out, cudaStream_t st);
