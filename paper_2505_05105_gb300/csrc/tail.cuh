// Single-block V-cycle on the smallest levels (see tail.cu).
#pragma once

#include "common.cuh"

#define MG_TAIL_MAX_LEVELS 6
#define MG_TAIL_MAX_N 64      // largest top level the tail block handles

template <class T> struct TailArgs {
  int nlev;                                   // levels, the last solved exactly
  int n[MG_TAIL_MAX_LEVELS];                  // cells per side, halving
  Layout L[MG_TAIL_MAX_LEVELS];
  const uint16_t* code[MG_TAIL_MAX_LEVELS];
  const int* tile_base[MG_TAIL_MAX_LEVELS];
  const T* rows[MG_TAIL_MAX_LEVELS];
  int n_bnd[MG_TAIL_MAX_LEVELS];              // boundary rows per level
  int rows_in_smem;                           // stage every level's rows in shared memory
  const double* Ainv;                         // coarsest inverse, m x m, by columns
  const T* F0;                                // right-hand side of the top level
  T* u0;                                      // top level u: initial guess (load_u0) / result
  int load_u0;
  int eta, nu1, nu2;
};

size_t tail_smem_bytes(const int* n, int nlev, size_t elem);
size_t tail_rows_bytes(const int* n_bnd, int nlev, size_t elem);
size_t tail_list_bytes(const int* n_bnd, int nlev);
template <class T> cudaError_t configure_tail(size_t smem);
template <class T> void launch_tail(const TailArgs<T>& a, size_t smem, cudaStream_t st);
