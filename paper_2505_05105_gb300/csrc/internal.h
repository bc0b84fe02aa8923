// Internal (non-ABI) view of a handle's fine-level operator, for entry points
// implemented outside api.cu.
#pragma once

#include "common.cuh"
#include "ghostmg.h"

struct FineOpView {
  Layout L;
  const uint16_t* code;
  const int* tile_base;
  const double* rows64;
  int n_rows;            // boundary rows of the fine level
  const int* active;     // active tiles of the fine level
  int n_active;
  int N;
  int device;            // the device the handle was set up on
  cudaStream_t st;
};

int mg_internal_fine_view(mg_handle h, FineOpView* out);

// Bind the bounds-checked build's device error word to each translation unit
// (MG_BOUNDS_BINDER; no-ops in the normal build).
cudaError_t bind_bounds_api(unsigned* word);
cudaError_t bind_bounds_batch(unsigned* word);
cudaError_t bind_bounds_cycle(unsigned* word);
cudaError_t bind_bounds_fused(unsigned* word);
cudaError_t bind_bounds_global(unsigned* word);
cudaError_t bind_bounds_noalloc(unsigned* word);
cudaError_t bind_bounds_oned(unsigned* word);
cudaError_t bind_bounds_restrict32(unsigned* word);
cudaError_t bind_bounds_scan(unsigned* word);
cudaError_t bind_bounds_setup(unsigned* word);
cudaError_t bind_bounds_sweep32(unsigned* word);
cudaError_t bind_bounds_tail(unsigned* word);
cudaError_t bind_bounds_tma(unsigned* word);
