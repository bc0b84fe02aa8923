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
  const int* active;     // active tiles of the fine level
  int n_active;
  int N;
  int device;            // the device the handle was set up on
  cudaStream_t st;
};

int mg_internal_fine_view(mg_handle h, FineOpView* out);
