// Fused smoothing step for the intermediate levels (see fused.cu).
#pragma once

#include "common.cuh"

template <class T> struct FusedArgs {
  Layout L;                 // this level
  const uint16_t* code;
  const int* tile_base;
  const T* rows;
  int n_rows;               // rows in the table
  const int* tiles;         // tiles to process
  const int* loff;          // [5 tile id ..] group offsets of the region lists
  const int2* lent;         // region boundary nodes {x | y << 16, row}
  int eta;
  const T* uin;             // u before the step (unused when starting from 0)
  T* uout;                  // u after the step
  const T* F;
  Layout Lc;                // next coarser level (prolongation source / restriction target)
  const T* ec;              // coarse correction to prolongate
  T* Fc;                    // restricted residual
};

int fused_halo(int eta);
size_t fused_smem_bytes(int eta, size_t elem);
template <class T> cudaError_t configure_fused(size_t smem);
template <class T>
void launch_smooth_step(const FusedArgs<T>& a, int ntiles, bool zero_in, bool prolong,
                        bool restrict_, size_t smem, cudaStream_t st);
