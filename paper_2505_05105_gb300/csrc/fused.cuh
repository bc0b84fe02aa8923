// Fused smoothing step for the intermediate levels (see fused.cu).
#pragma once

#include "tma.cuh"

template <class T> struct FusedArgs {
  Layout L;                 // this level
  const uint16_t* code;
  const int* tile_base;
  const T* rows;
  const int* tiles;         // tiles to process
  const int* loff;          // [5 tile id ..] group offsets of the region lists
  const int2* lent;         // region boundary nodes {x | y << 16, row}
  int eta;
  int uin_map;              // which of maps.u holds u before the step
  T* uout;                  // u after the step
  const T* F;
  Layout Lc;                // next coarser level (prolongation source / restriction target)
  const T* ec;              // coarse correction to prolongate
  T* Fc;                    // restricted residual
  unsigned* err;            // DEV_ERR_TIMEOUT if a TMA wait runs out
};

// TMA descriptors of the level's two u buffers, F and the codes (box
// fused_box_x x fused_box_y elements)
struct FusedMaps {
  CUtensorMap u[2];
  CUtensorMap F;
  CUtensorMap code;
};

int fused_box_x(int eta);
int fused_box_y(int eta);
int fused_halo(int eta);
size_t fused_smem_bytes(int eta, size_t elem);
template <class T> cudaError_t configure_fused(size_t smem);
template <class T>
void launch_smooth_step(const FusedArgs<T>& a, const FusedMaps& maps, int ntiles, bool zero_in,
                        bool prolong, bool restrict_, size_t smem, cudaStream_t st);
