// Single-block V-cycle on the smallest levels (see tail.cu).
#pragma once

#include "tma.cuh"

#define MG_TAIL_MAX_LEVELS 6
#define MG_TAIL_MAX_N 64      // largest top level the tail block handles

// Shared-memory layout of the tail block, byte offsets.  The first
// image_bytes are a static image built once at setup (node tags, colour-sorted
// boundary lists and their offsets, boundary rows, coarsest inverse) and
// copied in with one bulk copy per launch; u, F and the residual follow.
struct TailLayout {
  int nlev = 0;
  int n[MG_TAIL_MAX_LEVELS] = {};
  int n_bnd[MG_TAIL_MAX_LEVELS] = {};
  size_t G[MG_TAIL_MAX_LEVELS] = {};     // int16 tags, bordered (n+3)^2
  size_t BL[MG_TAIL_MAX_LEVELS] = {};    // uint16 bordered positions, by colour
  size_t off = 0;                        // int [level][5] colour offsets into BL
  size_t rows[MG_TAIL_MAX_LEVELS] = {};  // boundary rows (if rows_in_smem)
  size_t Ainv = 0;                       // coarsest inverse (if ainv_in_smem)
  size_t image_bytes = 0;
  size_t U[MG_TAIL_MAX_LEVELS] = {};
  size_t F[MG_TAIL_MAX_LEVELS] = {};
  size_t R = 0;
  size_t total = 0;
  bool rows_in_smem = false;
  bool ainv_in_smem = false;
};

// Layout for levels of n[k] cells (halving) with n_bnd[k] boundary rows and
// an m x m coarsest inverse, element size elem; rows and then the inverse
// are staged only if the total stays within max_bytes.  Returns false when
// even the minimum does not fit.
bool tail_layout(const int* n, const int* n_bnd, int nlev, int m, size_t elem, size_t max_bytes,
                 TailLayout* out);

template <class T> struct TailArgs {
  TailLayout lay;
  Layout L0;                                  // padded layout of the top level
  const unsigned char* image;                 // static image (global, 16-byte aligned)
  const T* rows[MG_TAIL_MAX_LEVELS];          // boundary rows in global memory
  const double* Ainv;                         // coarsest inverse, m x m, by columns
  const T* F0;                                // right-hand side of the top level
  T* u0;                                      // top level u: initial guess (load_u0) / result
  int load_u0;
  int eta, nu1, nu2;
  unsigned* err;                              // DEV_ERR_TIMEOUT if the image copy stalls
  unsigned wait_polls = kMbarSpinLimit;       // poll budget of the image copy's wait
  int transposed = 0;                         // run the transposed V-cycle
};

// Device arrays a level contributes to the image.
struct TailLevelSrc {
  Layout L;
  const uint16_t* code;
  const int* tile_base;
};

// Builds the tags, boundary lists and offsets of the image (one block);
// the caller copies rows and the inverse to their offsets.
void launch_tail_image(const TailLayout& lay, const TailLevelSrc* lv, unsigned char* image,
                       cudaStream_t st);
template <class T> cudaError_t configure_tail(size_t smem);
template <class T> void launch_tail(const TailArgs<T>& a, cudaStream_t st);
