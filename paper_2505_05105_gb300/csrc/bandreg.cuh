// The eta extra colour sweeps over the cut-cell vertices (Sec. 5.3) of one
// shared-memory region, with each thread's nodes held in registers.
#pragma once

#include "common.cuh"

// Runs 4 eta colour phases on the listed boundary nodes of a region whose
// values are in sU (row stride RS).  Colour c's nodes are the list entries
// g[c] .. g[c+1]-1.  The calling threads (nt of them, threadIdx.x < nt) each
// own the entry g[c] + threadIdx.x of every colour: its matrix row, F and
// position are fetched once by stage(e, w, p) (w[0..8] the 9-point row,
// w[9] 1/diagonal, w[MG_ROW] F) and kept in registers for all phases, so a
// phase is 9 shared loads, the dot product and one store.  Entries past
// g[c] + nt (a colour with more nodes than threads) go through extra(e)
// every phase.  Phases are separated by __syncwarp (nt == 32) or by named
// barrier 1 over the nt threads.
// REV: the colours in the reverse order (the transposed sweep).
template <class T, class Stage, class Extra, bool REV = false>
__device__ __forceinline__ void band_phases_reg(T* sU, int RS, const int* g, int eta, int nt,
                                                Stage stage, Extra extra) {
  T w[4][MG_ROW + 1];
  int p[4];
  bool has[4];
  bool more = false;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int e = g[c] + threadIdx.x;
    has[c] = e < g[c + 1];
    p[c] = 0;
#pragma unroll
    for (int k = 0; k <= MG_ROW; ++k) w[c][k] = T(0);
    if (has[c]) stage(e, w[c], p[c]);
    more |= g[c + 1] - g[c] > nt;
  }
  for (int it = 0; it < eta; ++it) {
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int c = REV ? 3 - cc : cc;
      if (has[c]) {
        const T* Up = sU + p[c];
        const T* W = w[c];
        T acc = W[0] * Up[-RS - 1] + W[1] * Up[-RS] + W[2] * Up[-RS + 1] + W[3] * Up[-1] +
                W[4] * Up[0] + W[5] * Up[1] + W[6] * Up[RS - 1] + W[7] * Up[RS] +
                W[8] * Up[RS + 1];
        sU[p[c]] = Up[0] + (W[MG_ROW] - acc) * W[9];
      }
      if (more)
        for (int e = g[c] + nt + threadIdx.x; e < g[c + 1]; e += nt) extra(e);
      if (nt == 32) __syncwarp();
      else asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
    }
  }
}

// As band_phases_reg, but each thread keeps only the position, F and the
// row index of its nodes (rows read from `rows`, normally shared memory):
// for kernels whose register budget cannot hold four rows.  stage(e, r, f, p).
template <class T, class Stage, class Extra, bool REV = false>
__device__ __forceinline__ void band_phases_idx(T* sU, int RS, const T* rows, const int* g,
                                                int eta, int nt, Stage stage, Extra extra) {
  int r[4], p[4];
  T f[4];
  bool more = false;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int e = g[c] + threadIdx.x;
    p[c] = -1;
    r[c] = 0;
    f[c] = T(0);
    if (e < g[c + 1]) stage(e, r[c], f[c], p[c]);
    more |= g[c + 1] - g[c] > nt;
  }
  for (int it = 0; it < eta; ++it) {
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int c = REV ? 3 - cc : cc;
      if (p[c] >= 0) {
        const T* Up = sU + p[c];
        const T* W = rows + (size_t)r[c] * MG_ROW;
        T acc = W[0] * Up[-RS - 1] + W[1] * Up[-RS] + W[2] * Up[-RS + 1] + W[3] * Up[-1] +
                W[4] * Up[0] + W[5] * Up[1] + W[6] * Up[RS - 1] + W[7] * Up[RS] +
                W[8] * Up[RS + 1];
        sU[p[c]] = Up[0] + (f[c] - acc) * W[9];
      }
      if (more)
        for (int e = g[c] + nt + threadIdx.x; e < g[c + 1]; e += nt) extra(e);
      if (nt == 32) __syncwarp();
      else asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
    }
  }
}
