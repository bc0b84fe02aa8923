// Batched mixed-precision solves of many independent geometries in one
// persistent kernel (see batch.cu).
#pragma once

#include "cycle.cuh"
#include "tail.cuh"

#define MG_BATCH_MAX_TOP 10      // levels above the tail block (N <= 32768)

// One level solved block-wide in global memory (the levels above the tail).
struct BatchLevel {
  Layout L;
  const uint16_t* code;
  const int* tile_base;
  const float* rows;           // fp32 boundary rows
  const float* srows;          // the listed nodes' rows by coefficient: [k n_bnd + e]
  const unsigned* xy;          // active tiles' first nodes, i0 | j0 << 16
  int n_active;
  const int2* blist;           // boundary nodes {padded offset, row}, grouped by colour
  int boff[5];                 // colour group offsets into blist
  // shared-memory window of the eta phases (win_n = 0: none, the phases run
  // in global memory): win[k] the padded offset of window node k (the
  // boundary nodes and their neighbours); wslot[10 e + s] the window index
  // of stencil position s (0..8, row order) of blist entry e
  const int* win;
  const uint16_t* wslot;
  int win_n;
  // static images of the resident eta phases (eta_resident_layout from
  // `rows` to `f`, or null): [0] the lead block alone, [1], [2] blocks 0 and 1
  // of a team of two
  const unsigned char* rimg[3];
  float* u;                    // iterate (in place)
  float* F;                    // right-hand side
  float* scr;                  // residual scratch (zero outside the active tiles)
};

// Shared memory of the resident eta phases of one level (batch.cu,
// eta_resident) for le entries per block: the window (win_n floats), then per
// entry its row (10 floats, by coefficient), position and the window indices
// of its three stencil rows (by row) -- the static image, one bulk copy --
// and its right-hand side.
struct EtaResidentLayout {
  size_t rows, pos, slot, f, total;
};
__host__ __device__ inline size_t eta_a16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline EtaResidentLayout eta_resident_layout(int win_n, int le) {
  EtaResidentLayout l;
  l.rows = eta_a16((size_t)win_n * sizeof(float));
  l.pos = l.rows + eta_a16((size_t)le * 10 * sizeof(float));
  l.slot = l.pos + eta_a16((size_t)le * sizeof(int));
  l.f = l.slot + eta_a16((size_t)le * 3 * sizeof(uint16_t));
  l.total = l.f + eta_a16((size_t)le * sizeof(float));
  return l;
}
// bytes for a level with colour group offsets boff (5) shared by nr blocks
// (entry j of a group to block j mod nr; the layout is that of the block
// with the most entries)
__host__ __device__ inline size_t eta_resident_bytes(int win_n, const int* boff, int nr) {
  int le = 0;
  for (int c = 0; c < 4; ++c) le += (boff[c + 1] - boff[c] + nr - 1) / nr;
  return eta_resident_layout(win_n, le).total;
}

struct BatchProblem {
  int n_top;                   // levels 0 .. n_top-1 block-wide, the tail from level n_top
  int res_cap;                 // shared memory the resident eta phases may use (bytes)
  BatchLevel lev[MG_BATCH_MAX_TOP];
  TailArgs<float> tail;        // the tail block's V-cycle (its top F and u: level n_top)
  const unsigned* tail_xy;     // active tiles of the tail's top level (i0 | j0 << 16)
  int tail_n_active;
  float* tail_F;               // the tail's top F (restriction target)
  // fine level in fp64
  Layout L0;
  const uint16_t* code0;
  const int* tile_base0;
  const double* rows64;
  const int* active0;          // active tiles (ids)
  const unsigned* xy0;         // and their first nodes, i0 | j0 << 16
  int n_active0;
  double* F64;
  double* u64;
  float* F32;                  // fine fp32 right-hand side (lev[0].F, or the tail's top F)
  float* e32;                  // fine fp32 correction (lev[0].u, or the tail's top u)
  int eta, nu1, nu2;
  // the member's data in the packed user arrays (row-major (N+1)^2 nodes)
  RhsArgs rhs;
  const double* f;
  const double* g;
  double* u_out;
};

struct BatchResult {
  int cycles, checks, status, pad;
  double rel_res;
};

// tuning knobs of the persistent kernel (chosen by mg_batch_tune)
struct BatchTune {
  int threads;                 // threads per block (256 .. 1024)
  int first_group;             // V-cycles before the first fp64 residual check
  int cluster;                 // blocks per thread-block cluster (1, 2, 4, 8)
  int coop_min_dof;            // members with at least this many DOFs (and levels
                               // above the tail) are solved by a whole cluster
};

// Per-member input check and right-hand side over all members at once:
// node_off[p] (count + 1 entries) is member p's first node in the packed user
// arrays, tile_off[p] its first active fine tile in the flattened tile range.
// F of every member (k_rhs's tile code); bad[p] (the member's RhsArgs.err)
// gets DEV_ERR_NAN where a NaN or Inf in f, g or g_N enters its F.
void launch_batch_rhs(const BatchProblem* probs, const int* tile_off, int count, int total_tiles,
                      cudaStream_t st);
// u_out of every member from its fine fp64 iterate (zero off the DOFs)
void launch_batch_unpack(const BatchProblem* probs, const size_t* node_off, int count,
                         size_t total_nodes, cudaStream_t st);

// Launches the persistent kernel: grid blocks take problems order[0..count)
// from the counter *next (zero on entry), largest first.
// Members with bad[p] != 0 get u = 0 and status MG_ERR_INVALID_ARG.
// params = {tol, max_cycles, fixed group size or 0} (device memory, read at
// launch).  words[0] and words[2] are the work counters (zero on entry),
// words[1] the error word.  order[0 .. n_coop) are solved by whole clusters
// of tune.cluster blocks, the rest by single blocks; grid is a multiple of
// tune.cluster.
void launch_batch(const BatchProblem* probs, const int* order, int count, int n_coop,
                  unsigned* words, const unsigned* bad, const double* params, BatchTune tune,
                  int grid, size_t smem, BatchResult* res, cudaStream_t st);
cudaError_t configure_batch(size_t smem);
// clusters of tune.cluster blocks that can be resident at once (0 if none)
int batch_max_clusters(const BatchTune& tune, size_t smem);
// out[k n + e] = rows[blist[e].y * MG_ROW + k] (n list entries)
void launch_soa_rows(const int2* blist, int n, const float* rows, float* out, cudaStream_t st);
// xy[k] = i0 | j0 << 16 of tile active[k] of layout L
void launch_tile_xy(const Layout& L, const int* active, int n, unsigned* xy, cudaStream_t st);
// builds blist / boff of one level from its codes (one block)
void launch_batch_lists(const Layout& L, const uint16_t* code, const int* tile_base,
                        int2* blist, int* boff, cudaStream_t st);
