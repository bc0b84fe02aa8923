// Shared definitions of the ghost-FEM multigrid library (CUDA, sm_103a).
//
// Node layout of every level (n cells per side, nodes 0..n in each direction):
// a padded row-major array, node (i, j) at (j + MG_G) * pitch + (i + MG_G).
// The node index of Sec. 5.1, k = i + j (n+1), is the unpadded version of the
// same row-major order.  Everything outside [0, n]^2 holds zero (code 0), so
// stencil kernels read halos without bounds checks.
//
// Per node a uint16 "code": 0 = not a DOF, 1 = interior DOF (all four adjacent
// cells internal: constant Q1 stencil 8/3, -1/3), >= 2 = boundary DOF (vertex
// of a cut cell), whose 9-point row is row[tile_base[tile] + code - 2] in a
// table compacted per 64 x 32 node tile.
#pragma once

#include <cstdint>
#include <cstddef>
#include <cuda_runtime.h>

#define MG_TX 64          // tile width in nodes
#define MG_TY 32          // tile height in nodes
#define MG_G 8            // zero margin around the node array
#define MG_ROW 10         // boundary row: 9 stencil coefficients + 1/diagonal

// 3 x 3 stencil offset order used by boundary rows: s = (di + 1) + 3 (dj + 1)

enum CellClass : uint8_t { CELL_EXT = 0, CELL_INT = 1, CELL_CUT = 2 };

// device error bits (ORed into a device word, turned into status codes)
enum : unsigned {
  DEV_ERR_NAN = 1u,          // NaN / Inf in an input array
  DEV_ERR_EDGE = 2u,         // Omega_h touches the outer ring of the box
  DEV_ERR_NOT_SPD = 4u,      // coarsest Cholesky pivot <= 0
  DEV_ERR_TILE = 8u,         // more boundary nodes in a tile than codes allow
  DEV_ERR_GEOM = 16u,        // unexpected cut configuration
  DEV_ERR_TIMEOUT = 32u,     // a bounded device wait ran out
  DEV_ERR_ALIGN = 64u,       // a TMA / bulk copy operand failed its alignment check
};

// Bounds-checked build (compiled with -DMG_CHECK_BOUNDS, a debug variant of
// the library): node indices (Layout::idx), boundary-row indices and the
// region positions of the boundary-node lists are checked where they are
// formed.  A failed check sets a device word (one per device, bound to every
// translation unit by the MG_BOUNDS_BINDER function it defines) and redirects
// the access to element 0 of its array, so the kernel reads and writes only
// inside its allocations and finishes; the host reports the word as
// MG_ERR_INTERNAL (mg_bounds_check).  In the normal build the checks compile
// to nothing.
#ifdef MG_CHECK_BOUNDS
static __constant__ unsigned* c_bounds_word;
__device__ __forceinline__ bool mg_checked(bool ok) {
  if (!ok && c_bounds_word) atomicOr(c_bounds_word, 1u);
  return ok;
}
#define MG_CHECKED(cond) mg_checked(cond)
#define MG_BOUNDS_BINDER(name)                                                        \
  cudaError_t name(unsigned* word) {                                                  \
    return cudaMemcpyToSymbol(c_bounds_word, &word, sizeof(word));                    \
  }
#else
#define MG_CHECKED(cond) true
#define MG_BOUNDS_BINDER(name)                                                        \
  cudaError_t name(unsigned*) { return cudaSuccess; }
#endif
// a boundary-row index r of a table of n rows (0 when out of range, checked
// builds only)
__device__ __forceinline__ int checked_row(int r, int n) {
  (void)n;
  return MG_CHECKED(r >= 0 && r < n) ? r : 0;
}
// region position {x, y} of a boundary-node list entry {x | y << 16, row}
// of an RX x RY region; `inner`: a colour-group entry, which the phases
// update and whose stencil must stay inside (checked builds only: (1, 1)
// when out of range)
__device__ __forceinline__ int2 region_pos(int2 en, bool inner, int RX, int RY) {
  int x = en.x & 0xffff, y = en.x >> 16;
  (void)inner; (void)RX; (void)RY;
  if (!MG_CHECKED(x < RX && y < RY &&
                  (!inner || (x >= 1 && y >= 1 && x < RX - 1 && y < RY - 1))))
    x = y = 1;
  return make_int2(x, y);
}

struct Layout {
  int n;       // cells per side
  int ntx;     // tiles along x covering nodes 0..n
  int nty;
  int pitch;   // elements per padded row
  int rows;    // padded rows
  __host__ __device__ __forceinline__ size_t idx(int i, int j) const {
#if defined(MG_CHECK_BOUNDS) && defined(__CUDA_ARCH__)
    if (!MG_CHECKED(i >= -MG_G && j >= -MG_G && i + MG_G < pitch && j + MG_G < rows)) return 0;
#endif
    return (size_t)(j + MG_G) * (size_t)pitch + (size_t)(i + MG_G);
  }
  __host__ __device__ __forceinline__ size_t size() const {
    return (size_t)pitch * (size_t)rows;
  }
  __host__ __device__ __forceinline__ int tile_of(int i, int j) const {
    return (j / MG_TY) * ntx + (i / MG_TX);
  }
};

inline Layout make_layout(int n) {
  Layout L;
  L.n = n;
  L.ntx = (n + 1 + MG_TX - 1) / MG_TX;
  L.nty = (n + 1 + MG_TY - 1) / MG_TY;
  // one spare tile column/row so that regions of the next finer level's
  // restriction blocks stay inside the allocation
  int w = (L.ntx + 1) * MG_TX + 2 * MG_G;
  L.pitch = (w + 31) / 32 * 32;
  L.rows = (L.nty + 1) * MG_TY + 2 * MG_G;
  return L;
}

// Operator data of one level, precision independent part.
struct LevelOp {
  Layout L;
  const uint16_t* code;     // padded layout
  const int* tile_base;     // per tile: first boundary row
};

template <class T> struct Vec2;
template <> struct Vec2<double> { typedef double2 type; };
template <> struct Vec2<float> { typedef float2 type; };

// Block-wide reductions ------------------------------------------------------

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// non-negative doubles order like their bit patterns
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr),
            (unsigned long long)__double_as_longlong(v));
}

// Max |x| kept as the bit pattern of |x|: non-negative doubles order like
// their bit patterns, so integer max replaces fmax (integer instructions
// instead of the scarce fp64 pipe), and a NaN (above +Inf in this order) is
// kept rather than dropped as fmax would.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ void max_abs(unsigned long long& m, double x) {
  const unsigned long long b = abs_bits(x);
  m = b > m ? b : m;
}
// finite (neither Inf nor NaN), by the exponent bits
__device__ __forceinline__ bool finite_bits(double x) {
  return (abs_bits(x) >> 52) != 0x7ffull;
}
__device__ __forceinline__ unsigned long long warp_max_bits(unsigned long long m) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, m, o);
    m = b > m ? b : m;
  }
  return m;
}

// Reduce (max |x| as bits, sum) over the block and take them into out[0]
// (max, by atomic max on the bit pattern) / out[1] (sum).  Requires
// blockDim.x a multiple of 32, <= 1024.
__device__ __forceinline__ void block_norms_to_global(unsigned long long vmax, double vsum,
                                                      double* out) {
  __shared__ unsigned long long s_max[32];
  __shared__ double s_sum[32];
  vmax = warp_max_bits(vmax);
  vsum = warp_sum(vsum);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { s_max[w] = vmax; s_sum[w] = vsum; }
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    vmax = l < nw ? s_max[l] : 0ull;
    vsum = l < nw ? s_sum[l] : 0.0;
    vmax = warp_max_bits(vmax);
    vsum = warp_sum(vsum);
    if (l == 0) {
      atomicMax(reinterpret_cast<unsigned long long*>(out), vmax);
      atomicAdd(out + 1, vsum);
    }
  }
}

// As block_norms_to_global, but the block's sum goes to *part (a slot of
// its own) for a later fixed-order total (sum_partials): the same bits on
// every run.
__device__ __forceinline__ void block_norms_partial(unsigned long long vmax, double vsum,
                                                    double* out, double* part) {
  __shared__ unsigned long long p_max[32];
  __shared__ double p_sum[32];
  vmax = warp_max_bits(vmax);
  vsum = warp_sum(vsum);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { p_max[w] = vmax; p_sum[w] = vsum; }
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    vmax = l < nw ? p_max[l] : 0ull;
    vsum = l < nw ? p_sum[l] : 0.0;
    vmax = warp_max_bits(vmax);
    vsum = warp_sum(vsum);
    if (l == 0) {
      atomicMax(reinterpret_cast<unsigned long long*>(out), vmax);
      *part = vsum;
    }
  }
}

// Programmatic dependent launch ---------------------------------------------
//
// The V-cycle kernels are launched with programmatic stream serialization:
// a kernel's blocks may start while the previous kernel's last blocks are
// still running.  Each kernel reads only static data (codes, lists, rows,
// tensor maps) before griddep_wait(); every read of data another kernel
// writes (u, F, bval, e, norms) and every global write comes after it.  The
// wait returns once the previous kernel has completed and its writes are
// visible (immediately when launched without the attribute).
//
// One exception: the band kernel (eta sweeps over the cut-cell vertices)
// lets its dependents launch only after its own wait, so when it starts the
// kernel after it, every kernel before the band kernel has completed.  A
// block of that next kernel whose input region holds none of the nodes the
// band kernel writes may then skip the wait (band_independent below); it
// reads through L2 (ld.global.cg), never from a possibly stale L1 line.  At
// least one block of such a launch always waits, so the launch completes
// only after the band kernel.
__device__ __forceinline__ void griddep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
// Lets the next kernel in the stream launch once every block of this one has
// started (it still waits in griddep_wait for this kernel to complete).
__device__ __forceinline__ void griddep_launch_next() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
// touch: per block, nonzero when the block's input region holds a node the
// directly preceding band kernel writes; nullptr when the launch does not
// directly follow a band kernel (every block waits).  Block 0 always waits.
__device__ __forceinline__ bool band_independent(const uint8_t* touch) {
  return touch != nullptr && blockIdx.x != 0 && touch[blockIdx.x] == 0;
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Host helpers ----------------------------------------------------------------

// Raises a kernel's dynamic shared-memory limit to at least `bytes`; never
// lowers it, since handles with different needs launch the same kernel.
template <class K>
cudaError_t raise_smem_limit(K* kernel, size_t bytes) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define MG_CUDA_TRY(expr)                                  \
  do {                                                     \
    cudaError_t e__ = (expr);                              \
    if (e__ != cudaSuccess) return mg_cuda_fail(e__);      \
  } while (0)

int mg_cuda_fail(cudaError_t e);   // records the message, returns MG_ERR_CUDA

// scan.cu: exclusive scan / compaction on the device
// out[i] = sum_{k<i} in[i]; *total (device) = sum of all.  tmp must hold
// scan_tmp_ints(n) ints.
size_t scan_tmp_ints(size_t n);
void exclusive_scan_int(const int* in, int* out, int* total, size_t n, int* tmp,
                        cudaStream_t st);
// list of indices i with flag[i] != 0, in increasing order; *count on device
void compact_flags_u8(const uint8_t* flag, int* list, int* count, size_t n, int* tmp,
                      int* tmp_offsets, cudaStream_t st);
