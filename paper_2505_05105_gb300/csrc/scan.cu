// Device-wide exclusive scan and stream compaction (three passes: per-chunk
// sums, one-block scan of the chunk sums, per-chunk local scan).  Used only
// by setup; results are deterministic (increasing index order).
#include "common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kPer = 16;
constexpr int kChunk = kThreads * kPer;   // 4096 elements per block

struct IntIn {
  const int* p;
  __device__ int operator()(size_t i) const { return p[i]; }
};
struct FlagIn {
  const uint8_t* p;
  __device__ int operator()(size_t i) const { return p[i] != 0; }
};

__device__ __forceinline__ int block_exclusive_scan(int v, int* total) {
  __shared__ int s_warp[kThreads / 32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = lane < kThreads / 32 ? s_warp[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kThreads / 32) s_warp[lane] = s;
  }
  __syncthreads();
  int warp_off = w > 0 ? s_warp[w - 1] : 0;
  *total = s_warp[kThreads / 32 - 1];
  __syncthreads();
  return warp_off + x - v;
}

template <class In>
__global__ void chunk_sums(In in, size_t n, int* sums) {
  size_t base = (size_t)blockIdx.x * kChunk + (size_t)threadIdx.x * kPer;
  int s = 0;
  for (int k = 0; k < kPer; ++k) {
    size_t i = base + k;
    if (i < n) s += in(i);
  }
  int tot;
  block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void scan_sums(int* sums, int nb, int* total) {
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += kThreads) {
    int i = base + threadIdx.x;
    int v = i < nb ? sums[i] : 0;
    int tot;
    int ex = block_exclusive_scan(v, &tot);
    if (i < nb) sums[i] = ex + carry;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

template <class In>
__global__ void chunk_scan_write(In in, size_t n, const int* offs, int* out) {
  size_t base = (size_t)blockIdx.x * kChunk + (size_t)threadIdx.x * kPer;
  int v[kPer];
  int s = 0;
  for (int k = 0; k < kPer; ++k) {
    size_t i = base + k;
    v[k] = i < n ? in(i) : 0;
    s += v[k];
  }
  int tot;
  int ex = block_exclusive_scan(s, &tot) + offs[blockIdx.x];
  for (int k = 0; k < kPer; ++k) {
    size_t i = base + k;
    if (i < n) out[i] = ex;
    ex += v[k];
  }
}

__global__ void chunk_compact_write(FlagIn in, size_t n, const int* offs, int* list) {
  size_t base = (size_t)blockIdx.x * kChunk + (size_t)threadIdx.x * kPer;
  int v[kPer];
  int s = 0;
  for (int k = 0; k < kPer; ++k) {
    size_t i = base + k;
    v[k] = i < n ? in(i) : 0;
    s += v[k];
  }
  int tot;
  int ex = block_exclusive_scan(s, &tot) + offs[blockIdx.x];
  for (int k = 0; k < kPer; ++k) {
    if (v[k]) list[ex++] = (int)(base + k);
  }
}

}  // namespace

size_t scan_tmp_ints(size_t n) { return (n + kChunk - 1) / kChunk + 1; }

void exclusive_scan_int(const int* in, int* out, int* total, size_t n, int* tmp,
                        cudaStream_t st) {
  int nb = (int)((n + kChunk - 1) / kChunk);
  if (nb == 0) {
    cudaMemsetAsync(total, 0, sizeof(int), st);
    return;
  }
  IntIn a{in};
  chunk_sums<<<nb, kThreads, 0, st>>>(a, n, tmp);
  scan_sums<<<1, kThreads, 0, st>>>(tmp, nb, total);
  chunk_scan_write<<<nb, kThreads, 0, st>>>(a, n, tmp, out);
}

void compact_flags_u8(const uint8_t* flag, int* list, int* count, size_t n, int* tmp,
                      int* /*tmp_offsets*/, cudaStream_t st) {
  int nb = (int)((n + kChunk - 1) / kChunk);
  if (nb == 0) {
    cudaMemsetAsync(count, 0, sizeof(int), st);
    return;
  }
  FlagIn a{flag};
  chunk_sums<<<nb, kThreads, 0, st>>>(a, n, tmp);
  scan_sums<<<1, kThreads, 0, st>>>(tmp, nb, count);
  chunk_compact_write<<<nb, kThreads, 0, st>>>(a, n, tmp, list);
}

// binds the bounds-checked build's device error word (see common.cuh)
MG_BOUNDS_BINDER(bind_bounds_scan)
