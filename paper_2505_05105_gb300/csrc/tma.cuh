// Tensor-memory-accelerator (TMA) loads of 2D node regions into shared memory.
//
// A level's padded node array (see common.cuh) is described to the TMA unit
// by a 2D tensor map: extent (pitch, rows) elements, row stride pitch *
// element size bytes.  One cp.async.bulk.tensor.2d copies a box of BX x BY
// elements starting at padded coordinates (x, y) into shared memory and
// signals an mbarrier with the byte count; boxes reaching outside the array
// are zero-filled.  The TMA unit requires the box's first column x to start
// on a 16-byte boundary: every caller rounds x down to a multiple of
// kTmaAlign elements (8, i.e. 16 bytes for 16-bit data, 32 bytes for fp32)
// and indexes shared memory from the remainder.
//
// Waits are bounded: after a poll budget (kMbarSpinLimit unless the handle
// sets another, mg_set_wait_limit) the waiting thread sets DEV_ERR_TIMEOUT,
// waits once more with the default budget for its copies still in flight,
// and the kernel returns without using the data.
#pragma once

#include <cuda.h>
#include "common.cuh"

constexpr int kTmaAlign = 8;                  // elements; 16 bytes at 2 bytes each
constexpr unsigned kMbarSpinLimit = 1u << 22;

// first box column for a region starting at padded column xs, and the
// region's offset inside the box
__host__ __device__ inline int tma_floor(int xs) { return xs & ~(kTmaAlign - 1); }
// box width covering a region of w columns at any offset 0..kTmaAlign-1
__host__ __device__ constexpr int tma_box_w(int w) {
  return (w + kTmaAlign - 1 + kTmaAlign - 1) / kTmaAlign * kTmaAlign;
}

// Tensor copies need a 128-byte aligned shared destination; the dynamic
// shared memory base follows the kernel's static shared variables and is not
// guaranteed to be, so kernels round it up and reserve kSmemSlack extra bytes.
constexpr size_t kSmemSlack = 128;
__device__ __forceinline__ unsigned char* smem_align128(unsigned char* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  return p + ((128u - (a & 127u)) & 127u);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  // make the initialised barrier visible to the async (TMA) proxy
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ends the barrier object's life (before its word is initialised again)
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// true once the barrier completed phase `parity`; false after `limit` polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          unsigned limit = kMbarSpinLimit) {
  const uint32_t a = smem_u32(bar);
  for (unsigned it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// operand checks made before a copy is issued (a failing copy is skipped and
// DEV_ERR_ALIGN recorded instead)
__device__ __forceinline__ bool tma_box_ok(const void* dst, int x) {
  return (smem_u32(dst) & 127u) == 0 && (x & (kTmaAlign - 1)) == 0;
}
__device__ __forceinline__ bool bulk_ok(const void* dst, const void* src, size_t bytes) {
  return (smem_u32(dst) & 15u) == 0 && (reinterpret_cast<uintptr_t>(src) & 15u) == 0 &&
         (bytes & 15u) == 0;
}

// box of the tensor map at padded coordinates (x, y) -> shared memory dst
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// contiguous bytes global -> shared (both 16-byte aligned, a multiple of 16
// bytes), completing on the mbarrier
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Host: tensor map of a padded level array (elem = 2, 4 or 8 bytes) with a
// box of bx x by elements; bx * elem must be a multiple of 16 bytes.
int make_level_map(CUtensorMap* out, const void* base, size_t elem, const Layout& L, int bx,
                   int by);
