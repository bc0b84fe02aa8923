// Host side of the TMA loads: tensor maps through the driver entry point
// (no link-time dependency on libcuda).
#include <mutex>
#include <cudaTypedefs.h>
#include "tma.cuh"

namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_once;

void resolve() {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  else
    cudaGetLastError();
}

}  // namespace

int make_level_map(CUtensorMap* out, const void* base, size_t elem, const Layout& L, int bx,
                   int by) {
  std::call_once(g_once, resolve);
  if (!g_encode) return mg_cuda_fail(cudaErrorNotSupported);
  if ((bx * elem) % 16 != 0 || bx > 256 || by > 256 || bx <= 0 || by <= 0)
    return mg_cuda_fail(cudaErrorInvalidValue);
  CUtensorMapDataType dt = elem == 2   ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                           : elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                       : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  cuuint64_t dims[2] = {(cuuint64_t)L.pitch, (cuuint64_t)L.rows};
  cuuint64_t strides[1] = {(cuuint64_t)L.pitch * elem};
  cuuint32_t box[2] = {(cuuint32_t)bx, (cuuint32_t)by};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(out, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return mg_cuda_fail(cudaErrorInvalidValue);
  return 0;
}

// binds the bounds-checked build's device error word (see common.cuh)
MG_BOUNDS_BINDER(bind_bounds_tma)
