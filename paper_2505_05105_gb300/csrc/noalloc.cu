// mg_residual_static: the fine-level residual r = F - A u and its norms
// without allocating anything.
//
// Some callers cannot call cudaMalloc while they use the solver: real-time
// loops that cannot take the device-wide synchronisation an allocation (or
// the release of one) may cause, and frameworks whose own caching allocator
// must own every byte of device memory (a memory cap, no fragmentation from
// a library's private allocations).  This entry point reads and writes only
// the caller's arrays and the handle's read-only operator; its reduction
// scratch is the file-scope device array below, which every GPU that loads
// the library holds until the process exits.
#include <mutex>

#include "ghostmg.h"
#include "internal.h"

namespace {

// Per active tile: (max |r|, sum r^2); then the final (||r||_inf, ||r||_2).
// Every slot a call reads is written earlier in the same call, so nothing
// has to be cleared between calls.
static __device__ __align__(256) double g_residual_scratch[2 * MG_NOALLOC_MAX_TILES + 2];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of g_residual_scratch on device `dev`, looked up once per
// device with that device current (host code may not use the symbol itself
// as a device address); the caller's current device is restored.
int scratch_address(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return MG_ERR_INTERNAL;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    int prev = 0;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return mg_cuda_fail(e);
    if (prev != dev && (e = cudaSetDevice(dev)) != cudaSuccess) return mg_cuda_fail(e);
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_residual_scratch);
    cudaError_t e2 = prev != dev ? cudaSetDevice(prev) : cudaSuccess;
    if (e != cudaSuccess) return mg_cuda_fail(e);
    if (e2 != cudaSuccess) return mg_cuda_fail(e2);
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return MG_OK;
}

// true for device (or managed) memory of device `dev`
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

constexpr int kRX = MG_TX + 2, kRY = MG_TY + 2;   // owned tile + 1-node halo

// Residual of the owned nodes of one active tile, reading u and F in the
// caller's unpadded (N+1)^2 layout; u is taken as 0 off the DOFs.  Writes r
// (if given) and the tile's partial norms to part[2 * blockIdx.x].
__global__ void __launch_bounds__(256)
k_residual_static(Layout L, const uint16_t* __restrict__ code, const int* __restrict__ tile_base,
                  const double* __restrict__ rows, int n_rows, const int* __restrict__ tiles,
                  int N,
                  const double* __restrict__ F, const double* __restrict__ u,
                  double* __restrict__ r, double* __restrict__ part) {
  __shared__ double sU[kRY * kRX];
  __shared__ uint16_t sC[kRY * kRX];
  __shared__ double s_max[8], s_sum[8];
  const int t = tiles[blockIdx.x];
  const int i0 = (t % L.ntx) * MG_TX, j0 = (t / L.ntx) * MG_TY;
  for (int p = threadIdx.x; p < kRY * kRX; p += blockDim.x) {
    int y = p / kRX, x = p - y * kRX;
    int gi = i0 - 1 + x, gj = j0 - 1 + y;
    uint16_t cd = code[L.idx(gi, gj)];      // margins keep this in bounds
    double v = 0.0;
    if (cd && gi >= 0 && gj >= 0 && gi <= N && gj <= N) v = u[(size_t)gj * (N + 1) + gi];
    sU[p] = v;
    sC[p] = cd;
  }
  __syncthreads();
  double vmax = 0.0, vsum = 0.0;
  for (int it = threadIdx.x; it < MG_TX * MG_TY; it += blockDim.x) {
    int rr = it / MG_TX, ii = it - rr * MG_TX;
    int gi = i0 + ii, gj = j0 + rr;
    if (gi > N || gj > N) continue;
    int p = (rr + 1) * kRX + ii + 1;
    uint16_t cd = sC[p];
    double res = 0.0;
    if (cd) {
      const double* Up = sU + p;
      double f = F[(size_t)gj * (N + 1) + gi];
      if (cd == 1) {
        double s8 = ((Up[-1] + Up[1]) + (Up[-kRX] + Up[kRX])) +
                    ((Up[-kRX - 1] + Up[-kRX + 1]) + (Up[kRX - 1] + Up[kRX + 1]));
        res = f - (8.0 * Up[0] - s8) * (1.0 / 3.0);
      } else {
        const double* R = rows + (size_t)checked_row(tile_base[t] + cd - 2, n_rows) * MG_ROW;
        double acc = R[0] * Up[-kRX - 1] + R[1] * Up[-kRX] + R[2] * Up[-kRX + 1] +
                     R[3] * Up[-1] + R[4] * Up[0] + R[5] * Up[1] + R[6] * Up[kRX - 1] +
                     R[7] * Up[kRX] + R[8] * Up[kRX + 1];
        res = f - acc;
      }
    }
    if (r) r[(size_t)gj * (N + 1) + gi] = res;
    vmax = fmax(vmax, fabs(res));
    vsum += res * res;
  }
  for (int o = 16; o > 0; o >>= 1) {
    vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    vsum += __shfl_xor_sync(0xffffffffu, vsum, o);
  }
  if ((threadIdx.x & 31) == 0) { s_max[threadIdx.x >> 5] = vmax; s_sum[threadIdx.x >> 5] = vsum; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0, s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { m = fmax(m, s_max[w]); s += s_sum[w]; }
    part[2 * blockIdx.x] = m;
    part[2 * blockIdx.x + 1] = s;
  }
}

// Fixed-order reduction of the n tile partials into out[0..1] (deterministic).
__global__ void __launch_bounds__(1024)
k_reduce_partials(const double* __restrict__ part, int n, double* __restrict__ out) {
  __shared__ double s_max[32], s_sum[32];
  double m = 0.0, s = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    m = fmax(m, part[2 * k]);
    s += part[2 * k + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  if ((threadIdx.x & 31) == 0) { s_max[threadIdx.x >> 5] = m; s_sum[threadIdx.x >> 5] = s; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0, ss = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { mm = fmax(mm, s_max[w]); ss += s_sum[w]; }
    out[0] = mm;
    out[1] = sqrt(ss);
  }
}

int run_residual(const FineOpView& v, const double* F, const double* u, double* r, double* norms,
                 double* scratch);

}  // namespace

extern "C" int mg_residual_static(mg_handle h, const double* F, const double* u, double* r,
                                  double* norms) {
  if (!h || !F || !u) return MG_ERR_INVALID_ARG;
  FineOpView v;
  int rc = mg_internal_fine_view(h, &v);
  if (rc != MG_OK) return rc;
  if (v.n_active > MG_NOALLOC_MAX_TILES) return MG_ERR_INVALID_ARG;   // scratch too small
  if (!on_device(F, v.device) || !on_device(u, v.device) || (r && !on_device(r, v.device)))
    return MG_ERR_INVALID_ARG;
  double* scratch = nullptr;
  rc = scratch_address(v.device, &scratch);
  if (rc != MG_OK) return rc;
  // the launches below go to the handle's device
  int prev = 0;
  cudaError_t e = cudaGetDevice(&prev);
  if (e != cudaSuccess) return mg_cuda_fail(e);
  if (prev != v.device && (e = cudaSetDevice(v.device)) != cudaSuccess) return mg_cuda_fail(e);
  rc = run_residual(v, F, u, r, norms, scratch);
  if (prev != v.device && (e = cudaSetDevice(prev)) != cudaSuccess && rc == MG_OK)
    rc = mg_cuda_fail(e);
  return rc;
}

namespace {

int run_residual(const FineOpView& v, const double* F, const double* u, double* r, double* norms,
                 double* scratch) {
  double* result = scratch + 2 * MG_NOALLOC_MAX_TILES;
  const size_t m = (size_t)(v.N + 1) * (v.N + 1);
  cudaError_t e;
  if (r) {
    // nodes outside the active tiles are not DOFs: their residual is 0
    e = cudaMemsetAsync(r, 0, m * sizeof(double), v.st);
    if (e != cudaSuccess) return mg_cuda_fail(e);
  }
  if (v.n_active > 0)
    k_residual_static<<<v.n_active, 256, 0, v.st>>>(v.L, v.code, v.tile_base, v.rows64, v.n_rows,
                                                     v.active, v.N, F, u, r, scratch);
  k_reduce_partials<<<1, 1024, 0, v.st>>>(scratch, v.n_active, result);
  e = cudaGetLastError();
  if (e != cudaSuccess) return mg_cuda_fail(e);
  if (norms) {
    e = cudaMemcpyAsync(norms, result, 2 * sizeof(double), cudaMemcpyDefault, v.st);
    if (e != cudaSuccess) return mg_cuda_fail(e);
  }
  e = cudaStreamSynchronize(v.st);
  if (e != cudaSuccess) return mg_cuda_fail(e);
  return MG_OK;
}

}  // namespace

// binds the bounds-checked build's device error word (see common.cuh)
MG_BOUNDS_BINDER(bind_bounds_noalloc)
