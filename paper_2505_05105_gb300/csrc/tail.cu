// The bottom of the V-cycle in one thread block.
//
// On the small levels (n <= 64 cells per side) every kernel of the V-cycle is
// latency bound: a launch costs more than its work.  k_tail runs the whole
// V-cycle below a given level (Alg. 1 applied recursively, Sec. 3.2) inside
// one thread block (512 threads in fp32, 1024 in fp64), with every level's
// u, F and node tags in shared
// memory and __syncthreads() between the colour phases: for each level
// nu1 smoothing steps (one 4-colour Gauss-Seidel sweep, Sec. 4.1, then eta
// sweeps over the cut-cell vertices, Sec. 5.3), residual and restriction
// R = P^T (Sec. 5.1), recursion, the exact coarsest solve (dense inverse),
// prolongation P, nu2 smoothing steps.  It reads F and writes u of its top
// level in that level's padded global layout, so it slots in where the
// multi-block kernels leave off.  The arithmetic and the colour order are
// those of the multi-block kernels.
//
// Everything that does not change between launches -- node tags, the
// colour-sorted boundary lists, the boundary rows and the coarsest inverse
// -- is a static image built at setup and copied into shared memory with
// one bulk copy, while the threads load F and u of the top level.
#include "tail_impl.cuh"

namespace {

constexpr int kThreads = kTailThreads;
// threads of k_tail: fp32 on 512 threads, which leaves the registers for the
// band phases' rows (the fp64 rows would not fit: 1024 threads, rows read
// from shared memory)
template <class T> struct TailBlock { static constexpr int threads = 1024; };
template <> struct TailBlock<float> { static constexpr int threads = 512; };

template <class T>
__global__ void __launch_bounds__(TailBlock<T>::threads, 1) k_tail(TailArgs<T> a) {
  griddep_launch_next();
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  tail_vcycle<T, sizeof(T) == sizeof(float)>(a, smem_align128(smem_dyn), a.load_u0 != 0, true);
}

// Setup: tags, colour-sorted boundary lists and their offsets of the image.
__global__ void k_tail_image(TailLayout lay, TailLevelSrc l0, TailLevelSrc l1, TailLevelSrc l2,
                             TailLevelSrc l3, TailLevelSrc l4, TailLevelSrc l5,
                             unsigned char* image) {
  __shared__ int cnt[MG_TAIL_MAX_LEVELS * 4];
  __shared__ int cur[MG_TAIL_MAX_LEVELS * 4];
  const TailLevelSrc lv[MG_TAIL_MAX_LEVELS] = {l0, l1, l2, l3, l4, l5};
  int* off = reinterpret_cast<int*>(image + lay.off);
  if (threadIdx.x < MG_TAIL_MAX_LEVELS * 4) cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int k = 0; k < lay.nlev; ++k) {
    const int n = lay.n[k], S = n + 3;
    int16_t* G = reinterpret_cast<int16_t*>(image + lay.G[k]);
    for (int q = threadIdx.x; q < S * S; q += blockDim.x) {
      const int j = q / S - 1, i = q % S - 1;
      const bool in = i >= 0 && j >= 0 && i <= n && j <= n;
      const uint16_t cd = in ? lv[k].code[lv[k].L.idx(i, j)] : (uint16_t)0;
      int tag = -2;
      if (cd == 1) tag = -1;
      else if (cd >= 2) tag = lv[k].tile_base[lv[k].L.tile_of(i, j)] + cd - 2;
      G[q] = (int16_t)tag;
      if (tag >= 0) atomicAdd(&cnt[k * 4 + (i & 1) + 2 * (j & 1)], 1);
    }
  }
  __syncthreads();
  if (threadIdx.x < lay.nlev) {
    const int k = threadIdx.x;
    int acc = 0;
    for (int c = 0; c < 4; ++c) {
      off[k * 5 + c] = acc;
      cur[k * 4 + c] = acc;
      acc += cnt[k * 4 + c];
    }
    off[k * 5 + 4] = acc;
  }
  __syncthreads();
  for (int k = 0; k < lay.nlev; ++k) {
    const int n = lay.n[k], S = n + 3;
    const int16_t* G = reinterpret_cast<const int16_t*>(image + lay.G[k]);
    uint16_t* BL = reinterpret_cast<uint16_t*>(image + lay.BL[k]);
    for (int q = threadIdx.x; q < S * S; q += blockDim.x) {
      if (G[q] < 0) continue;
      const int j = q / S - 1, i = q % S - 1;
      BL[atomicAdd(&cur[k * 4 + (i & 1) + 2 * (j & 1)], 1)] = (uint16_t)q;
    }
  }
}

}  // namespace

bool tail_layout(const int* n, const int* n_bnd, int nlev, int m, size_t elem, size_t max_bytes,
                 TailLayout* out) {
  if (nlev < 1 || nlev > MG_TAIL_MAX_LEVELS) return false;
  for (int rows = 1; rows >= 0; --rows) {
    for (int ainv = 1; ainv >= 0; --ainv) {
      TailLayout t;
      t.nlev = nlev;
      size_t o = 0;
      for (int k = 0; k < nlev; ++k) {
        t.n[k] = n[k];
        t.n_bnd[k] = n_bnd[k];
        const size_t S = (size_t)n[k] + 3;
        t.G[k] = o;
        o = align16(o + S * S * sizeof(int16_t));
      }
      for (int k = 0; k < nlev; ++k) {
        t.BL[k] = o;
        o = align16(o + (size_t)n_bnd[k] * sizeof(uint16_t));
      }
      t.off = o;
      o = align16(o + (size_t)nlev * 5 * sizeof(int));
      t.rows_in_smem = rows != 0;
      for (int k = 0; k < nlev && rows; ++k) {
        t.rows[k] = o;
        o = align16(o + (size_t)n_bnd[k] * MG_ROW * elem);
      }
      t.ainv_in_smem = ainv != 0;
      if (ainv) {
        t.Ainv = o;
        o = align16(o + (size_t)m * m * sizeof(double));
      }
      t.image_bytes = o;
      for (int k = 0; k < nlev; ++k) {
        const size_t S = (size_t)n[k] + 3;
        t.U[k] = o;
        o = align16(o + S * S * elem);
        t.F[k] = o;
        o = align16(o + S * S * elem);
      }
      t.R = o;
      const size_t S0 = (size_t)n[0] + 3;
      o = align16(o + S0 * S0 * elem);
      t.total = o + kSmemSlack;
      if (t.total <= max_bytes) {
        *out = t;
        return true;
      }
    }
  }
  return false;
}

void launch_tail_image(const TailLayout& lay, const TailLevelSrc* lv, unsigned char* image,
                       cudaStream_t st) {
  TailLevelSrc l[MG_TAIL_MAX_LEVELS] = {};
  for (int k = 0; k < lay.nlev; ++k) l[k] = lv[k];
  k_tail_image<<<1, kThreads, 0, st>>>(lay, l[0], l[1], l[2], l[3], l[4], l[5], image);
}

template <class T>
cudaError_t configure_tail(size_t smem) {
  return raise_smem_limit(k_tail<T>, (int)smem);
}

template <class T>
void launch_tail(const TailArgs<T>& a, cudaStream_t st) {
  launch_pdl(k_tail<T>, 1, TailBlock<T>::threads, a.lay.total, st, a);
}

template cudaError_t configure_tail<float>(size_t);
template cudaError_t configure_tail<double>(size_t);
template void launch_tail<float>(const TailArgs<float>&, cudaStream_t);
template void launch_tail<double>(const TailArgs<double>&, cudaStream_t);

// binds the bounds-checked build's device error word (see common.cuh)
MG_BOUNDS_BINDER(bind_bounds_tail)
