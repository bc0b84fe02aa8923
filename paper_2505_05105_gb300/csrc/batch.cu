// Batched solves: one persistent kernel V-cycles many independent geometries.
//
// Each block takes a whole problem from a work queue (largest first) and
// runs its entire mixed-precision solve without leaving the kernel: the fp64
// residual r = F - A u of the fine level, its l_inf norm and the stop test
// ||r|| / ||F|| <= tol; groups of fp32 V(nu1, nu2)-cycles on A e = sigma r
// (the group size predicted from the contraction seen so far, as in the
// single-problem solver); u += e / sigma in fp64.  The problems are
// independent, so blocks never wait for one another.  Per V-cycle, the
// levels above 64 x 64 cells are smoothed block-wide in global memory (a
// 4-colour Gauss-Seidel sweep over the level's active tiles with the colour's
// cut-cell vertices from a list, then eta sweeps over those vertices,
// Sec. 4.1 and Sec. 5.3), restricted (R = P^T) and prolongated (P) as in
// Sec. 5.1; the levels from 64 x 64 down run in shared memory by the tail
// code (tail_impl.cuh).  The arithmetic is that of the single-problem
// kernels.
#include "batch.cuh"
#include "ghostmg.h"
#include "rhs_impl.cuh"
#include "tail_impl.cuh"

namespace {

// ---------------------------------------------------------------------------
// Threads of a member: one block, or the blocks of a thread-block cluster
// that share a large member (each block its own SM).  Cluster members stay in
// step through the hardware cluster barrier (release / acquire at cluster
// scope, which orders their global-memory accesses); shared values go
// through distributed shared memory.

struct Team {
  int t0, ts;      // this thread's first node index and the stride over the team
  int rank, nr;    // block rank in the team and team size (1: a block alone)
};

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void team_sync(const Team& tm) {
  if (tm.nr > 1) cluster_sync_all();
  else __syncthreads();
}

// stores v into the shared word at p in block `rank` of the cluster
__device__ __forceinline__ void dsmem_store_u32(void* p, unsigned rank, unsigned v) {
  unsigned a = (unsigned)__cvta_generic_to_shared(p), ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(ra), "r"(v) : "memory");
}

// stores v into block `rank`'s shared word at the shared-window address a
__device__ __forceinline__ void dsmem_store_f32(unsigned a, unsigned rank, float v) {
  unsigned ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(ra), "f"(v) : "memory");
}

__device__ __forceinline__ void dsmem_store_f64(void* p, unsigned rank, double v) {
  unsigned a = (unsigned)__cvta_generic_to_shared(p), ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(ra), "d"(v) : "memory");
}

__device__ __forceinline__ double block_max(double v) {
  __shared__ double s[32];
  __syncthreads();
  v = warp_max(v);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0.0;
    v = warp_max(v);
    if (threadIdx.x == 0) s[0] = v;
  }
  __syncthreads();
  return s[0];
}

constexpr int kMaxCluster = 16;

// max over the team (every block gets the result); `parity` alternates the
// exchange slots between consecutive reductions
__device__ double team_max(double v, const Team& tm, int& parity) {
  v = block_max(v);
  if (tm.nr == 1) return v;
  __shared__ double slot[2][kMaxCluster];
  const int q = parity;
  parity ^= 1;
  if (threadIdx.x < (unsigned)tm.nr) dsmem_store_f64(&slot[q][tm.rank], threadIdx.x, v);
  cluster_sync_all();
  double m = 0.0;
  for (int r = 0; r < tm.nr; ++r) m = fmax(m, slot[q][r]);
  return m;
}

// ---------------------------------------------------------------------------
// Level routines.  Node q of the active tiles: tile xy[q >> 11] (i0 | j0 << 16),
// node (q & 63, (q >> 6) & 31) in it; node q of colour (ci, cj): tile
// xy[q >> 9], lattice node (q & 31, (q >> 5) & 15).  kU nodes per thread are
// in flight at once (all their loads issued before the arithmetic): 4 with up
// to 512 threads per block, 2 with 1024 (64 registers per thread).

__device__ __forceinline__ int tile_pos(const unsigned* __restrict__ xy, int q, int total, int n,
                                        int P, bool& ok, int& i, int& j) {
  const bool in = q < total;
  const unsigned t = in ? __ldg(xy + (q >> 11)) : 0u;
  i = (int)(t & 0xffffu) + (q & 63);
  j = (int)(t >> 16) + ((q >> 6) & 31);
  ok = in && i <= n && j <= n;
  return (j + MG_G) * P + (i + MG_G);
}

__device__ __forceinline__ int tile_pos(const unsigned* __restrict__ xy, int q, int total, int n,
                                        int P, bool& ok) {
  int i, j;
  return tile_pos(xy, q, total, n, P, ok, i, j);
}

__device__ __forceinline__ int colour_pos(const unsigned* __restrict__ xy, int q, int total,
                                          int ci, int cj, int n, int P, bool& ok) {
  const bool in = q < total;
  const unsigned t = in ? __ldg(xy + (q >> 9)) : 0u;
  const int i = (int)(t & 0xffffu) + 2 * (q & 31) + ci;
  const int j = (int)(t >> 16) + 2 * ((q >> 5) & 15) + cj;
  ok = in && i <= n && j <= n;
  return (j + MG_G) * P + (i + MG_G);
}

template <class T>
__device__ __forceinline__ T row_apply(const T* __restrict__ R, const T* U, int P) {
  return R[0] * U[-P - 1] + R[1] * U[-P] + R[2] * U[-P + 1] + R[3] * U[-1] + R[4] * U[0] +
         R[5] * U[1] + R[6] * U[P - 1] + R[7] * U[P] + R[8] * U[P + 1];
}

template <class T>
__device__ __forceinline__ T sum8(const T* U, int P) {
  return ((U[-1] + U[1]) + (U[-P] + U[P])) + ((U[-P - 1] + U[-P + 1]) + (U[P - 1] + U[P + 1]));
}

// Gauss-Seidel update of boundary node g with its row R and right-hand side f
__device__ __forceinline__ void row_update(float* u, int g, const float* __restrict__ R, float f,
                                           int P) {
  const float* U = u + g;
  const float acc = row_apply(R, U, P);
  u[g] = U[0] + (f - acc) * __ldg(R + 9);
}

// interior nodes of colour (ci, cj): the constant stencil 1/3 [-1 .. 8 .. -1]
template <int kU>
__device__ __forceinline__ void colour_interior(const BatchLevel& v, int ci, int cj,
                                                const Team& tm) {
  const int P = v.L.pitch, n = v.L.n, total = v.n_active * 512;
  float* u = v.u;
  for (int q0 = tm.t0; q0 < total; q0 += kU * tm.ts) {
    int g[kU];
    bool ok[kU];
#pragma unroll
    for (int k = 0; k < kU; ++k) g[k] = colour_pos(v.xy, q0 + k * tm.ts, total, ci, cj, n, P, ok[k]);
    float s[kU], f[kU];
    bool in[kU];
#pragma unroll
    for (int k = 0; k < kU; ++k) {
      in[k] = false;
      s[k] = 0.f;
      f[k] = 0.f;
      if (ok[k]) {
        in[k] = __ldg(v.code + g[k]) == 1;
        f[k] = v.F[g[k]];
        s[k] = sum8(u + g[k], P);
      }
    }
#pragma unroll
    for (int k = 0; k < kU; ++k)
      if (in[k]) u[g[k]] = (3.f * f[k] + s[k]) * 0.125f;
  }
}

// The Gauss-Seidel update of one cut-cell vertex in the eta phases from its
// row R (9 coefficients in row order, then the inverse diagonal), the 9
// stencil values x (row order) and its right-hand side f.  Every eta path
// evaluates this one expression, so that the result does not depend on the
// path a launch shape selects.
__device__ __forceinline__ float eta_row(const float (&R)[10], const float (&x)[9], float f) {
  const float acc = R[0] * x[0] + R[1] * x[1] + R[2] * x[2] + R[3] * x[3] + R[4] * x[4] +
                    R[5] * x[5] + R[6] * x[6] + R[7] * x[7] + R[8] * x[8];
  return x[4] + (f - acc) * R[9];
}

// Rows of the listed boundary nodes are read from a copy laid out by
// coefficient (R[k * n + e] for list entry e of n), so that a warp's loads of
// one coefficient are contiguous.
__device__ __forceinline__ void row_update_eta(float* u, int g, const float* __restrict__ R, int n,
                                               float f, int P) {
  const float* U = u + g;
  float r[10], x[9];
#pragma unroll
  for (int k = 0; k < 10; ++k) r[k] = __ldg(R + k * n);
  const int d[9] = {-P - 1, -P, -P + 1, -1, 0, 1, P - 1, P, P + 1};
#pragma unroll
  for (int k = 0; k < 9; ++k) x[k] = U[d[k]];
  u[g] = eta_row(r, x, f);
}

// The same update on values held in a shared-memory window: sl[k] is the
// window index of the node at stencil position k (row order)
__device__ __forceinline__ void row_update_win(float* w, const uint16_t* __restrict__ sl,
                                               const float* __restrict__ R, int n, float f) {
  uint16_t q[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) q[k] = __ldg(sl + k);
  float r[10], x[9];
#pragma unroll
  for (int k = 0; k < 10; ++k) r[k] = __ldg(R + k * n);
#pragma unroll
  for (int k = 0; k < 9; ++k) x[k] = w[q[k]];
  w[q[4]] = eta_row(r, x, f);
}

// The eta phases of a level (Sec. 5.3) in shared memory.  A block holds the
// window (the cut-cell vertices and their neighbours, gathered from u), the
// right-hand sides of its vertices (gathered from F) and their static image,
// built at setup and brought in by one bulk copy: their rows, positions and
// the window indices of their three stencil rows (the three nodes of a
// stencil row are consecutive in the sorted window).  With the solo image
// the lead block does every vertex (a phase ends on its block barrier; the
// team waits at the caller's team barrier).  With the pair images, in a team
// of two blocks, each block holds the whole window and the vertices j mod 2 =
// rank of each colour group: a vertex's new value goes to both windows (the
// other's through distributed shared memory) and each phase ends on the team
// barrier, which orders those stores before the next phase's loads.  At the
// end the vertices are written back to u.  Returns false, doing nothing,
// when the level has no image for this team; when it returns true, the
// tail's static image in the same shared memory is gone.
__device__ bool eta_resident(const BatchLevel& v, int eta, const Team& tm, unsigned char* smem,
                             int cap, unsigned* err) {
  const bool solo = v.rimg[0] != nullptr;
  if (!solo && !(tm.nr == 2 && v.rimg[1] != nullptr)) return false;
  const int nr = solo ? 1 : 2;
  if (v.win_n <= 0 || eta_resident_bytes(v.win_n, v.boff, nr) > (size_t)cap) return false;
  if (solo && tm.rank != 0) return true;
  const int rank = solo ? 0 : tm.rank;
  auto sync = [&]() {
    if (solo) __syncthreads();
    else team_sync(tm);
  };
  int lb[5], le = 0;
  lb[0] = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int cnt = v.boff[c + 1] - v.boff[c];
    le += (cnt + nr - 1) / nr;
    lb[c + 1] = lb[c] + (cnt - rank + nr - 1) / nr;   // entries j = k nr + rank < cnt
  }
  const EtaResidentLayout lay = eta_resident_layout(v.win_n, le);
  const unsigned char* img = v.rimg[solo ? 0 : 1 + rank];
  float* sw = reinterpret_cast<float*>(smem);
  const float* sR = reinterpret_cast<const float*>(smem + lay.rows);
  const int* sP = reinterpret_cast<const int*>(smem + lay.pos);
  const uint16_t* sS = reinterpret_cast<const uint16_t*>(smem + lay.slot);
  float* sF = reinterpret_cast<float*>(smem + lay.f);
  const int* gP = reinterpret_cast<const int*>(img + (lay.pos - lay.rows));
  __shared__ uint64_t bar;
  __shared__ int bad;
  // earlier generic accesses of this shared memory before the bulk copy
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    const size_t bytes = lay.f - lay.rows;
    bad = !bulk_ok(smem + lay.rows, img, bytes);
    if (bad) {
      atomicOr(err, DEV_ERR_ALIGN);
      mbar_arrive_expect_tx(&bar, 0);
    } else {
      mbar_arrive_expect_tx(&bar, (uint32_t)bytes);
      for (size_t o = 0; o < bytes; o += 65536) {
        const size_t n = bytes - o < 65536 ? bytes - o : 65536;
        bulk_load(smem + lay.rows + o, img + o, (uint32_t)n, &bar);
      }
    }
  }
  // the barrier initialised (and `bad` set) before any thread waits on it
  __syncthreads();
  // meanwhile the window and the right-hand sides, 8 nodes per thread in
  // flight
  constexpr int GU = 8;
  const int ng = v.win_n + lb[4];
  for (int k0 = threadIdx.x; k0 < ng; k0 += GU * blockDim.x) {
    int a[GU];
#pragma unroll
    for (int q = 0; q < GU; ++q) {
      const int k = k0 + q * blockDim.x;
      a[q] = k < v.win_n ? __ldg(v.win + k) : k < ng ? __ldg(gP + (k - v.win_n)) : -1;
    }
    float x[GU];
#pragma unroll
    for (int q = 0; q < GU; ++q) {
      const int k = k0 + q * blockDim.x;
      x[q] = a[q] < 0 ? 0.f : k < v.win_n ? v.u[a[q]] : v.F[a[q]];
    }
#pragma unroll
    for (int q = 0; q < GU; ++q) {
      const int k = k0 + q * blockDim.x;
      if (a[q] >= 0) {
        if (k < v.win_n) sw[k] = x[q];
        else sF[k - v.win_n] = x[q];
      }
    }
  }
  const bool ok = mbar_wait(&bar, 0, kMbarSpinLimit);
  const bool fail = __syncthreads_or(!ok || bad) != 0;
  if (threadIdx.x == 0) {
    if (!ok) {
      atomicOr(err, DEV_ERR_TIMEOUT);
      mbar_wait(&bar, 0);        // bounded: let copies still in flight land
    }
    mbar_inval(&bar);
  }
  // every block's window complete before any block's first update lands in it
  sync();
  const unsigned swa = (unsigned)__cvta_generic_to_shared(sw);
  for (int it = 0; it < eta; ++it) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      for (int x = lb[c] + threadIdx.x; x < lb[c + 1] && !fail; x += blockDim.x) {
        const int b0 = sS[x], b1 = sS[le + x], b2 = sS[2 * le + x];
        float r[10], xv[9];
#pragma unroll
        for (int k = 0; k < 10; ++k) r[k] = sR[k * le + x];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          xv[k] = sw[b0 + k];
          xv[3 + k] = sw[b1 + k];
          xv[6 + k] = sw[b2 + k];
        }
        const float nv = eta_row(r, xv, sF[x]);
        sw[b1 + 1] = nv;
        if (!solo) dsmem_store_f32(swa + 4u * (unsigned)(b1 + 1), (unsigned)(rank ^ 1), nv);
      }
      sync();
    }
  }
  if (!fail)
    for (int x = threadIdx.x; x < lb[4]; x += blockDim.x) v.u[sP[x]] = sw[sS[le + x] + 1];
  return true;
}

// One smoothing step of a level in global memory (Sec. 4.1, Sec. 5.3): four
// colour phases (interior nodes by the team, the colour's cut-cell vertices
// from the level's list by the lead block), then eta colour phases over the
// cut-cell vertices by the lead block alone.  The lead block's threads keep
// the position and F of one listed node per colour in registers for the
// whole step; longer colour lists go through the loops marked `more`.  When
// the level has a window (v.win_n > 0) the eta phases run in shared memory
// (sw): the cut-cell vertices and their neighbours are gathered once, the
// phases update the window (only the vertices change: their neighbours that
// are not vertices are constant during these phases), and the vertices are
// written back.  The eta phases run on every block of the team from shared
// memory (eta_resident) where the level's data fit in cap bytes; the return
// value says whether they did (the tail's image at smem is then gone).
template <int kU>
__device__ bool smooth_level(const BatchLevel& v, int eta, const Team& tm, float* sw,
                             unsigned char* smem, int cap, unsigned* err) {
  const int P = v.L.pitch;
  const bool lead = tm.rank == 0;
  int mc = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) mc = max(mc, v.boff[c + 1] - v.boff[c]);
  const int nt = min((int)blockDim.x, max(32, (mc + 31) & ~31));
  const bool own = lead && (int)threadIdx.x < nt;
  const bool more = mc > nt;
  const int nb = v.boff[4];
  int pos[4];
  float fv[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int e = v.boff[c] + threadIdx.x;
    pos[c] = -1;
    fv[c] = 0.f;
    if (own && e < v.boff[c + 1]) {
      pos[c] = __ldg(v.blist + e).x;
      fv[c] = v.F[pos[c]];
    }
  }
  auto listed = [&](int c, int stride) {
    if (pos[c] >= 0) row_update_eta(v.u, pos[c], v.srows + v.boff[c] + threadIdx.x, nb, fv[c], P);
    if (more)
      for (int e = v.boff[c] + nt + threadIdx.x; e < v.boff[c + 1]; e += stride) {
        const int g = __ldg(v.blist + e).x;
        row_update_eta(v.u, g, v.srows + e, nb, v.F[g], P);
      }
  };
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    colour_interior<kU>(v, c & 1, c >> 1, tm);
    if (own) listed(c, nt);
    team_sync(tm);
  }
  const bool resident = eta > 0 && eta_resident(v, eta, tm, smem, cap, err);
  if (!resident && eta > 0 && v.win_n > 0) {
    if (lead) {
      // gather: 8 nodes per thread in flight
      constexpr int GU = 8;
      for (int k0 = threadIdx.x; k0 < v.win_n; k0 += GU * blockDim.x) {
        int a[GU];
#pragma unroll
        for (int q = 0; q < GU; ++q) {
          const int k = k0 + q * blockDim.x;
          a[q] = k < v.win_n ? __ldg(v.win + k) : -1;
        }
        float x[GU];
#pragma unroll
        for (int q = 0; q < GU; ++q) x[q] = a[q] >= 0 ? v.u[a[q]] : 0.f;
#pragma unroll
        for (int q = 0; q < GU; ++q)
          if (a[q] >= 0) sw[k0 + q * blockDim.x] = x[q];
      }
      __syncthreads();
      if (own) {
        for (int it = 0; it < eta; ++it)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int e = v.boff[c] + threadIdx.x;
            if (pos[c] >= 0)
              row_update_win(sw, v.wslot + (size_t)e * 10, v.srows + e, nb, fv[c]);
            if (more)
              for (int e2 = e + nt; e2 < v.boff[c + 1]; e2 += nt)
                row_update_win(sw, v.wslot + (size_t)e2 * 10, v.srows + e2, nb,
                               v.F[__ldg(v.blist + e2).x]);
            if (nt == 32) __syncwarp();
            else asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
          }
      }
      __syncthreads();
      // scatter the updated vertices, 4 per thread in flight
      constexpr int SU = 4;
      for (int e0 = threadIdx.x; e0 < nb; e0 += SU * blockDim.x) {
        int g[SU], q[SU];
#pragma unroll
        for (int k = 0; k < SU; ++k) {
          const int e = e0 + k * blockDim.x;
          g[k] = e < nb ? __ldg(v.blist + e).x : -1;
          q[k] = e < nb ? __ldg(v.wslot + (size_t)e * 10 + 4) : 0;
        }
#pragma unroll
        for (int k = 0; k < SU; ++k)
          if (g[k] >= 0) v.u[g[k]] = sw[q[k]];
      }
    }
  } else if (!resident && eta > 0 && own) {
    for (int it = 0; it < eta; ++it)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        listed(c, nt);
        if (nt == 32) __syncwarp();
        else asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory");
      }
  }
  if (eta > 0) team_sync(tm);
  return resident;
}

__device__ void zero_level(const BatchLevel& v, const Team& tm) {
  const int total = v.n_active * 2048;
  for (int q = tm.t0; q < total; q += tm.ts) {
    bool ok;
    const int g = tile_pos(v.xy, q, total, v.L.n, v.L.pitch, ok);
    if (ok) v.u[g] = 0.f;
  }
}

// F_2h = P^T (F - A u) (Sec. 5.1): the residual of the active tiles into
// scr, then the 9-point restriction (weights 1, 1/2, 1/4) at every node of
// the coarse level's active tiles.
template <int kU>
__device__ void resid_restrict_level(const BatchLevel& v, const Layout& Lc, const unsigned* cxy,
                                     int nc_act, float* Fc, const Team& tm) {
  const int P = v.L.pitch, n = v.L.n, total = v.n_active * 2048;
  for (int q0 = tm.t0; q0 < total; q0 += kU * tm.ts) {
    int g[kU], ti[kU];
    bool ok[kU];
#pragma unroll
    for (int k = 0; k < kU; ++k) {
      int i, j;
      g[k] = tile_pos(v.xy, q0 + k * tm.ts, total, n, P, ok[k], i, j);
      ti[k] = v.L.tile_of(i, j);
    }
    float r[kU], f[kU], s[kU], c0[kU];
    uint16_t cd[kU];
#pragma unroll
    for (int k = 0; k < kU; ++k) {
      cd[k] = 0;
      f[k] = s[k] = c0[k] = 0.f;
      if (ok[k]) {
        cd[k] = __ldg(v.code + g[k]);
        f[k] = v.F[g[k]];
        c0[k] = v.u[g[k]];
        s[k] = sum8(v.u + g[k], P);
      }
    }
#pragma unroll
    for (int k = 0; k < kU; ++k) {
      r[k] = 0.f;
      if (cd[k] == 1) {
        r[k] = f[k] - (8.f * c0[k] - s[k]) * (1.f / 3.f);
      } else if (cd[k] >= 2) {
        const float* R = v.rows + (size_t)(__ldg(v.tile_base + ti[k]) + cd[k] - 2) * MG_ROW;
        r[k] = f[k] - row_apply(R, v.u + g[k], P);
      }
      if (ok[k]) v.scr[g[k]] = r[k];
    }
  }
  team_sync(tm);
  const int Pc = Lc.pitch, nc = Lc.n, totc = nc_act * 2048;
  for (int q0 = tm.t0; q0 < totc; q0 += kU * tm.ts) {
    int gc[kU], fo[kU];
    bool ok[kU];
#pragma unroll
    for (int k = 0; k < kU; ++k) {
      int I, J;
      gc[k] = tile_pos(cxy, q0 + k * tm.ts, totc, nc, Pc, ok[k], I, J);
      fo[k] = (2 * J + MG_G) * P + (2 * I + MG_G);
    }
    float rc[kU];
#pragma unroll
    for (int k = 0; k < kU; ++k) {
      rc[k] = 0.f;
      if (ok[k]) {
        const float* R = v.scr + fo[k];
        rc[k] = R[0] + 0.5f * ((R[-1] + R[1]) + (R[-P] + R[P])) +
                0.25f * ((R[-P - 1] + R[-P + 1]) + (R[P - 1] + R[P + 1]));
      }
    }
#pragma unroll
    for (int k = 0; k < kU; ++k)
      if (ok[k]) Fc[gc[k]] = rc[k];
  }
  team_sync(tm);
}

// u += P e_2h on the DOFs of the active tiles (the arithmetic of k_prolong)
template <int kU>
__device__ void prolong_level(const BatchLevel& v, const Layout& Lc, const float* ec,
                              const Team& tm) {
  const int P = v.L.pitch, n = v.L.n, total = v.n_active * 2048, Pc = Lc.pitch;
  for (int q0 = tm.t0; q0 < total; q0 += kU * tm.ts) {
    int g[kU], ii[kU], jj[kU];
    bool ok[kU];
#pragma unroll
    for (int k = 0; k < kU; ++k) g[k] = tile_pos(v.xy, q0 + k * tm.ts, total, n, P, ok[k], ii[k], jj[k]);
    float e[kU], u0[kU];
    bool dof[kU];
#pragma unroll
    for (int k = 0; k < kU; ++k) {
      e[k] = u0[k] = 0.f;
      dof[k] = false;
      if (ok[k]) {
        dof[k] = __ldg(v.code + g[k]) != 0;
        const int i = ii[k], j = jj[k];
        const float* E = ec + ((j >> 1) + MG_G) * Pc + ((i >> 1) + MG_G);
        u0[k] = v.u[g[k]];
        if (!(i & 1) && !(j & 1)) e[k] = E[0];
        else if (!(j & 1)) e[k] = 0.5f * (E[0] + E[1]);
        else if (!(i & 1)) e[k] = 0.5f * (E[0] + E[Pc]);
        else e[k] = 0.25f * ((E[0] + E[1]) + (E[Pc] + E[Pc + 1]));
      }
    }
#pragma unroll
    for (int k = 0; k < kU; ++k)
      if (dof[k]) v.u[g[k]] = u0[k] + e[k];
  }
  team_sync(tm);
}

// One fp32 V-cycle of problem p on the correction equation.  image_ok: the
// tail's static image is in the lead block's shared memory (the tail loads it
// otherwise; resident eta phases overwrite it).
template <int kU>
__device__ void vcycle(const BatchProblem& p, bool zero_init, unsigned char* smem,
                       bool& image_ok, const Team& tm) {
  // the eta windows use the tail's dynamic region (rewritten by every tail call)
  float* sw = reinterpret_cast<float*>(smem + p.tail.lay.U[0]);
  for (int l = 0; l < p.n_top; ++l) {
    const BatchLevel& v = p.lev[l];
    if (l > 0 || zero_init) {
      zero_level(v, tm);
      team_sync(tm);
    }
    for (int s = 0; s < p.nu1; ++s)
      if (smooth_level<kU>(v, p.eta, tm, sw, smem, p.res_cap, p.tail.err)) image_ok = false;
    if (l + 1 < p.n_top) {
      const BatchLevel& w = p.lev[l + 1];
      resid_restrict_level<kU>(v, w.L, w.xy, w.n_active, w.F, tm);
    } else {
      // the tail's top level (its active tiles; the tail ignores F off the DOFs)
      resid_restrict_level<kU>(v, p.tail.L0, p.tail_xy, p.tail_n_active, p.tail_F, tm);
    }
  }
  if (tm.rank == 0) tail_vcycle<float>(p.tail, smem, p.n_top == 0 && !zero_init, !image_ok);
  image_ok = true;
  team_sync(tm);
  for (int l = p.n_top - 1; l >= 0; --l) {
    const BatchLevel& v = p.lev[l];
    const bool next_top = l + 1 < p.n_top;
    prolong_level<kU>(v, next_top ? p.lev[l + 1].L : p.tail.L0,
                  next_top ? p.lev[l + 1].u : p.tail.u0, tm);
    for (int s = 0; s < p.nu2; ++s)
      if (smooth_level<kU>(v, p.eta, tm, sw, smem, p.res_cap, p.tail.err)) image_ok = false;
  }
}

// fp64 residual of the fine level: F32 = sigma r on the DOFs (0 elsewhere in
// the active tiles); returns ||r||_inf over the team
__device__ double residual64(const BatchProblem& p, double sigma, const Team& tm, int& parity) {
  const Layout& L = p.L0;
  const int P = L.pitch, n = L.n, total = p.n_active0 * 2048;
  constexpr int U = 2;
  double vmax = 0.0;
  for (int q0 = tm.t0; q0 < total; q0 += U * tm.ts) {
    int g[U], ti[U];
    bool ok[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      int i, j;
      g[k] = tile_pos(p.xy0, q0 + k * tm.ts, total, n, P, ok[k], i, j);
      ti[k] = L.tile_of(i, j);
    }
    double f[U], s[U], c0[U];
    uint16_t cd[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      cd[k] = 0;
      f[k] = s[k] = c0[k] = 0.0;
      if (ok[k]) {
        cd[k] = __ldg(p.code0 + g[k]);
        f[k] = p.F64[g[k]];
        c0[k] = p.u64[g[k]];
        s[k] = sum8(p.u64 + g[k], P);
      }
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      double r = 0.0;
      if (cd[k] == 1) {
        r = f[k] - (8.0 * c0[k] - s[k]) * (1.0 / 3.0);
      } else if (cd[k] >= 2) {
        const double* R = p.rows64 + (size_t)(__ldg(p.tile_base0 + ti[k]) + cd[k] - 2) * MG_ROW;
        r = f[k] - row_apply(R, p.u64 + g[k], P);
      }
      if (ok[k]) {
        vmax = fmax(vmax, fabs(r));
        p.F32[g[k]] = (float)(r * sigma);
      }
    }
  }
  return team_max(vmax, tm, parity);
}

__device__ double pow2_near_inverse(double x) {
  if (!(x > 0.0) || !isfinite(x)) return 1.0;
  int e;
  frexp(x, &e);
  return ldexp(1.0, -e);
}

// The whole mixed-precision solve of member pi by team tm (same arithmetic
// and check schedule as the single-problem solver); the result is written by
// the lead block.
template <int kU>
__device__ void solve_member(const BatchProblem& p, int pi, const unsigned* bad,
                             const double* params, int first_group, BatchResult* res,
                             unsigned char* smem, const Team& tm, int& parity) {
  const double tol = params[0];
  const int max_cycles = (int)params[1];
  const int fixed = (int)params[2];           // > 0: fixed group size
  const Layout& L = p.L0;
  const int P = L.pitch, n = L.n, total = p.n_active0 * 2048;
  const bool invalid = bad[pi] != 0;
  // u = 0 and ||F||_inf
  double fmax_ = 0.0;
  for (int q = tm.t0; q < total; q += tm.ts) {
    bool ok;
    const int g = tile_pos(p.xy0, q, total, n, P, ok);
    if (!ok) continue;
    p.u64[g] = 0.0;
    if (!invalid) fmax_ = fmax(fmax_, fabs(p.F64[g]));
  }
  const double Fn = team_max(fmax_, tm, parity);
  int cycles = 0, checks = 0, status = invalid ? MG_ERR_INVALID_ARG : MG_OK;
  double rel = 0.0;
  if (!invalid && Fn > 0.0) {
    double sigma = pow2_near_inverse(Fn), rmax = Fn, best = 1.0, rho = 0.1;
    // u = 0: the first refinement residual is F itself
    for (int q = tm.t0; q < total; q += tm.ts) {
      bool ok;
      const int g = tile_pos(p.xy0, q, total, n, P, ok);
      if (ok) p.F32[g] = (float)(p.F64[g] * sigma);
    }
    team_sync(tm);
    rel = 1.0;
    bool image_ok = false;                     // the tail's image is not loaded yet
    int kk = fixed > 0 ? fixed : first_group;
    while (rel > tol) {
      if (cycles >= max_cycles) { status = MG_ERR_NOT_CONVERGED; break; }
      kk = min(kk, max_cycles - cycles);
      for (int s = 0; s < kk; ++s) vcycle<kU>(p, s == 0, smem, image_ok, tm);
      cycles += kk;
      // u += e / sigma on the DOFs (same arithmetic as k_update)
      const double inv = 1.0 / sigma;
      for (int q0 = tm.t0; q0 < total; q0 += kU * tm.ts) {
        int g[kU];
        bool ok[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) g[k] = tile_pos(p.xy0, q0 + k * tm.ts, total, n, P, ok[k]);
        double u0[kU];
        float e[kU];
        bool dof[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) {
          dof[k] = ok[k] && __ldg(p.code0 + g[k]) != 0;
          u0[k] = ok[k] ? p.u64[g[k]] : 0.0;
          e[k] = ok[k] ? p.e32[g[k]] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < kU; ++k)
          if (dof[k]) p.u64[g[k]] = u0[k] + (double)e[k] * inv;
      }
      team_sync(tm);
      sigma = pow2_near_inverse(rmax * pow(rho, kk));
      const double rnew = residual64(p, sigma, tm, parity);
      ++checks;
      rel = rnew / Fn;
      if (!isfinite(rel) || rel > 1e3 * best) { status = MG_ERR_DIVERGED; break; }
      best = fmin(best, rel);
      rho = fmin(0.9, fmax(0.01, pow(rnew / rmax, 1.0 / kk)));
      rmax = rnew;
      if (fixed <= 0 && rel > tol) {
        const double need = log(tol / rel) / log(rho);
        kk = max(1, min(8, (int)ceil(need + 0.5)));
      }
    }
  }
  if (tm.rank == 0 && threadIdx.x == 0) {
    BatchResult r;
    r.cycles = cycles;
    r.checks = checks;
    r.status = status;
    r.pad = 0;
    r.rel_res = rel;
    res[pi] = r;
  }
  team_sync(tm);
}

// words[0]: next cooperative item (taken by cluster leaders), words[2]: next
// item taken by single blocks.  order[0 .. n_coop) are solved by whole
// clusters, the rest by single blocks.
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1)
k_batch(const BatchProblem* __restrict__ probs, const int* __restrict__ order, int count,
        int n_coop, unsigned* words, const unsigned* __restrict__ bad,
        const double* __restrict__ params, int first_group, BatchResult* res) {
  constexpr int kU = THREADS >= 1024 ? 2 : 4;
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  unsigned char* smem = smem_align128(smem_dyn);
  __shared__ unsigned cur;
  int parity = 0;
  const int nr = (int)cluster_size(), rank = (int)cluster_rank();
  if (nr > 1) {
    const Team tm{rank * (int)blockDim.x + (int)threadIdx.x, nr * (int)blockDim.x, rank, nr};
    for (;;) {
      if (rank == 0 && threadIdx.x == 0) {
        const unsigned k = atomicAdd(&words[0], 1u);
        for (int r = 0; r < nr; ++r) dsmem_store_u32(&cur, r, k);
      }
      cluster_sync_all();
      const int k = (int)cur;
      if (k >= n_coop) break;
      solve_member<kU>(probs[order[k]], order[k], bad, params, first_group, res, smem, tm, parity);
    }
  }
  const Team solo{(int)threadIdx.x, (int)blockDim.x, 0, 1};
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) cur = atomicAdd(&words[2], 1u);
    __syncthreads();
    const int k = (nr > 1 ? n_coop : 0) + (int)cur;
    if (k >= count) break;
    solve_member<kU>(probs[order[k]], order[k], bad, params, first_group, res, smem, solo, parity);
  }
}

// rows of a level's listed boundary nodes by coefficient: out[k n + e] =
// rows[blist[e].y * MG_ROW + k]
__global__ void k_soa_rows(const int2* __restrict__ blist, int n, const float* __restrict__ rows,
                           float* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float* R = rows + (size_t)blist[e].y * MG_ROW;
#pragma unroll
  for (int k = 0; k < MG_ROW; ++k) out[(size_t)k * n + e] = R[k];
}

// member p of the flattened range: off[p] <= x < off[p + 1]
template <class I>
__device__ __forceinline__ int member_of(const I* off, int count, I x) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

constexpr int kFlatThreads = 256;

__global__ void __launch_bounds__(kFlatThreads)
k_batch_rhs(const BatchProblem* __restrict__ probs, const int* __restrict__ tile_off,
            int count) {
  const int p = member_of(tile_off, count, (int)blockIdx.x);
  const BatchProblem& b = probs[p];
  rhs_tile(b.rhs, b.active0[blockIdx.x - tile_off[p]], b.f, b.g, b.F64);
}

__global__ void __launch_bounds__(kFlatThreads)
k_batch_unpack(const BatchProblem* __restrict__ probs, const size_t* __restrict__ node_off,
               int count, size_t total) {
  const size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (x >= total) return;
  const int p = member_of(node_off, count, x);
  const BatchProblem& b = probs[p];
  const int k = (int)(x - node_off[p]), W = b.L0.n + 1;
  const int j = k / W, i = k - j * W;
  const size_t g = b.L0.idx(i, j);
  b.u_out[k] = b.code0[g] ? b.u64[g] : 0.0;
}

// colour-sorted boundary-node list of one level (one block)
__global__ void k_batch_lists(Layout L, const uint16_t* __restrict__ code,
                              const int* __restrict__ tile_base, int2* __restrict__ blist,
                              int* __restrict__ boff) {
  __shared__ int cnt[4], cur[4];
  if (threadIdx.x < 4) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int W = L.n + 1;
  for (int q = threadIdx.x; q < W * W; q += blockDim.x) {
    const int j = q / W, i = q - j * W;
    if (code[L.idx(i, j)] >= 2) atomicAdd(&cnt[(i & 1) + 2 * (j & 1)], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int c = 0; c < 4; ++c) {
      boff[c] = acc;
      cur[c] = acc;
      acc += cnt[c];
    }
    boff[4] = acc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < W * W; q += blockDim.x) {
    const int j = q / W, i = q - j * W;
    const uint16_t cd = code[L.idx(i, j)];
    if (cd < 2) continue;
    const int pos = atomicAdd(&cur[(i & 1) + 2 * (j & 1)], 1);
    blist[pos] = make_int2((int)L.idx(i, j), tile_base[L.tile_of(i, j)] + cd - 2);
  }
}

}  // namespace

cudaError_t configure_batch(size_t smem) {
  cudaError_t e;
  e = raise_smem_limit(k_batch<1024>, smem);
  if (e != cudaSuccess) return e;
  e = raise_smem_limit(k_batch<512>, smem);
  if (e != cudaSuccess) return e;
  return raise_smem_limit(k_batch<256>, smem);
}

namespace {

template <int THREADS>
cudaLaunchConfig_t batch_config(const BatchTune& tune, int grid, size_t smem, cudaStream_t st,
                                cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = tune.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

template <int THREADS>
int max_clusters(const BatchTune& tune, size_t smem) {
  cudaLaunchAttribute attr[1];
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaLaunchConfig_t cfg = batch_config<THREADS>(tune, nsm, smem, nullptr, attr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_batch<THREADS>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <int THREADS>
void launch_k(const BatchProblem* probs, const int* order, int count, int n_coop,
              unsigned* words, const unsigned* bad, const double* params, const BatchTune& tune,
              int grid, size_t smem, BatchResult* res, cudaStream_t st) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = batch_config<THREADS>(tune, grid, smem, st, attr);
  cudaLaunchKernelEx(&cfg, k_batch<THREADS>, probs, order, count, n_coop, words, bad, params,
                     tune.first_group, res);
}

__global__ void k_tile_xy(Layout L, const int* __restrict__ active, int n,
                          unsigned* __restrict__ xy) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int t = active[k];
  xy[k] = (unsigned)((t % L.ntx) * MG_TX) | ((unsigned)((t / L.ntx) * MG_TY) << 16);
}

}  // namespace

int batch_max_clusters(const BatchTune& tune, size_t smem) {
  if (tune.threads >= 1024) return max_clusters<1024>(tune, smem);
  if (tune.threads >= 512) return max_clusters<512>(tune, smem);
  return max_clusters<256>(tune, smem);
}

void launch_batch(const BatchProblem* probs, const int* order, int count, int n_coop,
                  unsigned* words, const unsigned* bad, const double* params, BatchTune tune,
                  int grid, size_t smem, BatchResult* res, cudaStream_t st) {
  if (tune.threads >= 1024)
    launch_k<1024>(probs, order, count, n_coop, words, bad, params, tune, grid, smem, res, st);
  else if (tune.threads >= 512)
    launch_k<512>(probs, order, count, n_coop, words, bad, params, tune, grid, smem, res, st);
  else
    launch_k<256>(probs, order, count, n_coop, words, bad, params, tune, grid, smem, res, st);
}

void launch_soa_rows(const int2* blist, int n, const float* rows, float* out, cudaStream_t st) {
  if (n > 0) k_soa_rows<<<(n + 255) / 256, 256, 0, st>>>(blist, n, rows, out);
}

void launch_tile_xy(const Layout& L, const int* active, int n, unsigned* xy, cudaStream_t st) {
  if (n > 0) k_tile_xy<<<(n + 255) / 256, 256, 0, st>>>(L, active, n, xy);
}

static unsigned flat_grid(size_t total) {
  return (unsigned)((total + kFlatThreads - 1) / kFlatThreads);
}

void launch_batch_rhs(const BatchProblem* probs, const int* tile_off, int count, int total_tiles,
                      cudaStream_t st) {
  if (total_tiles == 0) return;
  k_batch_rhs<<<total_tiles, kFlatThreads, 0, st>>>(probs, tile_off, count);
}

void launch_batch_unpack(const BatchProblem* probs, const size_t* node_off, int count,
                         size_t total_nodes, cudaStream_t st) {
  if (total_nodes == 0) return;
  k_batch_unpack<<<flat_grid(total_nodes), kFlatThreads, 0, st>>>(probs, node_off, count,
                                                                  total_nodes);
}

void launch_batch_lists(const Layout& L, const uint16_t* code, const int* tile_base,
                        int2* blist, int* boff, cudaStream_t st) {
  k_batch_lists<<<1, 1024, 0, st>>>(L, code, tile_base, blist, boff);
}

// binds the bounds-checked build's device error word (see common.cuh)
MG_BOUNDS_BINDER(bind_bounds_batch)
