// C ABI of the ghost-FEM multigrid solver: handle, setup pipeline, V-cycle
// driver (Alg. 1 applied recursively, Sec. 3.2) and mixed-precision
// iterative refinement.  See include/ghostmg.h for the contract.
#include "ghostmg.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "cycle.cuh"
#include "internal.h"
#include "setup.cuh"
#include "fused.cuh"
#include "tail.cuh"
#include "global.cuh"

namespace {

thread_local char g_cuda_msg[256] = "";

struct Level {
  Layout L{};
  int n = 0;
  // cells
  uint8_t* cls = nullptr;
  int* cell_cut = nullptr;
  int n_cut = 0;
  int* cut_list = nullptr;
  double* Ke = nullptr;
  // nodes
  uint16_t* code = nullptr;
  int* tile_base = nullptr;
  int n_bnd = 0;
  int* bnode = nullptr;
  double* rows64 = nullptr;
  float* rows32 = nullptr;
  int n_active = 0;
  int* active = nullptr;
  uint8_t* tile_act = nullptr;  // per tile: holds a DOF
  int n_band = 0;
  int* band = nullptr;
  int* band_off = nullptr;      // [5 n_band + 1] group offsets into band_ent
  int2* band_ent = nullptr;     // boundary nodes of each band tile's region
  BandMaps bmap[2]{};           // TMA maps of u32[0..1] (fp32) and u64[0..1] (fp64)
  // the fp32 sweep's region lists (active tiles, 4-node halo)
  int* soff = nullptr;
  int2* sent = nullptr;
  // per block, whether its input region holds a boundary node that the band
  // kernel launched directly before it writes (launch_touch_flags): the
  // sweep's region (after this level's band kernel), the coarse nodes the
  // prolongating sweep reads (after the next coarser level's band kernel),
  // the residual + restriction region (after this level's band kernel)
  uint8_t* sw_touch = nullptr;
  uint8_t* pl_touch = nullptr;
  uint8_t* rr_touch = nullptr;
  unsigned long long band_seq = 0;  // launch number of this level's last band kernel
  int nbx = 0;
  int n_dof = 0;
  int n_rtiles = 0;
  int* rtiles = nullptr;        // tiles covering the coarse DOFs (fused restriction)
  // fused smoothing steps (intermediate levels with few active tiles)
  bool fused_ok = false;
  int* foff = nullptr;          // [5 tile id ..] group offsets into fent
  int2* fent = nullptr;         // boundary nodes of each tile's fused region
  // vectors
  double* u64[2] = {nullptr, nullptr};
  double* F64 = nullptr;
  double* bval64 = nullptr;
  float* u32[2] = {nullptr, nullptr};
  float* F32 = nullptr;
  float* bval32 = nullptr;
  int cur64 = 0, cur32 = 0;
};

}  // namespace

struct mg_ctx {
  cudaStream_t st = nullptr;
  int device = 0;                // current device at setup
  mg_grid grid{};
  mg_stab stab{};
  int N = 0;
  double h = 0.0;
  std::vector<Level> lev;
  double* psi_s = nullptr;
  double* Mk = nullptr;
  double* Gk = nullptr;
  double* Cl = nullptr;
  int* cfg = nullptr;
  double* Adense = nullptr;
  double* Ainv = nullptr;
  unsigned* d_err = nullptr;
  double* d_norms = nullptr;     // 8 slots of (max, sum)
  double* h_norms = nullptr;     // pinned mirror
  double* stage[4] = {nullptr, nullptr, nullptr, nullptr};
  const uint8_t* nmask_in = nullptr;   // caller's Neumann cell mask (setup only)
  double* Nk = nullptr;          // Neumann load per cut cell (null: all Dirichlet)
  int box = 0;                   // strong Dirichlet box sides
  double* adj_tmp = nullptr;     // padded fp64 scratch of mg_adjoint_bc
  int* all_tiles = nullptr;      // every tile of the fine level (box adjoint)
  std::vector<void*> allocs;
  double last_tol = 1e-10;
  double c_global = 0.0;         // the global constant used (given or computed)
  int global_steps = 0, global_cg = 0;   // Lanczos steps / CG iterations when computed
  int tail_level = -1;           // first level run by the single-block tail kernel
  TailLayout tail_lay[2];          // [float, double] shared-memory layout of the tail block
  unsigned char* tail_image[2] = {nullptr, nullptr};   // its static image
  bool fused[2] = {false, false};  // fused smoothing steps on the intermediate levels
  size_t fused_smem[2] = {0, 0};
  int fused_max_tiles = 0;         // levels with more active tiles use the separate kernels
  unsigned wait_polls = kMbarSpinLimit;   // poll budget of every bounded device wait
  float setup_ms = 0.f;
  float solve_ms = 0.f;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // side stream that zeroes a mapped host u outside the active tiles while
  // the solve runs
  cudaStream_t st_zero = nullptr;
  cudaEvent_t ev_z0 = nullptr, ev_z1 = nullptr;
  // profiling: device time per kernel class between event pairs
  bool prof = false;
  long long launches = 0;
  // kernel launches through Launch so far, never reset: a band kernel's
  // launch number tells whether it is the launch directly before another
  unsigned long long seq = 1;
  double* d_part = nullptr;     // per-tile partial sums of mg_residual's l2 norm
  struct Pend { int cls; cudaEvent_t a, b; };
  std::vector<Pend> pend;
  std::vector<cudaEvent_t> evpool;
  long long kcount[MG_PROF_SLOTS] = {};
  double kms[MG_PROF_SLOTS] = {};
};

int mg_cuda_fail(cudaError_t e) {
  snprintf(g_cuda_msg, sizeof(g_cuda_msg), "CUDA error: %s", cudaGetErrorString(e));
  return MG_ERR_CUDA;
}

namespace {

template <class T>
int dalloc(mg_ctx* c, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return MG_ERR_OUT_OF_MEMORY;
  }
  if (e != cudaSuccess) return mg_cuda_fail(e);
  c->allocs.push_back(*p);
  e = cudaMemsetAsync(*p, 0, count * sizeof(T), c->st);
  if (e != cudaSuccess) return mg_cuda_fail(e);
  return MG_OK;
}

#define TRY(expr)                 \
  do {                            \
    int rc__ = (expr);            \
    if (rc__ != MG_OK) return rc__; \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// --- bounds-checked build ------------------------------------------------------

#ifdef MG_CHECK_BOUNDS
constexpr bool kBoundsChecked = true;
#else
constexpr bool kBoundsChecked = false;
#endif
constexpr int kMaxDevices = 64;
std::mutex g_bounds_mu;
unsigned* g_bounds_word[kMaxDevices] = {};

// The current device's bounds-check word, allocated and bound to every
// translation unit on first use (checked builds; nullptr otherwise or on a
// CUDA error).
unsigned* bounds_word() {
  if (!kBoundsChecked) return nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_bounds_mu);
  if (!g_bounds_word[dev]) {
    unsigned* w = nullptr;
    if (cudaMalloc(&w, sizeof(unsigned)) != cudaSuccess) return nullptr;
    cudaError_t (*const bind[])(unsigned*) = {
        bind_bounds_api,   bind_bounds_batch, bind_bounds_cycle,   bind_bounds_fused,
        bind_bounds_global, bind_bounds_noalloc, bind_bounds_oned, bind_bounds_restrict32,
        bind_bounds_scan,
        bind_bounds_setup, bind_bounds_sweep32, bind_bounds_tail,  bind_bounds_tma};
    bool ok = cudaMemset(w, 0, sizeof(unsigned)) == cudaSuccess;
    for (auto f : bind) ok = ok && f(w) == cudaSuccess;
    if (!ok || cudaDeviceSynchronize() != cudaSuccess) {
      cudaFree(w);
      return nullptr;
    }
    g_bounds_word[dev] = w;
  }
  return g_bounds_word[dev];
}

int sync_check(mg_ctx* c) {
  cudaError_t e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return mg_cuda_fail(e);
  e = cudaGetLastError();
  if (e != cudaSuccess) return mg_cuda_fail(e);
  unsigned err = 0;
  e = cudaMemcpy(&err, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return mg_cuda_fail(e);
  if (err) {
    cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->st);
    cudaStreamSynchronize(c->st);
    if (err & DEV_ERR_NOT_SPD) return MG_ERR_NOT_SPD;
    if (err & (DEV_ERR_NAN | DEV_ERR_EDGE)) return MG_ERR_INVALID_ARG;
    if (err & DEV_ERR_TIMEOUT) return MG_ERR_TIMEOUT;
    return MG_ERR_INTERNAL;
  }
  if (kBoundsChecked) {
    // a failed index check in any kernel of this device (the word stays
    // set until mg_bounds_check resets it)
    unsigned* w = bounds_word();
    unsigned hits = 0;
    if (!w || cudaMemcpy(&hits, w, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
      return MG_ERR_CUDA;
    if (hits) return MG_ERR_INTERNAL;
  }
  return MG_OK;
}

int read_int(mg_ctx* c, const int* d, int* out) {
  cudaError_t e = cudaMemcpyAsync(out, d, sizeof(int), cudaMemcpyDeviceToHost, c->st);
  if (e != cudaSuccess) return mg_cuda_fail(e);
  e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return mg_cuda_fail(e);
  return MG_OK;
}

// --- profiling ----------------------------------------------------------------

cudaEvent_t ev_get(mg_ctx* c) {
  if (!c->evpool.empty()) {
    cudaEvent_t e = c->evpool.back();
    c->evpool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Counts `nk` kernel launches and, when profiling, brackets them with events
// attributed to class `cls`.
struct Launch {
  mg_ctx* c;
  int cls;
  cudaEvent_t a = nullptr;
  Launch(mg_ctx* ctx, int k, int nk) : c(ctx), cls(k) {
    c->launches += nk;
    if (nk) c->seq += 1;
    if (c->prof) {
      a = ev_get(c);
      cudaEventRecord(a, c->st);
    }
  }
  ~Launch() {
    if (c->prof) {
      cudaEvent_t b = ev_get(c);
      cudaEventRecord(b, c->st);
      c->pend.push_back({cls, a, b});
    }
  }
};

// Accumulates the finished event pairs (call after a stream synchronize).
void harvest(mg_ctx* c) {
  for (auto& p : c->pend) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->kms[p.cls] += ms;
      c->kcount[p.cls] += 1;
    } else {
      cudaGetLastError();
    }
    c->evpool.push_back(p.a);
    c->evpool.push_back(p.b);
  }
  c->pend.clear();
}

// Boundary-node lists (5 groups per tile, see launch_region_list) of the
// regions of halo H around ntl tiles of tw x th nodes (tiles == nullptr: all
// tiles, indexed by tile id).
int build_region_lists(mg_ctx* c, Level& V, const int* tiles, int ntl, int tpr, int tw, int th,
                       int H, int** off, int2** ent) {
  const size_t ng = 5 * (size_t)ntl;
  int *gcnt, *gtmp;
  TRY(dalloc(c, &gcnt, ng));
  TRY(dalloc(c, &gtmp, scan_tmp_ints(ng) + 8));
  TRY(dalloc(c, off, ng + 1));
  launch_region_list(V.L, V.code, V.tile_base, tiles, ntl, tpr, tw, th, H, gcnt, nullptr, nullptr,
                     c->st);
  exclusive_scan_int(gcnt, *off, *off + ng, ng, gtmp, c->st);
  int nent = 0;
  TRY(read_int(c, *off + ng, &nent));
  TRY(dalloc(c, ent, (size_t)nent));
  launch_region_list(V.L, V.code, V.tile_base, tiles, ntl, tpr, tw, th, H, nullptr, *off, *ent,
                     c->st);
  return MG_OK;
}

// Codes, boundary rows and tile lists of a level whose cells are ready.
int build_nodes(mg_ctx* c, Level& V) {
  const Layout& L = V.L;
  const int ntiles = L.ntx * L.nty;
  int *tile_cnt, *d_cnt, *tmp;
  uint8_t* tile_active;
  TRY(dalloc(c, &tile_cnt, ntiles));
  TRY(dalloc(c, &V.tile_base, ntiles));
  TRY(dalloc(c, &tile_active, ntiles));
  TRY(dalloc(c, &d_cnt, 4));
  size_t tmpn = scan_tmp_ints((size_t)ntiles);
  int nbx = (V.n + 1 + 31) / 32, nby = nbx;
  size_t tmpn2 = scan_tmp_ints((size_t)nbx * nby);
  TRY(dalloc(c, &tmp, (tmpn > tmpn2 ? tmpn : tmpn2) + 8));
  CellData cd{V.n, V.cls, V.cell_cut, V.Ke, c->box};
  launch_tile_counts(cd, L, tile_cnt, tile_active, d_cnt + 0, c->st);
  exclusive_scan_int(tile_cnt, V.tile_base, d_cnt + 1, (size_t)ntiles, tmp, c->st);
  int h_cnt[2];
  MG_CUDA_TRY(cudaMemcpyAsync(h_cnt, d_cnt, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->st));
  MG_CUDA_TRY(cudaStreamSynchronize(c->st));
  V.n_dof = h_cnt[0];
  V.n_bnd = h_cnt[1];
  TRY(dalloc(c, &V.code, L.size()));
  TRY(dalloc(c, &V.rows64, (size_t)V.n_bnd * MG_ROW));
  TRY(dalloc(c, &V.rows32, (size_t)V.n_bnd * MG_ROW));
  TRY(dalloc(c, &V.bnode, (size_t)V.n_bnd));
  launch_tile_assemble(cd, L, V.tile_base, V.code, V.rows64, V.bnode, c->d_err, c->st);
  launch_rows_to_f32(V.rows64, V.rows32, (size_t)V.n_bnd * MG_ROW, c->st);
  TRY(dalloc(c, &V.active, ntiles));
  V.tile_act = tile_active;
  compact_flags_u8(tile_active, V.active, d_cnt + 2, (size_t)ntiles, tmp, nullptr, c->st);
  TRY(read_int(c, d_cnt + 2, &V.n_active));
  uint8_t* bflag;
  TRY(dalloc(c, &bflag, (size_t)nbx * nby));
  launch_band_flags(V.bnode, V.n_bnd, nbx, bflag, c->st);
  TRY(dalloc(c, &V.band, (size_t)nbx * nby));
  compact_flags_u8(bflag, V.band, d_cnt + 3, (size_t)nbx * nby, tmp, nullptr, c->st);
  TRY(read_int(c, d_cnt + 3, &V.n_band));
  V.nbx = nbx;
  if (V.n_band > 0 && c->stab.eta > 0)
    TRY(build_region_lists(c, V, V.band, V.n_band, nbx, 32, 32, 4 * c->stab.eta + 1, &V.band_off,
                           &V.band_ent));
  size_t sz = L.size();
  TRY(dalloc(c, &V.u64[0], sz));
  TRY(dalloc(c, &V.u64[1], sz));
  TRY(dalloc(c, &V.F64, sz));
  TRY(dalloc(c, &V.bval64, (size_t)V.n_bnd));
  TRY(dalloc(c, &V.u32[0], sz));
  TRY(dalloc(c, &V.u32[1], sz));
  TRY(dalloc(c, &V.F32, sz));
  TRY(dalloc(c, &V.bval32, (size_t)V.n_bnd));
  if (V.n_band > 0 && c->stab.eta > 0) {
    const int bx = band_box_x(c->stab.eta), by = band_box_y(c->stab.eta);
    for (int k = 0; k < 2; ++k) {
      TRY(make_level_map(&V.bmap[0].u[k], V.u32[k], sizeof(float), L, bx, by));
      TRY(make_level_map(&V.bmap[1].u[k], V.u64[k], sizeof(double), L, bx, by));
    }
  }
  return MG_OK;
}

int build_cut_list(mg_ctx* c, Level& V, const uint8_t* cut_flag) {
  size_t ncell = (size_t)V.n * V.n;
  int *cnt, *tmp;
  TRY(dalloc(c, &cnt, 1));
  TRY(dalloc(c, &tmp, scan_tmp_ints(ncell) + 8));
  TRY(dalloc(c, &V.cut_list, ncell));
  compact_flags_u8(cut_flag, V.cut_list, cnt, ncell, tmp, nullptr, c->st);
  TRY(read_int(c, cnt, &V.n_cut));
  TRY(dalloc(c, &V.cell_cut, ncell));
  launch_fill_int(V.cell_cut, ncell, -1, c->st);
  launch_scatter_cut_id(V.cut_list, V.n_cut, V.cell_cut, c->st);
  TRY(dalloc(c, &V.Ke, (size_t)V.n_cut * 16));
  return MG_OK;
}

// ---------------------------------------------------------------------------
// V-cycle driver, templated on the arithmetic type
// ---------------------------------------------------------------------------

template <class T> struct P;
template <> struct P<double> {
  static double* u(Level& v, int b) { return v.u64[b]; }
  static double* F(Level& v) { return v.F64; }
  static double* bval(Level& v) { return v.bval64; }
  static const double* rows(Level& v) { return v.rows64; }
  static int& cur(Level& v) { return v.cur64; }
};
template <> struct P<float> {
  static float* u(Level& v, int b) { return v.u32[b]; }
  static float* F(Level& v) { return v.F32; }
  static float* bval(Level& v) { return v.bval32; }
  static const float* rows(Level& v) { return v.rows32; }
  static int& cur(Level& v) { return v.cur32; }
};

template <class T>
OpArgs<T> op_of(Level& v) {
  OpArgs<T> o;
  o.L = v.L;
  o.code = v.code;
  o.tile_base = v.tile_base;
  o.rows = P<T>::rows(v);
  o.n_rows = v.n_bnd;
  return o;
}

// One smoothing step (full sweep, then the eta band sweeps).  With `coarse`
// the sweep first adds the prolongated correction of that level to u.
template <class T>
void smooth(mg_ctx* c, Level& v, bool zero_in, bool fine, Level* coarse = nullptr) {
  OpArgs<T> op = op_of<T>(v);
  int& cur = P<T>::cur(v);
  const int eta = c->stab.eta;
  // directly after a band kernel that writes what this sweep reads (this
  // level's, or the coarser level's when prolongating), blocks away from the
  // boundary need not wait for it
  const uint8_t* touch = nullptr;
  if (coarse) {
    if (coarse->band_seq == c->seq) touch = v.pl_touch;
  } else if (!zero_in && v.band_seq == c->seq) {
    touch = v.sw_touch;
  }
  {
    Launch k(c, fine ? MG_PROF_SWEEP : MG_PROF_LEVELS, v.n_active > 0);
    if constexpr (sizeof(T) == 4) {
      launch_gs_sweep_f32(op, v.active, v.n_active, v.u32[cur], v.u32[cur ^ 1], v.F32,
                          eta > 0 ? v.bval32 : nullptr, zero_in, coarse ? &coarse->L : nullptr,
                          coarse ? coarse->u32[coarse->cur32] : nullptr, v.soff, v.sent, touch,
                          c->st);
    } else {
      launch_gs_sweep<T>(op, v.active, v.n_active, P<T>::u(v, cur), P<T>::u(v, cur ^ 1),
                         P<T>::F(v), eta > 0 ? P<T>::bval(v) : (T*)nullptr, zero_in,
                         coarse ? &coarse->L : nullptr,
                         coarse ? P<T>::u(*coarse, P<T>::cur(*coarse)) : (const T*)nullptr,
                         c->st);
    }
  }
  cur ^= 1;
  if (eta > 0 && v.n_band > 0) {
    Launch k(c, fine ? MG_PROF_BAND : MG_PROF_LEVELS_BAND, 1);
    launch_band<T>(op, v.band, v.n_band, v.nbx, eta, P<T>::u(v, cur), P<T>::F(v), P<T>::bval(v),
                   v.band_off, v.band_ent, v.bmap[sizeof(T) == 8 ? 1 : 0], cur, c->d_err,
                   c->wait_polls, c->st);
    v.band_seq = c->seq;
  }
}

// Cycles on level l + 1 per visit of level l: gamma* of Alg. 1 (1 V, 2 W);
// the two-grid scheme (stab.cycle = 0) solves the coarse equation of the
// finest level exactly, here by kTwoGridInner V-cycles of the coarser
// hierarchy (their contraction makes the error vanish to rounding), and
// runs V-cycles below.
constexpr int kTwoGridInner = 40;
int coarse_cycles(const mg_ctx* c, int l) {
  if (c->stab.cycle == 0) return l == 0 ? kTwoGridInner : 1;
  return c->stab.cycle;
}

template <class T>
void tail_cycle(mg_ctx* c, int l, bool zero_init, bool transposed = false) {
  const int pi = sizeof(T) == 8 ? 1 : 0;
  TailArgs<T> a;
  a.lay = c->tail_lay[pi];
  for (int k = 0; k < a.lay.nlev; ++k) a.rows[k] = P<T>::rows(c->lev[l + k]);
  Level& v = c->lev[l];
  a.L0 = v.L;
  a.image = c->tail_image[pi];
  a.Ainv = c->Ainv;
  a.F0 = P<T>::F(v);
  a.u0 = P<T>::u(v, P<T>::cur(v));
  a.load_u0 = zero_init ? 0 : 1;
  a.eta = c->stab.eta;
  a.nu1 = c->stab.nu1;
  a.nu2 = c->stab.nu2;
  a.err = c->d_err;
  a.wait_polls = c->wait_polls;
  a.transposed = transposed ? 1 : 0;
  Launch k(c, MG_PROF_TAIL, 1);
  launch_tail<T>(a, c->st);
}

template <class T>
void vcycle(mg_ctx* c, int l, bool zero_init);

// One V-cycle level with fused smoothing steps: nu1 steps (the first from
// u = 0, the last also restricting the residual), recursion, nu2 steps (the
// first adding the prolongated correction).
template <class T>
void fused_cycle(mg_ctx* c, int l, bool zero_init) {
  Level& v = c->lev[l];
  Level& w = c->lev[l + 1];
  const size_t smem = c->fused_smem[sizeof(T) == 8 ? 1 : 0];
  int& cur = P<T>::cur(v);
  FusedArgs<T> a;
  a.L = v.L;
  a.code = v.code;
  a.tile_base = v.tile_base;
  a.rows = P<T>::rows(v);
  a.n_rows = v.n_bnd;
  a.loff = v.foff;
  a.lent = v.fent;
  a.eta = c->stab.eta;
  a.F = P<T>::F(v);
  a.Lc = w.L;
  a.Fc = P<T>::F(w);
  a.ec = nullptr;
  const int nu1 = c->stab.nu1, nu2 = c->stab.nu2;
  for (int s = 0; s < nu1; ++s) {
    const bool last = s == nu1 - 1;
    a.uin = P<T>::u(v, cur);
    a.uout = P<T>::u(v, cur ^ 1);
    a.tiles = last ? v.rtiles : v.active;
    Launch k(c, MG_PROF_FUSED, 1);
    launch_smooth_step<T>(a, last ? v.n_rtiles : v.n_active, zero_init && s == 0, false, last,
                          smem, c->st);
    cur ^= 1;
  }
  if (nu1 == 0) {
    if (zero_init) cudaMemsetAsync(P<T>::u(v, cur), 0, v.L.size() * sizeof(T), c->st);
    Launch k(c, MG_PROF_FUSED, w.n_active > 0);
    launch_resid_restrict<T>(op_of<T>(v), P<T>::u(v, cur), P<T>::F(v), w.L, w.active, w.n_active,
                             P<T>::F(w), nullptr, c->st);
  }
  // gamma* cycles on the coarse level (Alg. 1: 1 V, 2 W), the first from zero
  const int gs = coarse_cycles(c, l);
  for (int k = 0; k < gs; ++k) vcycle<T>(c, l + 1, k == 0);
  a.ec = P<T>::u(w, P<T>::cur(w));
  a.tiles = v.active;
  for (int s = 0; s < nu2; ++s) {
    a.uin = P<T>::u(v, cur);
    a.uout = P<T>::u(v, cur ^ 1);
    Launch k(c, MG_PROF_FUSED, 1);
    launch_smooth_step<T>(a, v.n_active, false, s == 0, false, smem, c->st);
    cur ^= 1;
  }
  if (nu2 == 0) {
    Launch k(c, MG_PROF_FUSED, v.n_active > 0);
    launch_prolong<T>(op_of<T>(v), v.active, v.n_active, P<T>::u(v, cur), w.L,
                      P<T>::u(w, P<T>::cur(w)), c->st);
  }
}

template <class T>
void vcycle(mg_ctx* c, int l, bool zero_init) {
  Level& v = c->lev[l];
  const int nlev = (int)c->lev.size();
  if (l == c->tail_level) {
    tail_cycle<T>(c, l, zero_init);
    return;
  }
  if (l == nlev - 1) {
    Launch k(c, MG_PROF_COARSE, 1);
    launch_coarse_solve<T>(v.L, c->Ainv, P<T>::F(v), P<T>::u(v, 0), c->st);
    P<T>::cur(v) = 0;
    return;
  }
  const bool fine = l == 0;
  int& cur = P<T>::cur(v);
  if (!fine && sizeof(T) == 4 && v.fused_ok) {
    fused_cycle<T>(c, l, zero_init);
    return;
  }
  if (zero_init && c->stab.nu1 == 0)
    cudaMemsetAsync(P<T>::u(v, cur), 0, v.L.size() * sizeof(T), c->st);
  for (int s = 0; s < c->stab.nu1; ++s) smooth<T>(c, v, zero_init && s == 0, fine);
  Level& w = c->lev[l + 1];
  OpArgs<T> op = op_of<T>(v);
  {
    const uint8_t* touch = v.band_seq == c->seq ? v.rr_touch : nullptr;
    Launch k(c, fine ? MG_PROF_RESTRICT : MG_PROF_LEVELS_RESTRICT, w.n_active > 0);
    launch_resid_restrict<T>(op, P<T>::u(v, cur), P<T>::F(v), w.L, w.active, w.n_active,
                             P<T>::F(w), nullptr, c->st, touch);
  }
  // gamma* cycles on the coarse level (Alg. 1: 1 V, 2 W), the first from zero
  const int gs = coarse_cycles(c, l);
  for (int k = 0; k < gs; ++k) vcycle<T>(c, l + 1, k == 0);
  if (c->stab.nu2 == 0) {
    Launch k(c, fine ? MG_PROF_PROLONG : MG_PROF_LEVELS_RESTRICT, v.n_active > 0);
    launch_prolong<T>(op, v.active, v.n_active, P<T>::u(v, cur), w.L, P<T>::u(w, P<T>::cur(w)),
                      c->st);
  }
  // the first post-smoothing sweep adds the prolongated correction itself
  for (int s = 0; s < c->stab.nu2; ++s) smooth<T>(c, v, false, fine, s == 0 ? &w : nullptr);
}

// The transposed smoothing step (fp64): the eta band sweeps first (on a
// snapshot of the boundary values in bval, since no full sweep has just
// written it), then the full sweep, all colours in the reverse order.
void smooth_transposed(mg_ctx* c, Level& v) {
  OpArgs<double> op = op_of<double>(v);
  int& cur = v.cur64;
  const int eta = c->stab.eta;
  if (eta > 0 && v.n_band > 0) {
    Launch k(c, MG_PROF_COARSE, 2);
    launch_gather_bval<double>(v.L, v.bnode, v.n_bnd, v.u64[cur], v.bval64, c->st);
    launch_band_rev<double>(op, v.band, v.n_band, v.nbx, eta, v.u64[cur], v.F64, v.bval64,
                            v.band_off, v.band_ent, v.bmap[1], cur, c->d_err, c->wait_polls,
                            c->st);
  }
  {
    Launch k(c, MG_PROF_COARSE, v.n_active > 0);
    launch_gs_sweep_rev<double>(op, v.active, v.n_active, v.u64[cur], v.u64[cur ^ 1], v.F64,
                                nullptr, c->st);
  }
  cur ^= 1;
}

// The transposed V-cycle (fp64): a V-cycle is u <- u + B (F - A u); B^T
// takes B's steps in the reverse order, each transposed: nu2 transposed
// smoothing steps, restriction, the transposed cycle(s) on the coarse level,
// prolongation, nu1 transposed smoothing steps (Sec. 3.2 with R = P^T,
// Sec. 4.1, Sec. 5.3).  A is symmetric, so k of these from w = 0 applied to
// dL/du give the gradient of k V-cycles from 0: the adjoint of the iteration.
void vcycle_transposed(mg_ctx* c, int l, bool zero_init) {
  Level& v = c->lev[l];
  const int nlev = (int)c->lev.size();
  if (l == c->tail_level) {
    tail_cycle<double>(c, l, zero_init, true);
    return;
  }
  if (l == nlev - 1) {
    Launch k(c, MG_PROF_COARSE, 1);
    launch_coarse_solve<double>(v.L, c->Ainv, v.F64, v.u64[0], c->st);
    v.cur64 = 0;
    return;
  }
  if (zero_init) cudaMemsetAsync(v.u64[v.cur64], 0, v.L.size() * sizeof(double), c->st);
  for (int s = 0; s < c->stab.nu2; ++s) smooth_transposed(c, v);
  Level& w = c->lev[l + 1];
  OpArgs<double> op = op_of<double>(v);
  {
    Launch k(c, MG_PROF_COARSE, w.n_active > 0);
    launch_resid_restrict<double>(op, v.u64[v.cur64], v.F64, w.L, w.active, w.n_active, w.F64,
                                  nullptr, c->st);
  }
  const int gs = coarse_cycles(c, l);
  for (int k = 0; k < gs; ++k) vcycle_transposed(c, l + 1, k == 0);
  {
    Launch k(c, MG_PROF_COARSE, v.n_active > 0);
    launch_prolong<double>(op, v.active, v.n_active, v.u64[v.cur64], w.L, w.u64[w.cur64],
                           c->st);
  }
  for (int s = 0; s < c->stab.nu1; ++s) smooth_transposed(c, v);
}

// ||F - A u||_inf of the fine level in fp64 (host value); optionally writes
// sigma (F - A u) in fp32 to the fine level's fp32 right-hand side.
int fine_residual(mg_ctx* c, double sigma, bool to_f32, double* rmax) {
  Level& v = c->lev[0];
  MG_CUDA_TRY(cudaMemsetAsync(c->d_norms, 0, 2 * sizeof(double), c->st));
  OpArgs<double> op = op_of<double>(v);
  {
    Launch k(c, MG_PROF_RESIDUAL, v.n_active > 0);
    // the stop test and the scaling need only max |r|
    if (to_f32)
      launch_residual<double, float>(op, v.active, v.n_active, v.u64[v.cur64], v.F64, v.F32,
                                     sigma, c->d_norms, c->st, false);
    else
      launch_residual<double, double>(op, v.active, v.n_active, v.u64[v.cur64], v.F64,
                                      (double*)nullptr, 1.0, c->d_norms, c->st, false);
  }
  MG_CUDA_TRY(cudaMemcpyAsync(c->h_norms, c->d_norms, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                              c->st));
  // a kernel of the cycles that stopped on a device error (a bounded wait
  // that ran out, a failed copy check) ends the solve at this check
  unsigned* h_err = reinterpret_cast<unsigned*>(c->h_norms + 4);
  MG_CUDA_TRY(cudaMemcpyAsync(h_err, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st));
  MG_CUDA_TRY(cudaStreamSynchronize(c->st));
  if (c->prof) harvest(c);
  *rmax = c->h_norms[0];
  if (*h_err) return sync_check(c);
  return MG_OK;
}

double pow2_near_inverse(double x) {
  if (!(x > 0.0) || !std::isfinite(x)) return 1.0;
  int e;
  std::frexp(x, &e);
  return std::ldexp(1.0, -e);
}

// One refinement step on sigma r (fp32, already in the fine level's fp32
// right-hand side): `inner` fp32 V-cycles on A e = sigma r, the first from
// e = 0, then u += e / sigma in fp64.
void refinement_step(mg_ctx* c, double sigma, int inner) {
  Level& v = c->lev[0];
  for (int s = 0; s < inner; ++s) vcycle<float>(c, 0, s == 0);
  Launch k(c, MG_PROF_UPDATE, v.n_active > 0);
  launch_update(v.L, v.active, v.n_active, v.code, v.u64[v.cur64], v.u32[v.cur32], 1.0 / sigma,
                c->st);
}

// Cycles from the current fine-level u64 with F64 set; Fn = ||F||_inf.
// The fp64 residual is checked after groups of V-cycles: a fixed group size
// (stab.inner > 0) or, by default, the size predicted to reach tol from the
// contraction per cycle seen in the previous group, plus half a cycle (first
// group 4, at most 8).  In MG_MIXED a group is one refinement step whose fp32 right-hand side
// sigma r is scaled by a power of two sigma chosen from the predicted
// residual, so the fp32 V-cycles work on O(1) values; the update divides by
// the same sigma exactly.
int solve_loop(mg_ctx* c, double Fn, double tol, int max_cycles, mg_info* info, bool u_zero,
               bool transposed = false) {
  const bool mixed = c->stab.precision == MG_MIXED && !transposed;
  const bool adaptive = c->stab.inner == 0;
  double rmax;
  int cycles = 0, checks = 0, status = MG_OK;
  double sigma = mixed ? pow2_near_inverse(Fn) : 1.0;
  if (u_zero) {
    // u = 0: the residual is F itself (bit for bit what fine_residual gives)
    Level& v = c->lev[0];
    rmax = Fn;
    if (mixed) {
      Launch kk(c, MG_PROF_RESIDUAL, v.n_active > 0);
      launch_scale_to_f32(v.L, v.active, v.n_active, v.F64, v.F32, sigma, c->st);
    }
  } else {
    TRY(fine_residual(c, sigma, mixed, &rmax));
  }
  double rel = rmax / Fn, best = rel, rho = 0.1;
  if (info) info->res_hist[0] = rel;
  int k = adaptive ? 4 : c->stab.inner;
  while (rel > tol) {
    if (cycles >= max_cycles) { status = MG_ERR_NOT_CONVERGED; break; }
    k = std::min(k, max_cycles - cycles);
    if (mixed) refinement_step(c, sigma, k);
    else if (transposed)
      for (int s = 0; s < k; ++s) vcycle_transposed(c, 0, false);
    else
      for (int s = 0; s < k; ++s) vcycle<double>(c, 0, false);
    cycles += k;
    if (mixed) sigma = pow2_near_inverse(rmax * std::pow(rho, k));
    double rnew;
    TRY(fine_residual(c, sigma, mixed, &rnew));
    ++checks;
    rel = rnew / Fn;
    if (info && checks < 64) info->res_hist[checks] = rel;
    // diverged: not finite, or grown far past the best residual seen (at the
    // rounding floor the residual only jitters within a small factor)
    if (!std::isfinite(rel) || rel > 1e3 * best) { status = MG_ERR_DIVERGED; break; }
    best = std::min(best, rel);
    rho = std::min(0.9, std::max(0.01, std::pow(rnew / rmax, 1.0 / k)));
    rmax = rnew;
    if (adaptive && rel > tol) {
      // half a cycle of margin: a V-cycle too many costs less than a check
      // plus another group
      const double need = std::log(tol / rel) / std::log(rho);
      k = std::max(1, std::min(8, (int)std::ceil(need + 0.5)));
    }
  }
  if (info) {
    info->cycles = cycles;
    info->checks = checks;
    info->rel_res = rel;
  }
  return status;
}

struct Staged {
  const double* dev = nullptr;
  bool host = false;
};

// Page-locked host memory mapped into the device address space (cudaHostAlloc,
// cudaMallocHost, cudaHostRegister, pinned torch tensors): the kernels read
// and write it in place over the host link, touching only the entries the
// computation uses, instead of copying whole arrays.  nullptr otherwise.
const double* mapped_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || a.devicePointer == nullptr) return nullptr;
  return static_cast<const double*>(a.devicePointer);
}

int stage_in(mg_ctx* c, int slot, const double* p, Staged& s) {
  size_t m = (size_t)(c->N + 1) * (c->N + 1);
  if (is_device_ptr(p)) {
    s.dev = p;
    s.host = false;
    return MG_OK;
  }
  if (const double* d = mapped_host(p)) {
    s.dev = d;
    s.host = false;
    return MG_OK;
  }
  if (!c->stage[slot]) TRY(dalloc(c, &c->stage[slot], m));
  MG_CUDA_TRY(cudaMemcpyAsync(c->stage[slot], p, m * sizeof(double), cudaMemcpyHostToDevice, c->st));
  s.dev = c->stage[slot];
  s.host = true;
  return MG_OK;
}

// output pointer: device pointer as is, host pointer via a staging slot
int stage_out(mg_ctx* c, int slot, double* p, double** dev, bool* host) {
  size_t m = (size_t)(c->N + 1) * (c->N + 1);
  if (is_device_ptr(p)) {
    *dev = p;
    *host = false;
    return MG_OK;
  }
  if (const double* d = mapped_host(p)) {
    *dev = const_cast<double*>(d);
    *host = false;
    return MG_OK;
  }
  if (!c->stage[slot]) TRY(dalloc(c, &c->stage[slot], m));
  *dev = c->stage[slot];
  *host = true;
  return MG_OK;
}

int finish_out(mg_ctx* c, double* user, const double* dev, bool host) {
  size_t m = (size_t)(c->N + 1) * (c->N + 1);
  if (host)
    MG_CUDA_TRY(cudaMemcpyAsync(user, dev, m * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  return MG_OK;
}

// The zeroing of a mapped host u outside the active tiles, on the side
// stream: start() after the inputs were read, join() makes the solver's
// stream wait for it; a call that returns early waits for it here, so no
// write to the caller's memory outlives the call.
int ensure_side_stream(mg_ctx* c) {
  if (!c->st_zero) {
    MG_CUDA_TRY(cudaStreamCreateWithFlags(&c->st_zero, cudaStreamNonBlocking));
    MG_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_z0, cudaEventDisableTiming));
    MG_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_z1, cudaEventDisableTiming));
  }
  return MG_OK;
}

struct ZeroSide {
  mg_ctx* c;
  bool running = false;
  int start(const Level& v, double* dst) {
    TRY(ensure_side_stream(c));
    MG_CUDA_TRY(cudaEventRecord(c->ev_z0, c->st));
    MG_CUDA_TRY(cudaStreamWaitEvent(c->st_zero, c->ev_z0, 0));
    launch_zero_inactive(v.L, v.tile_act, dst, 16, c->st_zero);
    c->launches += 1;
    MG_CUDA_TRY(cudaEventRecord(c->ev_z1, c->st_zero));
    running = true;
    return MG_OK;
  }
  int join() {
    if (running) MG_CUDA_TRY(cudaStreamWaitEvent(c->st, c->ev_z1, 0));
    running = false;
    return MG_OK;
  }
  ~ZeroSide() {
    if (running) cudaStreamSynchronize(c->st_zero);
  }
};

}  // namespace

// ===========================================================================
// public API
// ===========================================================================

extern "C" {

int mg_default_stab(mg_stab* out) {
  if (!out) return MG_ERR_INVALID_ARG;
  out->gamma = 2.0;
  out->alpha = 1.75;
  out->eta = 4;
  out->nu1 = 2;
  out->nu2 = 1;
  out->lambda_mode = MG_LAMBDA_LOCAL;
  out->precision = MG_FP64;
  out->max_cycles = 100;
  out->inner = 0;
  out->cycle = 1;
  out->coarse_op = MG_COARSE_GALERKIN;
  out->c_global = 0.0;
  out->fuse_max_tiles = 0;
  return MG_OK;
}

const char* mg_strerror(int code) {
  switch (code) {
    case MG_OK: return "ok";
    case MG_ERR_INVALID_ARG: return "invalid argument";
    case MG_ERR_CUDA: return g_cuda_msg[0] ? g_cuda_msg : "CUDA error";
    case MG_ERR_NOT_CONVERGED: return "not converged within max_cycles";
    case MG_ERR_DIVERGED: return "diverged";
    case MG_ERR_NOT_SPD: return "coarsest matrix not positive definite";
    case MG_ERR_TIMEOUT: return "device wait timed out";
    case MG_ERR_UNIMPLEMENTED: return "not implemented";
    case MG_ERR_INTERNAL: return "internal error";
    case MG_ERR_OUT_OF_MEMORY: return "out of device memory";
    default: return "unknown status";
  }
}

void mg_destroy(mg_handle c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  for (void* p : c->allocs) cudaFree(p);
  if (c->h_norms) cudaFreeHost(c->h_norms);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->st_zero) {
    cudaStreamSynchronize(c->st_zero);
    cudaStreamDestroy(c->st_zero);
  }
  if (c->ev_z0) cudaEventDestroy(c->ev_z0);
  if (c->ev_z1) cudaEventDestroy(c->ev_z1);
  harvest(c);
  for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
  delete c;
}

// The global constant of Sec. 5.2, Lambda_max of the fine level's global
// pencil (K, M) modulo constants, times h (cell units), on the GPU: per
// cut-cell pencils, the pencil's rows, Lanczos with inner CG solves
// (global.cu).  Work space is allocated here and released before return.
static int global_constant(mg_ctx* c, Level& v, const uint8_t* nmask, double* ch) {
  const int N = c->N;
  const size_t m = (size_t)(N + 1) * (N + 1);
  constexpr int kmax = 100, cg_max = 20000;
  constexpr double cg_tol = 1e-13;
  int blocks = 1;
  MG_CUDA_TRY(lanczos_blocks(N, &blocks));
  double *S = nullptr, *Kn = nullptr, *Mr = nullptr, *Kr = nullptr, *work = nullptr;
  double* out = nullptr;
  uint8_t* dof = nullptr;
  std::vector<uint8_t> hdof(m);
  double hout[4] = {0, 0, 0, 0};
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes > 0 ? bytes : 16);
  };
  A((void**)&S, (size_t)v.n_cut * 16 * sizeof(double));
  A((void**)&Kn, (size_t)v.n_cut * 16 * sizeof(double));
  A((void**)&Mr, m * 9 * sizeof(double));
  A((void**)&Kr, m * 9 * sizeof(double));
  A((void**)&dof, m);
  A((void**)&work, lanczos_doubles(N, kmax, blocks) * sizeof(double));
  A((void**)&out, 4 * sizeof(double));
  if (e == cudaSuccess) {
    launch_cut_pencil(c->psi_s, N, v.cut_list, v.n_cut, nmask, S, Kn, c->st);
    launch_pencil_rows(N, v.cls, v.cell_cut, S, Kn, Mr, Kr, dof, c->st);
    e = cudaMemcpyAsync(hdof.data(), dof, m, cudaMemcpyDeviceToHost, c->st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  int ndof = 0;
  for (uint8_t d : hdof) ndof += d != 0;
  if (e == cudaSuccess && ndof > 0)
    e = launch_lanczos(N, Mr, Kr, dof, ndof, work, kmax, cg_max, cg_tol, blocks, out, c->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hout, out, sizeof(hout), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  for (void* p : {(void*)S, (void*)Kn, (void*)Mr, (void*)Kr, (void*)dof, (void*)work, (void*)out})
    if (p) cudaFree(p);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return MG_ERR_OUT_OF_MEMORY;
  }
  if (e != cudaSuccess) return mg_cuda_fail(e);
  if (!(hout[0] > 0.0) || !std::isfinite(hout[0])) return MG_ERR_INTERNAL;
  *ch = hout[0];
  c->global_steps = (int)hout[1];
  c->global_cg = (int)hout[2];
  return MG_OK;
}

static int setup_impl(mg_ctx* c, const double* levelset) {
  const int N = c->N;
  MG_CUDA_TRY(cudaGetDevice(&c->device));
  MG_CUDA_TRY(cudaMallocHost((void**)&c->h_norms, 16 * sizeof(double)));
  MG_CUDA_TRY(cudaEventCreate(&c->ev0));
  MG_CUDA_TRY(cudaEventCreate(&c->ev1));
  TRY(dalloc(c, &c->d_err, 4));
  TRY(dalloc(c, &c->d_norms, 16));
  // level set on the device
  Staged ps;
  TRY(stage_in(c, 0, levelset, ps));
  TRY(dalloc(c, &c->psi_s, (size_t)(N + 1) * (N + 1)));
  launch_snap(ps.dev, c->psi_s, N, std::pow(c->h, c->stab.alpha), c->d_err, c->st, c->box);
  // fine level cells
  c->lev.emplace_back();
  {
    Level& v = c->lev[0];
    v.n = N;
    v.L = make_layout(N);
    uint8_t* cut_flag;
    TRY(dalloc(c, &v.cls, (size_t)N * N));
    TRY(dalloc(c, &cut_flag, (size_t)N * N));
    launch_cell_class(c->psi_s, N, v.cls, cut_flag, c->st);
    TRY(sync_check(c));
    TRY(build_cut_list(c, v, cut_flag));
    TRY(dalloc(c, &c->Mk, (size_t)v.n_cut * 16));
    TRY(dalloc(c, &c->Gk, (size_t)v.n_cut * 16));
    TRY(dalloc(c, &c->Cl, (size_t)v.n_cut * 4));
    TRY(dalloc(c, &c->cfg, (size_t)v.n_cut));
    const uint8_t* nmask = nullptr;
    if (c->nmask_in) {
      // the caller's cell mask (host or device), read only by this launch
      if (is_device_ptr(c->nmask_in)) {
        nmask = c->nmask_in;
      } else {
        uint8_t* d;
        TRY(dalloc(c, &d, (size_t)N * N));
        MG_CUDA_TRY(cudaMemcpyAsync(d, c->nmask_in, (size_t)N * N, cudaMemcpyHostToDevice, c->st));
        nmask = d;
      }
      TRY(dalloc(c, &c->Nk, (size_t)v.n_cut * 16));
    }
    double ch_global = -1.0;
    if (c->stab.lambda_mode == MG_LAMBDA_GLOBAL) {
      if (c->stab.c_global > 0.0) {
        ch_global = c->stab.c_global * c->h;
        c->c_global = c->stab.c_global;
      } else {
        TRY(global_constant(c, v, nmask, &ch_global));
        c->c_global = ch_global / c->h;
      }
    }
    launch_cut_cells(c->psi_s, N, c->h, c->stab.gamma, v.cut_list, v.n_cut, v.Ke, c->Mk, c->Gk,
                     c->Cl, c->cfg, nmask, c->Nk, c->st, ch_global);
    TRY(build_nodes(c, v));
  }
  // coarse levels by element-wise Galerkin products
  while (c->lev.back().n > c->grid.coarsest_cells) {
    c->lev.emplace_back();
    Level& f = c->lev[c->lev.size() - 2];
    Level& v = c->lev.back();
    v.n = f.n / 2;
    v.L = make_layout(v.n);
    uint8_t* cut_flag;
    TRY(dalloc(c, &v.cls, (size_t)v.n * v.n));
    TRY(dalloc(c, &cut_flag, (size_t)v.n * v.n));
    if (c->stab.coarse_op == MG_COARSE_REDISCRETISE) {
      // the level assembled from scratch on its own grid: the level set at
      // its nodes, snapped with h_l^alpha, its own cut cells and lambda_K
      const int step = N / v.n;
      const double hl = c->h * step;
      double *raw, *snapped, *Mk, *Gk, *Cl;
      int* cfg;
      TRY(dalloc(c, &raw, (size_t)(v.n + 1) * (v.n + 1)));
      TRY(dalloc(c, &snapped, (size_t)(v.n + 1) * (v.n + 1)));
      launch_subsample(ps.dev, N, step, raw, v.n, c->st);
      launch_snap(raw, snapped, v.n, std::pow(hl, c->stab.alpha), c->d_err, c->st, c->box);
      launch_cell_class(snapped, v.n, v.cls, cut_flag, c->st);
      TRY(sync_check(c));
      TRY(build_cut_list(c, v, cut_flag));
      TRY(dalloc(c, &Mk, (size_t)v.n_cut * 16));
      TRY(dalloc(c, &Gk, (size_t)v.n_cut * 16));
      TRY(dalloc(c, &Cl, (size_t)v.n_cut * 4));
      TRY(dalloc(c, &cfg, (size_t)v.n_cut));
      launch_cut_cells(snapped, v.n, hl, c->stab.gamma, v.cut_list, v.n_cut, v.Ke, Mk, Gk, Cl,
                       cfg, nullptr, nullptr, c->st);
    } else {
      launch_coarse_class(f.cls, f.n, v.cls, cut_flag, c->st);
      TRY(build_cut_list(c, v, cut_flag));
      CellData fd{f.n, f.cls, f.cell_cut, f.Ke, c->box};
      launch_coarse_cut(fd, v.cut_list, v.n_cut, v.n, v.Ke, c->st);
    }
    TRY(build_nodes(c, v));
  }
  {
    Level& v = c->lev.back();
    int m = (v.n + 1) * (v.n + 1);
    TRY(dalloc(c, &c->Adense, (size_t)m * m));
    TRY(dalloc(c, &c->Ainv, (size_t)m * m));
    CellData cd{v.n, v.cls, v.cell_cut, v.Ke, c->box};
    launch_coarsest(cd, c->Adense, c->Ainv, c->d_err, c->st);
  }
  MG_CUDA_TRY(configure_kernels<double>(c->stab.eta));
  MG_CUDA_TRY(configure_kernels<float>(c->stab.eta));
  {
    // fused smoothing steps on the intermediate levels, if they fit
    int dev = 0, optin = 0;
    MG_CUDA_TRY(cudaGetDevice(&dev));
    MG_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    optin -= 1024;   // static shared memory of the kernel
    int nsm = 0;
    MG_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // the fused step recomputes a wide halo per tile and holds one block per
    // SM: it pays while the level's tiles fit in one wave (a second wave
    // repeats the step's whole latency; on the 4096^2 flower, level 2's 196
    // tiles run 1 % faster in the separate sweep, band, restriction and
    // prolongation kernels)
    c->fused_max_tiles = c->stab.fuse_max_tiles == 0 ? nsm
                         : c->stab.fuse_max_tiles < 0 ? -1 : c->stab.fuse_max_tiles;
    // fp32 only: on GB300 the redundant halo arithmetic of the fused step is
    // cheap in fp32 but fp64 arithmetic is a small fraction of the fp32 rate
    for (int pi = 0; pi < 1; ++pi) {
      size_t sm = fused_smem_bytes(c->stab.eta, pi ? sizeof(double) : sizeof(float));
      if (sm <= (size_t)optin) {
        c->fused[pi] = true;
        c->fused_smem[pi] = sm;
        MG_CUDA_TRY(pi ? configure_fused<double>(sm) : configure_fused<float>(sm));
      }
    }
    const int nlev = (int)c->lev.size();
    for (int l = 1; l + 1 < nlev; ++l) {
      Level& v = c->lev[l];
      Level& w = c->lev[l + 1];
      const int nt = v.L.ntx * v.L.nty;
      uint8_t* flag;
      int *cnt, *tmp;
      TRY(dalloc(c, &flag, (size_t)nt));
      TRY(dalloc(c, &cnt, 1));
      TRY(dalloc(c, &tmp, scan_tmp_ints((size_t)nt) + 8));
      TRY(dalloc(c, &v.rtiles, (size_t)nt));
      launch_restrict_tile_flags(v.L, w.L, w.code, flag, c->st);
      compact_flags_u8(flag, v.rtiles, cnt, (size_t)nt, tmp, nullptr, c->st);
      TRY(read_int(c, cnt, &v.n_rtiles));
    }
  }
  {
    // the levels with n <= MG_TAIL_MAX_N run inside one block
    const int nlev = (int)c->lev.size();
    int t = 0;
    while (t < nlev && c->lev[t].n > MG_TAIL_MAX_N) ++t;
    // the two-grid scheme treats the finest level on its own
    if (c->stab.cycle == 0 && t == 0) t = 1;
    int dev = 0, optin = 0;
    MG_CUDA_TRY(cudaGetDevice(&dev));
    MG_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    optin -= 1024;   // static shared memory of the kernel
    // (the tail block runs a V-cycle below its top level: W-cycles use the
    // per-level kernels all the way down)
    if (c->stab.cycle != 2 && t < nlev && nlev - t <= MG_TAIL_MAX_LEVELS) {
      const int nl = nlev - t;
      int n[MG_TAIL_MAX_LEVELS], nb[MG_TAIL_MAX_LEVELS];
      TailLevelSrc src[MG_TAIL_MAX_LEVELS];
      for (int k = 0; k < nl; ++k) {
        Level& w = c->lev[t + k];
        n[k] = w.n;
        nb[k] = w.n_bnd;
        src[k] = TailLevelSrc{w.L, w.code, w.tile_base};
      }
      const int m = (n[nl - 1] + 1) * (n[nl - 1] + 1);
      TailLayout l32, l64;
      if (tail_layout(n, nb, nl, m, sizeof(float), (size_t)optin, &l32) &&
          tail_layout(n, nb, nl, m, sizeof(double), (size_t)optin, &l64)) {
        c->tail_level = t;
        const TailLayout* lay[2] = {&l32, &l64};
        for (int pi = 0; pi < 2; ++pi) {
          const TailLayout& y = *lay[pi];
          c->tail_lay[pi] = y;
          TRY(dalloc(c, &c->tail_image[pi], y.image_bytes));
          launch_tail_image(y, src, c->tail_image[pi], c->st);
          for (int k = 0; k < nl && y.rows_in_smem; ++k) {
            Level& w = c->lev[t + k];
            const size_t elem = pi ? sizeof(double) : sizeof(float);
            const void* r = pi ? (const void*)w.rows64 : (const void*)w.rows32;
            if (w.n_bnd)
              MG_CUDA_TRY(cudaMemcpyAsync(c->tail_image[pi] + y.rows[k], r,
                                          (size_t)w.n_bnd * MG_ROW * elem,
                                          cudaMemcpyDeviceToDevice, c->st));
          }
          if (y.ainv_in_smem)
            MG_CUDA_TRY(cudaMemcpyAsync(c->tail_image[pi] + y.Ainv, c->Ainv,
                                        (size_t)m * m * sizeof(double),
                                        cudaMemcpyDeviceToDevice, c->st));
        }
        MG_CUDA_TRY(configure_tail<float>(l32.total));
        MG_CUDA_TRY(configure_tail<double>(l64.total));
      }
    }
  }
  if (c->fused[0]) {
    // boundary-node lists of the levels run by fused steps:
    // between the fine level and the tail, with at most fused_max_tiles
    // active tiles
    const int nlev = (int)c->lev.size();
    const int end = c->tail_level >= 0 ? c->tail_level : nlev - 1;
    const int eta = c->stab.eta;
    for (int l = 1; l < end; ++l) {
      Level& v = c->lev[l];
      if (v.n_active > c->fused_max_tiles) continue;
      TRY(build_region_lists(c, v, nullptr, v.L.ntx * v.L.nty, v.L.ntx, MG_TX, MG_TY,
                             fused_halo(eta), &v.foff, &v.fent));
      v.fused_ok = true;
    }
  }
  {
    // region lists of the fp32 sweep on the levels that run it (the finest,
    // and those above the tail without fused steps)
    const int nlev = (int)c->lev.size();
    const int end = c->tail_level >= 0 ? c->tail_level : nlev - 1;
    for (int l = 0; l < end; ++l) {
      Level& v = c->lev[l];
      if (v.fused_ok || v.n_active == 0) continue;
      TRY(build_region_lists(c, v, v.active, v.n_active, v.L.ntx, MG_TX, MG_TY, 4, &v.soff,
                             &v.sent));
    }
    // which blocks of the kernels after a band kernel may start before it
    // ends (levels whose smoothing runs the separate kernels)
    for (int l = 0; l < end && c->stab.eta > 0; ++l) {
      Level& v = c->lev[l];
      if (v.fused_ok || v.n_active == 0) continue;
      TRY(dalloc(c, &v.sw_touch, (size_t)v.n_active));
      launch_touch_flags(TOUCH_SWEEP, v.L, v.code, v.active, v.L.ntx, v.n_active, v.sw_touch,
                         c->st);
      if (l + 1 < nlev) {
        Level& w = c->lev[l + 1];
        TRY(dalloc(c, &v.pl_touch, (size_t)v.n_active));
        launch_touch_flags(TOUCH_PROLONG, w.L, w.code, v.active, v.L.ntx, v.n_active, v.pl_touch,
                           c->st);
        if (w.n_active > 0) {
          TRY(dalloc(c, &v.rr_touch, 4 * (size_t)w.n_active));
          launch_touch_flags(TOUCH_RESTRICT, v.L, v.code, w.active, w.L.ntx, 4 * w.n_active,
                             v.rr_touch, c->st);
        }
      }
    }
  }
  TRY(sync_check(c));
  return MG_OK;
}

int mg_setup(mg_handle* out, const double* levelset, const mg_grid* grid, const mg_bc* bc,
             const mg_stab* stab, void* cuda_stream) {
  if (!out) return MG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!levelset || !grid) return MG_ERR_INVALID_ARG;
  mg_stab s;
  mg_default_stab(&s);
  if (stab) s = *stab;
  if (bc) {
    if (bc->kind == MG_BC_DIRICHLET && bc->neumann_mask) return MG_ERR_INVALID_ARG;
    if (bc->kind == MG_BC_MIXED && !bc->neumann_mask) return MG_ERR_INVALID_ARG;
    if (bc->kind != MG_BC_DIRICHLET && bc->kind != MG_BC_MIXED) return MG_ERR_INVALID_ARG;
  }
  mg_grid g = *grid;
  if (g.coarsest_cells <= 0) g.coarsest_cells = 8;
  if (!pow2(g.n_cells) || g.n_cells < 8 || g.n_cells > 32768) return MG_ERR_INVALID_ARG;
  if (!pow2(g.coarsest_cells) || g.coarsest_cells < 2 || g.coarsest_cells > 32 ||
      g.coarsest_cells > g.n_cells)
    return MG_ERR_INVALID_ARG;
  if (!(g.h > 0.0) || !std::isfinite(g.h) || !std::isfinite(g.x0) || !std::isfinite(g.y0))
    return MG_ERR_INVALID_ARG;
  if (!(s.gamma > 0.0) || !(s.alpha > 0.0) || s.eta < 0 || s.eta > 8 || s.nu1 < 0 || s.nu1 > 8 ||
      s.nu2 < 0 || s.nu2 > 8 || s.nu1 + s.nu2 == 0 || s.max_cycles < 0 || s.inner < 0 ||
      s.inner > 8 || s.cycle < 0 || s.cycle > 2 || s.fuse_max_tiles < -1 ||
      (s.coarse_op != MG_COARSE_GALERKIN && s.coarse_op != MG_COARSE_REDISCRETISE))
    return MG_ERR_INVALID_ARG;
  if (s.lambda_mode != MG_LAMBDA_LOCAL && s.lambda_mode != MG_LAMBDA_GLOBAL)
    return MG_ERR_INVALID_ARG;
  // c_global = 0: computed at setup (the global eigenvalue problem on the GPU)
  if (s.lambda_mode == MG_LAMBDA_GLOBAL && !(s.c_global >= 0.0 && std::isfinite(s.c_global)))
    return MG_ERR_INVALID_ARG;
  if (s.lambda_mode == MG_LAMBDA_GLOBAL && s.c_global == 0.0 &&
      (g.n_cells > 1024 || (bc && bc->box_sides)))
    return MG_ERR_UNIMPLEMENTED;
  // the global constant belongs to the fine grid; re-discretised coarse
  // levels would each need their own
  if (s.lambda_mode == MG_LAMBDA_GLOBAL && s.coarse_op == MG_COARSE_REDISCRETISE)
    return MG_ERR_UNIMPLEMENTED;
  // the two-grid scheme's "exact" coarse solve needs fp64 cycles
  if (s.cycle == 0 && s.precision != MG_FP64) return MG_ERR_UNIMPLEMENTED;
  // a Neumann mask is given for the fine cells only
  if (s.coarse_op == MG_COARSE_REDISCRETISE && bc && bc->kind == MG_BC_MIXED)
    return MG_ERR_UNIMPLEMENTED;
  if (s.precision != MG_FP64 && s.precision != MG_MIXED) return MG_ERR_INVALID_ARG;
  if (kBoundsChecked && !bounds_word()) return MG_ERR_CUDA;
  mg_ctx* c = new mg_ctx();
  c->st = (cudaStream_t)cuda_stream;
  c->grid = g;
  c->stab = s;
  c->N = g.n_cells;
  c->h = g.h;
  c->nmask_in = (bc && bc->kind == MG_BC_MIXED) ? bc->neumann_mask : nullptr;
  c->box = (bc && bc->box_sides) ? 1 : 0;
  auto t0 = std::chrono::steady_clock::now();
  int rc = setup_impl(c, levelset);
  c->nmask_in = nullptr;
  if (rc != MG_OK) {
    mg_destroy(c);
    return rc;
  }
  c->setup_ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = c;
  return MG_OK;
}

int mg_bounds_check(int* enabled, unsigned* hits, int reset) {
  if (enabled) *enabled = kBoundsChecked ? 1 : 0;
  if (hits) *hits = 0;
  if (!kBoundsChecked) return MG_OK;
  unsigned* w = bounds_word();
  if (!w) return MG_ERR_CUDA;
  MG_CUDA_TRY(cudaDeviceSynchronize());
  unsigned v = 0;
  MG_CUDA_TRY(cudaMemcpy(&v, w, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (hits) *hits = v;
  if (reset) MG_CUDA_TRY(cudaMemset(w, 0, sizeof(unsigned)));
  return MG_OK;
}

int mg_get_c_global(mg_handle c, double* c_global, int* lanczos_steps, int* cg_iterations) {
  if (!c) return MG_ERR_INVALID_ARG;
  if (c_global) *c_global = c->c_global;
  if (lanczos_steps) *lanczos_steps = c->global_steps;
  if (cg_iterations) *cg_iterations = c->global_cg;
  return MG_OK;
}

int mg_set_wait_limit(mg_handle c, long long polls) {
  if (!c || polls > 0xffffffffLL) return MG_ERR_INVALID_ARG;
  c->wait_polls = polls < 0 ? kMbarSpinLimit : (unsigned)polls;
  return MG_OK;
}

int mg_get_counts(mg_handle c, int* n_levels, int* n_dof, int* n_cut, int* n_boundary) {
  if (!c) return MG_ERR_INVALID_ARG;
  if (n_levels) *n_levels = (int)c->lev.size();
  if (n_dof) *n_dof = c->lev[0].n_dof;
  if (n_cut) *n_cut = c->lev[0].n_cut;
  if (n_boundary) *n_boundary = c->lev[0].n_bnd;
  return MG_OK;
}

int mg_level_cells(mg_handle c, int level) {
  if (!c || level < 0 || level >= (int)c->lev.size()) return -1;
  return c->lev[level].n;
}

int mg_level_dofs(mg_handle c, int level) {
  if (!c || level < 0 || level >= (int)c->lev.size()) return -1;
  return c->lev[level].n_dof;
}

static int fill_info(mg_ctx* c, mg_info* info) {
  if (!info) return MG_OK;
  info->n_dof = c->lev[0].n_dof;
  info->n_cut = c->lev[0].n_cut;
  info->n_levels = (int)c->lev.size();
  info->setup_ms = c->setup_ms;
  info->solve_ms = c->solve_ms;
  return MG_OK;
}

int mg_solve(mg_handle c, const double* f, const double* g, double* u, double tol, mg_info* info) {
  return mg_solve_bc(c, f, g, nullptr, u, tol, info);
}

int mg_solve_bc(mg_handle c, const double* f, const double* g, const double* gN, double* u,
                double tol, mg_info* info) {
  if (!c || !f || !g || !u || !(tol >= 0.0)) return MG_ERR_INVALID_ARG;
  if (info) memset(info, 0, sizeof(*info));
  c->last_tol = tol;
  Level& v = c->lev[0];
  MG_CUDA_TRY(cudaEventRecord(c->ev0, c->st));
  Staged sf, sg, su;
  TRY(stage_in(c, 0, f, sf));
  TRY(stage_in(c, 1, g, sg));
  TRY(stage_in(c, 2, u, su));
  Staged sn;
  const bool neu = gN != nullptr && c->Nk != nullptr;
  if (neu) TRY(stage_in(c, 3, gN, sn));
  // u in mapped host memory: its tiles without DOFs are zeroed on a side
  // stream during the solve, so the end writes only the active tiles
  const bool u_mapped = !su.host && !is_device_ptr(u);
  ZeroSide zs{c};
  // d_norms[0..1]: ||F||; the word at d_norms[2]: u has a nonzero DOF value
  unsigned* d_nz = reinterpret_cast<unsigned*>(c->d_norms + 2);
  MG_CUDA_TRY(cudaMemsetAsync(c->d_norms, 0, 3 * sizeof(double), c->st));
  {
    // f, g, g_N are read only where they enter F (the vertices of active
    // cells, of cut cells for g and g_N): a NaN/Inf there makes some F_p
    // non-finite, which k_rhs flags; u only on the DOFs (k_pack flags it)
    // with u in mapped host memory, its read (k_pack) runs beside k_rhs on
    // the side stream: both wait on the host link's latency more than on
    // its bandwidth
    Launch k(c, MG_PROF_IO, 2);
    cudaStream_t sp = c->st;
    if (u_mapped) {
      TRY(ensure_side_stream(c));
      MG_CUDA_TRY(cudaEventRecord(c->ev_z0, c->st));
      MG_CUDA_TRY(cudaStreamWaitEvent(c->st_zero, c->ev_z0, 0));
      sp = c->st_zero;
    }
    RhsArgs ra{v.L, c->h, v.code, v.cls, v.cell_cut, c->Mk, c->Gk, c->Nk,
               neu ? sn.dev : nullptr, v.Ke, c->box, c->d_err};
    launch_rhs(ra, v.active, v.n_active, sf.dev, sg.dev, v.F64, c->d_norms, c->st);
    v.cur64 = 0;
    launch_pack<double>(v.L, v.code, su.dev, v.u64[0], c->d_err, sp, d_nz);
    if (u_mapped) {
      MG_CUDA_TRY(cudaEventRecord(c->ev_z1, c->st_zero));
      MG_CUDA_TRY(cudaStreamWaitEvent(c->st, c->ev_z1, 0));
    }
  }
  MG_CUDA_TRY(cudaMemcpyAsync(c->h_norms, c->d_norms, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                              c->st));
  TRY(sync_check(c));
  if (u_mapped) TRY(zs.start(c->lev[0], const_cast<double*>(su.dev)));
  double Fn = c->h_norms[0];
  unsigned nz = 0;
  memcpy(&nz, c->h_norms + 2, sizeof(unsigned));
  int status = MG_OK;
  if (Fn == 0.0) {
    // F = 0: the solution is u = 0
    MG_CUDA_TRY(cudaMemsetAsync(v.u64[0], 0, v.L.size() * sizeof(double), c->st));
    if (info) info->rel_res = 0.0;
  } else {
    status = solve_loop(c, Fn, tol, c->stab.max_cycles, info, nz == 0);
    if (status == MG_ERR_CUDA) return status;
  }
  double* ud = const_cast<double*>(su.dev);
  {
    Launch k(c, MG_PROF_IO, 1);
    if (u_mapped) {
      launch_unpack_tiles(v.L, v.code, v.active, v.n_active, v.u64[v.cur64], ud, c->st);
      TRY(zs.join());
    } else {
      launch_unpack(v.L, v.code, v.u64[v.cur64], ud, c->st);
    }
  }
  if (su.host) TRY(finish_out(c, u, ud, true));
  MG_CUDA_TRY(cudaEventRecord(c->ev1, c->st));
  TRY(sync_check(c));
  harvest(c);
  MG_CUDA_TRY(cudaEventElapsedTime(&c->solve_ms, c->ev0, c->ev1));
  fill_info(c, info);
  return status;
}

int mg_rhs(mg_handle c, const double* f, const double* g, double* F) {
  return mg_rhs_bc(c, f, g, nullptr, F);
}

int mg_rhs_bc(mg_handle c, const double* f, const double* g, const double* gN, double* F) {
  if (!c || !f || !g || !F) return MG_ERR_INVALID_ARG;
  Level& v = c->lev[0];
  Staged sf, sg, sn;
  TRY(stage_in(c, 0, f, sf));
  TRY(stage_in(c, 1, g, sg));
  const bool neu = gN != nullptr && c->Nk != nullptr;
  if (neu) TRY(stage_in(c, 3, gN, sn));
  double* Fd;
  bool Fh;
  TRY(stage_out(c, 2, F, &Fd, &Fh));
  MG_CUDA_TRY(cudaMemsetAsync(c->d_norms, 0, 2 * sizeof(double), c->st));
  RhsArgs ra{v.L, c->h, v.code, v.cls, v.cell_cut, c->Mk, c->Gk, c->Nk,
             neu ? sn.dev : nullptr, v.Ke, c->box, c->d_err};
  launch_rhs(ra, v.active, v.n_active, sf.dev, sg.dev, v.F64, c->d_norms, c->st);
  launch_unpack(v.L, v.code, v.F64, Fd, c->st);
  TRY(finish_out(c, F, Fd, Fh));
  return sync_check(c);
}

int mg_cycles(mg_handle c, const double* F, double* u, int k, int precision) {
  if (!c || !F || !u || k < 0) return MG_ERR_INVALID_ARG;
  if (precision != MG_FP64 && precision != MG_MIXED) return MG_ERR_INVALID_ARG;
  Level& v = c->lev[0];
  Staged sF, su;
  TRY(stage_in(c, 0, F, sF));
  TRY(stage_in(c, 2, u, su));
  launch_pack<double>(v.L, v.code, sF.dev, v.F64, c->d_err, c->st);
  v.cur64 = 0;
  launch_pack<double>(v.L, v.code, su.dev, v.u64[0], c->d_err, c->st);
  for (int s = 0; s < k; ++s) {
    if (precision == MG_FP64) {
      vcycle<double>(c, 0, false);
    } else {
      double rmax;
      // scale by the residual's magnitude (exact power of two)
      TRY(fine_residual(c, 1.0, false, &rmax));
      double sigma = pow2_near_inverse(rmax);
      OpArgs<double> op = op_of<double>(v);
      launch_residual<double, float>(op, v.active, v.n_active, v.u64[v.cur64], v.F64, v.F32, sigma,
                                     (double*)nullptr, c->st);
      refinement_step(c, sigma, c->stab.inner > 0 ? c->stab.inner : 1);
    }
  }
  double* ud = const_cast<double*>(su.dev);
  launch_unpack(v.L, v.code, v.u64[v.cur64], ud, c->st);
  if (su.host) TRY(finish_out(c, u, ud, true));
  return sync_check(c);
}

int mg_cycles_transposed(mg_handle c, const double* F, double* u, int k) {
  if (!c || !F || !u || k < 0) return MG_ERR_INVALID_ARG;
  Level& v = c->lev[0];
  Staged sF, su;
  TRY(stage_in(c, 0, F, sF));
  TRY(stage_in(c, 2, u, su));
  launch_pack<double>(v.L, v.code, sF.dev, v.F64, c->d_err, c->st);
  v.cur64 = 0;
  launch_pack<double>(v.L, v.code, su.dev, v.u64[0], c->d_err, c->st);
  for (int s = 0; s < k; ++s) vcycle_transposed(c, 0, false);
  double* ud = const_cast<double*>(su.dev);
  launch_unpack(v.L, v.code, v.u64[v.cur64], ud, c->st);
  if (su.host) TRY(finish_out(c, u, ud, true));
  return sync_check(c);
}

int mg_residual(mg_handle c, const double* F, const double* u, double* r, double* norms) {
  if (!c || !F || !u) return MG_ERR_INVALID_ARG;
  Level& v = c->lev[0];
  Staged sF, su;
  TRY(stage_in(c, 0, F, sF));
  TRY(stage_in(c, 1, u, su));
  launch_pack<double>(v.L, v.code, sF.dev, v.F64, c->d_err, c->st);
  v.cur64 = 0;
  launch_pack<double>(v.L, v.code, su.dev, v.u64[0], c->d_err, c->st);
  MG_CUDA_TRY(cudaMemsetAsync(c->d_norms, 0, 2 * sizeof(double), c->st));
  if (!c->d_part) TRY(dalloc(c, &c->d_part, (size_t)std::max(1, v.n_active)));
  OpArgs<double> op = op_of<double>(v);
  launch_residual<double, double>(op, v.active, v.n_active, v.u64[0], v.F64, v.u64[1], 1.0,
                                  c->d_norms, c->st, true, c->d_part);
  if (r) {
    double* rd;
    bool rh;
    TRY(stage_out(c, 2, r, &rd, &rh));
    launch_unpack(v.L, v.code, v.u64[1], rd, c->st);
    TRY(finish_out(c, r, rd, rh));
  }
  MG_CUDA_TRY(cudaMemcpyAsync(c->h_norms, c->d_norms, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                              c->st));
  TRY(sync_check(c));
  if (norms) {
    norms[0] = c->h_norms[0];
    norms[1] = std::sqrt(c->h_norms[1]);
  }
  return MG_OK;
}

int mg_export_stencil(mg_handle c, int level, double* out) {
  if (!c || !out || level < 0 || level >= (int)c->lev.size()) return MG_ERR_INVALID_ARG;
  Level& v = c->lev[level];
  size_t m = (size_t)(v.n + 1) * (v.n + 1) * 9;
  double* d = out;
  bool host = !is_device_ptr(out);
  if (host) MG_CUDA_TRY(cudaMalloc((void**)&d, m * sizeof(double)));
  launch_export_stencil<double>(op_of<double>(v), d, c->st);
  int rc = MG_OK;
  if (host) {
    cudaError_t e = cudaMemcpyAsync(out, d, m * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    cudaFree(d);
    if (e != cudaSuccess) rc = mg_cuda_fail(e);
  }
  if (rc != MG_OK) return rc;
  return sync_check(c);
}

int mg_export_cut_cells(mg_handle c, int max_cells, int* cells, double* data, int* n_total) {
  if (!c || max_cells < 0) return MG_ERR_INVALID_ARG;
  Level& v = c->lev[0];
  if (n_total) *n_total = v.n_cut;
  int m = max_cells < v.n_cut ? max_cells : v.n_cut;
  if (m == 0) return MG_OK;
  std::vector<int> hc(m);
  std::vector<double> cl((size_t)m * 4), ke((size_t)m * 16), mk((size_t)m * 16), gk((size_t)m * 16);
  MG_CUDA_TRY(cudaStreamSynchronize(c->st));
  MG_CUDA_TRY(cudaMemcpy(hc.data(), v.cut_list, m * sizeof(int), cudaMemcpyDeviceToHost));
  MG_CUDA_TRY(cudaMemcpy(cl.data(), c->Cl, cl.size() * sizeof(double), cudaMemcpyDeviceToHost));
  MG_CUDA_TRY(cudaMemcpy(ke.data(), v.Ke, ke.size() * sizeof(double), cudaMemcpyDeviceToHost));
  MG_CUDA_TRY(cudaMemcpy(mk.data(), c->Mk, mk.size() * sizeof(double), cudaMemcpyDeviceToHost));
  MG_CUDA_TRY(cudaMemcpy(gk.data(), c->Gk, gk.size() * sizeof(double), cudaMemcpyDeviceToHost));
  std::vector<double> d((size_t)m * 52);
  for (int t = 0; t < m; ++t) {
    double* o = d.data() + (size_t)t * 52;
    for (int q = 0; q < 4; ++q) o[q] = cl[(size_t)t * 4 + q];
    for (int q = 0; q < 16; ++q) {
      o[4 + q] = ke[(size_t)t * 16 + q];
      o[20 + q] = mk[(size_t)t * 16 + q];
      o[36 + q] = gk[(size_t)t * 16 + q];
    }
  }
  if (cells) {
    if (is_device_ptr(cells))
      MG_CUDA_TRY(cudaMemcpy(cells, hc.data(), m * sizeof(int), cudaMemcpyHostToDevice));
    else
      memcpy(cells, hc.data(), m * sizeof(int));
  }
  if (data) {
    if (is_device_ptr(data))
      MG_CUDA_TRY(cudaMemcpy(data, d.data(), d.size() * sizeof(double), cudaMemcpyHostToDevice));
    else
      memcpy(data, d.data(), d.size() * sizeof(double));
  }
  return MG_OK;
}

}  // extern "C"

int mg_internal_fine_view(mg_handle c, FineOpView* out) {
  if (!c || !out || c->lev.empty()) return MG_ERR_INVALID_ARG;
  Level& v = c->lev[0];
  out->L = v.L;
  out->code = v.code;
  out->tile_base = v.tile_base;
  out->rows64 = v.rows64;
  out->n_rows = v.n_bnd;
  out->active = v.active;
  out->n_active = v.n_active;
  out->N = c->N;
  out->device = c->device;
  out->st = c->st;
  return MG_OK;
}

extern "C" {

int mg_set_profiling(mg_handle c, int enable) {
  if (!c) return MG_ERR_INVALID_ARG;
  MG_CUDA_TRY(cudaStreamSynchronize(c->st));
  harvest(c);
  if (enable) {
    for (int k = 0; k < MG_PROF_SLOTS; ++k) { c->kcount[k] = 0; c->kms[k] = 0.0; }
    c->launches = 0;
  }
  c->prof = enable != 0;
  return MG_OK;
}

int mg_get_profile(mg_handle c, long long* launches, long long* counts, double* ms) {
  if (!c) return MG_ERR_INVALID_ARG;
  MG_CUDA_TRY(cudaStreamSynchronize(c->st));
  harvest(c);
  if (launches) *launches = c->launches;
  for (int k = 0; k < MG_PROF_SLOTS; ++k) {
    if (counts) counts[k] = c->kcount[k];
    if (ms) ms[k] = c->kms[k];
  }
  return MG_OK;
}

// A is symmetric (Sec. 4.1): w solves A w = dL/du with the handle's own
// cycle and precision, to the tolerance of the last solve; F = M f + G g is
// linear in f and g (Eq. disc_rhs), so dL/df = M^T w and dL/dg = G^T w.
int mg_adjoint(mg_handle c, const double* dLdu, double* dLdf, double* dLdg) {
  return mg_adjoint_bc(c, dLdu, dLdf, dLdg, nullptr);
}

int mg_adjoint_bc(mg_handle c, const double* dLdu, double* dLdf, double* dLdg, double* dLdgN) {
  if (!c || !dLdu || (!dLdf && !dLdg && !dLdgN)) return MG_ERR_INVALID_ARG;
  Level& v = c->lev[0];
  const double tol = c->last_tol > 0.0 ? c->last_tol : 1e-10;
  Staged sd;
  TRY(stage_in(c, 0, dLdu, sd));
  double *fd = nullptr, *gd = nullptr;
  bool fh = false, gh = false;
  if (dLdf) TRY(stage_out(c, 1, dLdf, &fd, &fh));
  if (dLdg) TRY(stage_out(c, 2, dLdg, &gd, &gh));
  double* nd = nullptr;
  bool nh = false;
  if (dLdgN) {
    TRY(stage_out(c, 3, dLdgN, &nd, &nh));
    if (!c->adj_tmp) TRY(dalloc(c, &c->adj_tmp, v.L.size()));
  }
  // right-hand side dL/du on the DOFs (NaN / Inf rejected), w from 0
  launch_pack<double>(v.L, v.code, sd.dev, v.F64, c->d_err, c->st);
  v.cur64 = 0;
  MG_CUDA_TRY(cudaMemsetAsync(v.u64[0], 0, v.L.size() * sizeof(double), c->st));
  TRY(sync_check(c));
  double Fn = 0.0;
  TRY(fine_residual(c, 1.0, false, &Fn));     // ||dL/du||_inf on the DOFs (w = 0)
  int status = MG_OK;
  if (Fn > 0.0) {
    // w by transposed fp64 V-cycles (whatever the handle's precision)
    status = solve_loop(c, Fn, tol, c->stab.max_cycles, nullptr, true, true);
    if (status == MG_ERR_CUDA) return status;
  }
  const double* w = v.u64[v.cur64];
  double* tf = v.F64;                          // dL/du is no longer needed
  double* tg = v.u64[v.cur64 ^ 1];
  RhsArgs ra{v.L, c->h, v.code, v.cls, v.cell_cut, c->Mk, c->Gk, c->Nk, nullptr, v.Ke, c->box};
  const int* atiles = v.active;
  int n_atiles = v.n_active;
  if (c->box) {
    // box nodes can sit in tiles without DOFs (the last tile row or column):
    // visit every tile
    const int nt = v.L.ntx * v.L.nty;
    if (!c->all_tiles) {
      std::vector<int> all(nt);
      for (int t = 0; t < nt; ++t) all[t] = t;
      TRY(dalloc(c, &c->all_tiles, (size_t)nt));
      MG_CUDA_TRY(cudaMemcpyAsync(c->all_tiles, all.data(), (size_t)nt * sizeof(int),
                                  cudaMemcpyHostToDevice, c->st));
      MG_CUDA_TRY(cudaStreamSynchronize(c->st));
    }
    atiles = c->all_tiles;
    n_atiles = nt;
    // the outputs are read on every tile
    if (dLdf) MG_CUDA_TRY(cudaMemsetAsync(tf, 0, v.L.size() * sizeof(double), c->st));
    if (dLdg) MG_CUDA_TRY(cudaMemsetAsync(tg, 0, v.L.size() * sizeof(double), c->st));
  }
  double* tn = c->adj_tmp;
  if (dLdgN) MG_CUDA_TRY(cudaMemsetAsync(tn, 0, v.L.size() * sizeof(double), c->st));
  launch_rhs_adj(ra, atiles, n_atiles, w, dLdf ? tf : nullptr, dLdg ? tg : nullptr, c->st,
                 dLdgN ? tn : nullptr);
  if (dLdgN) {
    launch_unpack(v.L, v.code, tn, nd, c->st);
    TRY(finish_out(c, dLdgN, nd, nh));
  }
  if (dLdf) {
    launch_unpack(v.L, v.code, tf, fd, c->st, c->box);
    TRY(finish_out(c, dLdf, fd, fh));
  }
  if (dLdg) {
    launch_unpack(v.L, v.code, tg, gd, c->st, c->box);
    TRY(finish_out(c, dLdg, gd, gh));
  }
  TRY(sync_check(c));
  return status;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched solves (batch.cu): per-member hierarchies built by the setup above,
// a table of their device arrays, and one CUDA graph per launch shape.

#include "batch.cuh"

struct mg_batch_ctx {
  cudaStream_t user_st = nullptr;   // the caller's stream (ordering only)
  cudaStream_t st = nullptr;        // the batch's own stream (captured, launched)
  int count = 0;
  mg_stab stab{};
  std::vector<mg_ctx*> mem;
  std::vector<void*> allocs;
  std::vector<size_t> node_off;     // count + 1
  size_t total_nodes = 0;
  int total_tiles = 0;
  BatchProblem* d_probs = nullptr;
  int* d_order = nullptr;
  size_t* d_node_off = nullptr;
  int* d_tile_off = nullptr;
  unsigned* d_words = nullptr;      // [0], [2] work counters, [1] error word, [3..] bad flags
  double* d_params = nullptr;       // tol, max_cycles, fixed group (0: adaptive)
  double* h_params = nullptr;       // pinned
  BatchResult* d_res = nullptr;
  BatchResult* h_res = nullptr;     // pinned (the graph copies into it)
  unsigned* h_err = nullptr;        // pinned
  double *f = nullptr, *g = nullptr, *u = nullptr;
  double* gN = nullptr;             // packed Neumann data (members with Neumann cells)
  // the member table on the host, and the packed arrays it points at now
  // (the batch's own buffers, or the caller's device or mapped host arrays)
  std::vector<BatchProblem> h_probs;
  const double *io_f = nullptr, *io_g = nullptr, *io_gN = nullptr;
  double* io_u = nullptr;
  bool mixed = false;
  size_t smem = 0;
  int grid = 0;
  int n_coop = 0;
  BatchTune tune{1024, 4, 2, 8192};
  std::vector<int> n_dof, n_top;    // per member
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev_in = nullptr, ev0 = nullptr, ev1 = nullptr;
  float setup_ms = 0.f, solve_ms = 0.f;
};

namespace {

template <class T>
int balloc(mg_batch_ctx* b, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return MG_ERR_OUT_OF_MEMORY;
  }
  if (e != cudaSuccess) return mg_cuda_fail(e);
  b->allocs.push_back(*p);
  e = cudaMemsetAsync(*p, 0, count * sizeof(T), b->st);
  return e == cudaSuccess ? MG_OK : mg_cuda_fail(e);
}

// The eta window of one level: the boundary nodes (blist, host copy) and
// their 8 neighbours, sorted by padded offset; per entry the window index of
// each stencil position.  Returns false (no window) if it would not fit in
// `avail` bytes of shared memory or in 16-bit indices.
bool build_window(const std::vector<int2>& bl, int P, size_t avail, std::vector<int>& win,
                  std::vector<uint16_t>& slot) {
  const int d[9] = {-P - 1, -P, -P + 1, -1, 0, 1, P - 1, P, P + 1};
  win.clear();
  win.reserve(bl.size() * 9);
  for (const int2& e : bl)
    for (int k = 0; k < 9; ++k) win.push_back(e.x + d[k]);
  std::sort(win.begin(), win.end());
  win.erase(std::unique(win.begin(), win.end()), win.end());
  if (win.empty() || win.size() > 65535 || win.size() * sizeof(float) > avail) return false;
  slot.assign(bl.size() * 10, 0);
  for (size_t e = 0; e < bl.size(); ++e)
    for (int k = 0; k < 9; ++k)
      slot[e * 10 + k] = (uint16_t)(std::lower_bound(win.begin(), win.end(), bl[e].x + d[k]) -
                                    win.begin());
  return true;
}

// The static image of the resident eta phases of one level for block `rank`
// of nr (batch.cu, eta_resident): rows (srows: n entries by coefficient),
// positions (blist) and the window indices of the three stencil rows (slot:
// 10 per entry) of the entries j = k nr + rank of each colour group (boff),
// laid out as eta_resident_layout places them from `rows` to `f`.
std::vector<unsigned char> eta_image(int win_n, const int* boff, int nr, int rank,
                                     const std::vector<float>& srows, int n,
                                     const std::vector<int2>& blist,
                                     const std::vector<uint16_t>& slot) {
  int lb[5], le = 0;
  lb[0] = 0;
  for (int c = 0; c < 4; ++c) {
    const int cnt = boff[c + 1] - boff[c];
    le += (cnt + nr - 1) / nr;
    lb[c + 1] = lb[c] + (cnt - rank + nr - 1) / nr;
  }
  const EtaResidentLayout lay = eta_resident_layout(win_n, le);
  std::vector<unsigned char> img(lay.f - lay.rows, 0);
  float* R = reinterpret_cast<float*>(img.data());
  int* P = reinterpret_cast<int*>(img.data() + (lay.pos - lay.rows));
  uint16_t* S = reinterpret_cast<uint16_t*>(img.data() + (lay.slot - lay.rows));
  // each colour group in the order of the padded offsets, so that a warp's
  // vertices lie close together in the window (the order of the updates in a
  // colour phase is free: vertices of one colour are not stencil neighbours)
  std::vector<int> ord((size_t)boff[4]);
  for (int e = 0; e < boff[4]; ++e) ord[e] = e;
  for (int c = 0; c < 4; ++c)
    std::sort(ord.begin() + boff[c], ord.begin() + boff[c + 1],
              [&](int x, int y) { return blist[x].x < blist[y].x; });
  for (int c = 0; c < 4; ++c)
    for (int k = 0; k < lb[c + 1] - lb[c]; ++k) {
      const int x = lb[c] + k, e = ord[boff[c] + k * nr + rank];
      for (int r = 0; r < MG_ROW; ++r) R[(size_t)r * le + x] = srows[(size_t)r * n + e];
      P[x] = blist[e].x;
      for (int q = 0; q < 3; ++q) S[(size_t)q * le + x] = slot[(size_t)e * 10 + 3 * q];
    }
  return img;
}

// the device table entry of one member (its hierarchy is set up, mixed);
// win_bytes: shared memory the member's eta windows may use; res_cap: the
// shared memory of the resident eta phases
int batch_member(mg_batch_ctx* b, int p, BatchProblem* out, size_t win_bytes, size_t res_cap) {
  mg_ctx* c = b->mem[p];
  const int t = c->tail_level;
  if (t < 0 || t > MG_BATCH_MAX_TOP) return MG_ERR_UNIMPLEMENTED;
  BatchProblem& q = *out;
  memset(&q, 0, sizeof(q));
  q.n_top = t;
  // first nodes of the active tiles of every level the batch kernel walks
  unsigned* xy[MG_BATCH_MAX_TOP + 1];
  for (int l = 0; l <= t; ++l) {
    Level& v = c->lev[l];
    TRY(dalloc(c, &xy[l], (size_t)v.n_active));
    launch_tile_xy(v.L, v.active, v.n_active, xy[l], c->st);
  }
  for (int l = 0; l < t; ++l) {
    Level& v = c->lev[l];
    BatchLevel& w = q.lev[l];
    int2* blist;
    int* boff;
    TRY(dalloc(c, &blist, (size_t)v.n_bnd));
    TRY(dalloc(c, &boff, 5));
    launch_batch_lists(v.L, v.code, v.tile_base, blist, boff, c->st);
    MG_CUDA_TRY(cudaMemcpyAsync(w.boff, boff, 5 * sizeof(int), cudaMemcpyDeviceToHost, c->st));
    std::vector<int2> hb((size_t)v.n_bnd);
    if (v.n_bnd)
      MG_CUDA_TRY(cudaMemcpyAsync(hb.data(), blist, (size_t)v.n_bnd * sizeof(int2),
                                  cudaMemcpyDeviceToHost, c->st));
    MG_CUDA_TRY(cudaStreamSynchronize(c->st));
    float* srows;
    TRY(dalloc(c, &srows, (size_t)v.n_bnd * MG_ROW));
    launch_soa_rows(blist, v.n_bnd, v.rows32, srows, c->st);
    w.srows = srows;
    std::vector<int> hw;
    std::vector<uint16_t> hs;
    w.win = nullptr;
    w.wslot = nullptr;
    w.win_n = 0;
    if (v.n_bnd && build_window(hb, v.L.pitch, win_bytes, hw, hs)) {
      int* dw;
      uint16_t* ds;
      TRY(dalloc(c, &dw, hw.size()));
      TRY(dalloc(c, &ds, hs.size()));
      MG_CUDA_TRY(cudaMemcpyAsync(dw, hw.data(), hw.size() * sizeof(int), cudaMemcpyHostToDevice,
                                  c->st));
      MG_CUDA_TRY(cudaMemcpyAsync(ds, hs.data(), hs.size() * sizeof(uint16_t),
                                  cudaMemcpyHostToDevice, c->st));
      MG_CUDA_TRY(cudaStreamSynchronize(c->st));
      w.win = dw;
      w.wslot = ds;
      w.win_n = (int)hw.size();
    }
    w.rimg[0] = w.rimg[1] = w.rimg[2] = nullptr;
    if (w.win_n > 0) {
      const bool one = eta_resident_bytes(w.win_n, w.boff, 1) <= res_cap;
      if (one || eta_resident_bytes(w.win_n, w.boff, 2) <= res_cap) {
        std::vector<float> hr((size_t)v.n_bnd * MG_ROW);
        MG_CUDA_TRY(cudaMemcpyAsync(hr.data(), srows, hr.size() * sizeof(float),
                                    cudaMemcpyDeviceToHost, c->st));
        MG_CUDA_TRY(cudaStreamSynchronize(c->st));
        for (int k = one ? 0 : 1; k < (one ? 1 : 3); ++k) {
          const std::vector<unsigned char> img =
              eta_image(w.win_n, w.boff, one ? 1 : 2, one ? 0 : k - 1, hr, v.n_bnd, hb, hs);
          unsigned char* d;
          TRY(dalloc(c, &d, img.size()));
          MG_CUDA_TRY(cudaMemcpyAsync(d, img.data(), img.size(), cudaMemcpyHostToDevice, c->st));
          MG_CUDA_TRY(cudaStreamSynchronize(c->st));
          w.rimg[k] = d;
        }
      }
    }
    w.L = v.L;
    w.code = v.code;
    w.tile_base = v.tile_base;
    w.rows = v.rows32;
    w.xy = xy[l];
    w.n_active = v.n_active;
    w.blist = blist;
    w.u = v.u32[0];
    w.F = v.F32;
    w.scr = v.u32[1];           // zero from allocation; the batch writes it on active tiles only
  }
  Level& top = c->lev[t];
  TailArgs<float>& a = q.tail;
  a.lay = c->tail_lay[0];
  for (int k = 0; k < a.lay.nlev; ++k) a.rows[k] = c->lev[t + k].rows32;
  a.L0 = top.L;
  a.image = c->tail_image[0];
  a.Ainv = c->Ainv;
  a.F0 = top.F32;
  a.u0 = top.u32[0];
  a.load_u0 = 0;
  a.eta = c->stab.eta;
  a.nu1 = c->stab.nu1;
  a.nu2 = c->stab.nu2;
  a.err = b->d_words + 1;
  a.wait_polls = kMbarSpinLimit;
  q.tail_xy = xy[t];
  q.tail_n_active = top.n_active;
  q.tail_F = top.F32;
  Level& v = c->lev[0];
  q.L0 = v.L;
  q.code0 = v.code;
  q.tile_base0 = v.tile_base;
  q.rows64 = v.rows64;
  q.active0 = v.active;
  q.xy0 = xy[0];
  q.n_active0 = v.n_active;
  q.F64 = v.F64;
  q.u64 = v.u64[0];
  q.F32 = v.F32;
  q.e32 = v.u32[0];
  q.eta = c->stab.eta;
  q.nu1 = c->stab.nu1;
  q.nu2 = c->stab.nu2;
  // a NaN/Inf in f, g or g_N where it enters F marks the member bad
  q.rhs = RhsArgs{v.L, c->h, v.code, v.cls, v.cell_cut, c->Mk, c->Gk, c->Nk,
                 (b->gN && c->Nk) ? b->gN + b->node_off[p] : nullptr, v.Ke, c->box,
                 b->d_words + 3 + p};
  q.f = b->f + b->node_off[p];
  q.g = b->g + b->node_off[p];
  q.u_out = b->u + b->node_off[p];
  return MG_OK;
}

// (re)captures the solve graph for the current launch shape: the work order
// (members a cluster shares first, each part largest first) and the grid
int batch_capture(mg_batch_ctx* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  const int n = b->count;
  const BatchTune& tu = b->tune;
  auto coop = [&](int p) {
    return tu.cluster > 1 && b->n_top[p] > 0 && b->n_dof[p] >= tu.coop_min_dof;
  };
  std::vector<int> order(n);
  for (int p = 0; p < n; ++p) order[p] = p;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    if (coop(x) != coop(y)) return coop(x);
    return b->n_dof[x] > b->n_dof[y];
  });
  b->n_coop = 0;
  while (b->n_coop < n && coop(order[b->n_coop])) ++b->n_coop;
  MG_CUDA_TRY(cudaMemcpyAsync(b->d_order, order.data(), (size_t)n * sizeof(int),
                              cudaMemcpyHostToDevice, b->st));
  MG_CUDA_TRY(cudaStreamSynchronize(b->st));
  const int nc = batch_max_clusters(tu, b->smem);
  if (nc <= 0) return MG_ERR_INVALID_ARG;          // the shape does not fit on the device
  b->grid = nc * tu.cluster;
  MG_CUDA_TRY(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
  cudaMemsetAsync(b->d_words, 0, (3 + (size_t)n) * sizeof(unsigned), b->st);
  launch_batch_rhs(b->d_probs, b->d_tile_off, n, b->total_tiles, b->st);
  launch_batch(b->d_probs, b->d_order, n, b->n_coop, b->d_words, b->d_words + 3, b->d_params,
               tu, b->grid, b->smem, b->d_res, b->st);
  launch_batch_unpack(b->d_probs, b->d_node_off, b->count, b->total_nodes, b->st);
  cudaMemcpyAsync(b->h_res, b->d_res, (size_t)b->count * sizeof(BatchResult),
                  cudaMemcpyDeviceToHost, b->st);
  cudaMemcpyAsync(b->h_err, b->d_words + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, b->st);
  cudaError_t e = cudaStreamEndCapture(b->st, &b->graph);
  if (e != cudaSuccess) return mg_cuda_fail(e);
  MG_CUDA_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
  return MG_OK;
}

int status_rank(int s) {
  switch (s) {
    case MG_OK: return 0;
    case MG_ERR_NOT_CONVERGED: return 1;
    case MG_ERR_DIVERGED: return 2;
    default: return 3;
  }
}

// one solve of the inputs the member table points at; results where it
// points (u_out) and in b->h_res
int batch_run(mg_batch_ctx* b, double tol, int* worst) {
  b->h_params[0] = tol;
  b->h_params[1] = (double)b->stab.max_cycles;
  b->h_params[2] = (double)b->stab.inner;
  MG_CUDA_TRY(cudaMemcpyAsync(b->d_params, b->h_params, 3 * sizeof(double),
                              cudaMemcpyHostToDevice, b->st));
  MG_CUDA_TRY(cudaEventRecord(b->ev0, b->st));
  MG_CUDA_TRY(cudaGraphLaunch(b->exec, b->st));
  MG_CUDA_TRY(cudaEventRecord(b->ev1, b->st));
  MG_CUDA_TRY(cudaStreamSynchronize(b->st));
  MG_CUDA_TRY(cudaGetLastError());
  MG_CUDA_TRY(cudaEventElapsedTime(&b->solve_ms, b->ev0, b->ev1));
  if (*b->h_err) {
    const unsigned err = *b->h_err;
    if (err & DEV_ERR_TIMEOUT) return MG_ERR_TIMEOUT;
    return MG_ERR_INTERNAL;
  }
  int w = MG_OK;
  for (int p = 0; p < b->count; ++p)
    if (status_rank(b->h_res[p].status) > status_rank(w)) w = b->h_res[p].status;
  *worst = w;
  return MG_OK;
}

// The packed arrays of one solve.  Device arrays and mapped host arrays are
// used in place (the kernels read f, g, g_N only where they enter F and
// write u); pageable host arrays are copied through the batch's buffers.
// gN_given: a g_N argument exists (NULL meaning g_N = 0).  Re-points the
// member table when the arrays differ from the last solve's.
int batch_io(mg_batch_ctx* b, const double* f, const double* g, bool gN_given,
             const double* gN, double* u, double** u_used) {
  MG_CUDA_TRY(cudaEventRecord(b->ev_in, b->user_st));
  MG_CUDA_TRY(cudaStreamWaitEvent(b->st, b->ev_in, 0));
  const size_t bytes = b->total_nodes * sizeof(double);
  auto direct = [](const double* p) -> const double* {
    return is_device_ptr(p) ? p : mapped_host(p);
  };
  auto input = [&](const double* p, double* own, const double** out) -> int {
    const double* d = direct(p);
    if (!d) {
      MG_CUDA_TRY(cudaMemcpyAsync(own, p, bytes, cudaMemcpyHostToDevice, b->st));
      d = own;
    }
    *out = d;
    return MG_OK;
  };
  const double *F, *G, *GN = b->gN;
  TRY(input(f, b->f, &F));
  TRY(input(g, b->g, &G));
  if (b->gN && gN_given) {
    if (gN == nullptr) MG_CUDA_TRY(cudaMemsetAsync(b->gN, 0, bytes, b->st));
    else TRY(input(gN, b->gN, &GN));
  }
  double* U = const_cast<double*>(direct(u));
  if (!U) U = b->u;
  *u_used = U;
  if (F != b->io_f || G != b->io_g || GN != b->io_gN || U != b->io_u) {
    for (int p = 0; p < b->count; ++p) {
      BatchProblem& q = b->h_probs[p];
      const size_t o = b->node_off[p];
      q.f = F + o;
      q.g = G + o;
      if (q.rhs.Nk) q.rhs.gN = GN ? GN + o : nullptr;
      q.u_out = U + o;
    }
    MG_CUDA_TRY(cudaMemcpyAsync(b->d_probs, b->h_probs.data(),
                                (size_t)b->count * sizeof(BatchProblem), cudaMemcpyHostToDevice,
                                b->st));
    b->io_f = F;
    b->io_g = G;
    b->io_gN = GN;
    b->io_u = U;
  }
  return MG_OK;
}

// mean device time per solve of `reps` replays after one warm-up; false if
// the shape does not fit or a member did not converge
int time_shape(mg_batch_ctx* b, const BatchTune& t, double tol, int reps, float* ms, bool* ok) {
  *ok = false;
  b->tune = t;
  const int rc = batch_capture(b);
  if (rc == MG_ERR_INVALID_ARG) return MG_OK;
  TRY(rc);
  int worst = MG_OK;
  TRY(batch_run(b, tol, &worst));
  if (worst != MG_OK) return MG_OK;
  float total = 0.f;
  for (int r = 0; r < reps; ++r) {
    TRY(batch_run(b, tol, &worst));
    if (worst != MG_OK) return MG_OK;
    total += b->solve_ms;
  }
  *ms = total / reps;
  *ok = true;
  return MG_OK;
}

int batch_setup_impl(mg_batch_ctx* b, const mg_grid* grids, const double* levelsets,
                     const mg_bc* bc) {
  const int n = b->count;
  MG_CUDA_TRY(cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking));
  MG_CUDA_TRY(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
  MG_CUDA_TRY(cudaEventCreate(&b->ev0));
  MG_CUDA_TRY(cudaEventCreate(&b->ev1));
  MG_CUDA_TRY(cudaEventRecord(b->ev_in, b->user_st));
  MG_CUDA_TRY(cudaStreamWaitEvent(b->st, b->ev_in, 0));
  b->node_off.assign(n + 1, 0);
  for (int p = 0; p < n; ++p) {
    const size_t m = (size_t)grids[p].n_cells + 1;
    if (grids[p].n_cells <= 0 || grids[p].n_cells > 32768) return MG_ERR_INVALID_ARG;
    b->node_off[p + 1] = b->node_off[p] + m * m;
  }
  b->total_nodes = b->node_off[n];
  TRY(balloc(b, &b->f, b->total_nodes));
  TRY(balloc(b, &b->g, b->total_nodes));
  TRY(balloc(b, &b->u, b->total_nodes));
  TRY(balloc(b, &b->d_words, 3 + (size_t)n));
  TRY(balloc(b, &b->d_params, 4));
  TRY(balloc(b, &b->d_res, (size_t)n));
  TRY(balloc(b, &b->d_order, (size_t)n));
  TRY(balloc(b, &b->d_node_off, (size_t)n + 1));
  TRY(balloc(b, &b->d_tile_off, (size_t)n + 1));
  TRY(balloc(b, &b->d_probs, (size_t)n));
  MG_CUDA_TRY(cudaMallocHost((void**)&b->h_params, 4 * sizeof(double)));
  MG_CUDA_TRY(cudaMallocHost((void**)&b->h_res, (size_t)n * sizeof(BatchResult)));
  MG_CUDA_TRY(cudaMallocHost((void**)&b->h_err, sizeof(unsigned)));
  *b->h_err = 0;
  b->mixed = bc && bc->kind == MG_BC_MIXED;
  if (b->mixed) TRY(balloc(b, &b->gN, b->total_nodes));
  size_t cell_off = 0;
  for (int p = 0; p < n; ++p) {
    mg_handle h = nullptr;
    const double* ls = levelsets + b->node_off[p];
    mg_bc mb{MG_BC_DIRICHLET, nullptr, 0};
    if (bc) {
      mb = *bc;
      // a batch's Neumann mask holds the members' masks one after another
      if (b->mixed) mb.neumann_mask = bc->neumann_mask + cell_off;
    }
    cell_off += (size_t)grids[p].n_cells * grids[p].n_cells;
    TRY(mg_setup(&h, ls, &grids[p], bc ? &mb : nullptr, &b->stab, b->st));
    b->mem.push_back(h);
  }
  std::vector<BatchProblem> probs(n);
  std::vector<int> tile_off(n + 1, 0);
  size_t smem = 0;
  for (int p = 0; p < n; ++p) smem = std::max(smem, (size_t)b->mem[p]->tail_lay[0].total);
  // The resident eta phases take what the block's shared memory allows
  // without a larger carve-out (which would shrink the L1 cache the level
  // sweeps read through): 192 KB, or the tail's own need if larger.
  {
    int dev = 0, optin = 0;
    MG_CUDA_TRY(cudaGetDevice(&dev));
    MG_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t target = 192 * 1024;                 // usable bytes, the slack apart
    const size_t limit = (size_t)optin > 4096 + kSmemSlack ? (size_t)optin - 4096 - kSmemSlack : 0;
    smem = std::max(smem, std::min(target, limit));
  }
  for (int p = 0; p < n; ++p) {
    // the eta windows live in the tail's dynamic region, up to the end of
    // the batch's shared memory
    const size_t start = b->mem[p]->tail_lay[0].U[0];
    TRY(batch_member(b, p, &probs[p], smem - kSmemSlack > start ? smem - kSmemSlack - start : 0,
                     smem - kSmemSlack));
    probs[p].res_cap = (int)(smem - kSmemSlack);
    tile_off[p + 1] = tile_off[p] + probs[p].n_active0;
  }
  b->total_tiles = tile_off[n];
  b->n_dof.resize(n);
  b->n_top.resize(n);
  for (int p = 0; p < n; ++p) {
    b->n_dof[p] = b->mem[p]->lev[0].n_dof;
    b->n_top[p] = probs[p].n_top;
  }
  MG_CUDA_TRY(cudaMemcpyAsync(b->d_probs, probs.data(), (size_t)n * sizeof(BatchProblem),
                              cudaMemcpyHostToDevice, b->st));
  b->h_probs = probs;
  b->io_f = b->f;
  b->io_g = b->g;
  b->io_gN = b->gN;
  b->io_u = b->u;
  MG_CUDA_TRY(cudaMemcpyAsync(b->d_node_off, b->node_off.data(), (size_t)(n + 1) * sizeof(size_t),
                              cudaMemcpyHostToDevice, b->st));
  MG_CUDA_TRY(cudaMemcpyAsync(b->d_tile_off, tile_off.data(), (size_t)(n + 1) * sizeof(int),
                              cudaMemcpyHostToDevice, b->st));
  MG_CUDA_TRY(cudaStreamSynchronize(b->st));
  b->smem = smem + kSmemSlack;
  MG_CUDA_TRY(configure_batch(b->smem));
  const int rc = batch_capture(b);
  if (rc != MG_ERR_INVALID_ARG) return rc;
  // the default shape does not fit on this device: one block per member
  b->tune = BatchTune{512, 4, 1, 0};
  return batch_capture(b);
}

}  // namespace

extern "C" {

int mg_batch_setup(mg_batch* out, int count, const mg_grid* grids, const double* levelsets,
                   const mg_bc* bc, const mg_stab* stab, void* cuda_stream) {
  if (!out) return MG_ERR_INVALID_ARG;
  *out = nullptr;
  if (count < 1 || !grids || !levelsets) return MG_ERR_INVALID_ARG;
  mg_stab s;
  mg_default_stab(&s);
  if (stab) s = *stab;
  else s.precision = MG_MIXED;
  if (s.precision == MG_FP64) return MG_ERR_UNIMPLEMENTED;
  if (s.precision != MG_MIXED) return MG_ERR_INVALID_ARG;
  if (s.cycle != 1) return (s.cycle == 0 || s.cycle == 2) ? MG_ERR_UNIMPLEMENTED : MG_ERR_INVALID_ARG;
  // one global constant per geometry would need a per-member value
  if (s.lambda_mode != MG_LAMBDA_LOCAL)
    return s.lambda_mode == MG_LAMBDA_GLOBAL ? MG_ERR_UNIMPLEMENTED : MG_ERR_INVALID_ARG;
  if (kBoundsChecked && !bounds_word()) return MG_ERR_CUDA;
  mg_batch_ctx* b = new mg_batch_ctx();
  b->user_st = (cudaStream_t)cuda_stream;
  b->count = count;
  b->stab = s;
  auto t0 = std::chrono::steady_clock::now();
  int rc = batch_setup_impl(b, grids, levelsets, bc);
  if (rc != MG_OK) {
    mg_batch_destroy(b);
    return rc;
  }
  b->setup_ms =
      std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = b;
  return MG_OK;
}

int mg_batch_buffers(mg_batch b, long long* total_nodes, double** f, double** g, double** u) {
  if (!b) return MG_ERR_INVALID_ARG;
  if (total_nodes) *total_nodes = (long long)b->total_nodes;
  if (f) *f = b->f;
  if (g) *g = b->g;
  if (u) *u = b->u;
  return MG_OK;
}

int mg_batch_solve(mg_batch b, const double* f, const double* g, double* u, double tol,
                   mg_batch_info* info) {
  return mg_batch_solve_bc(b, f, g, nullptr, u, tol, info);
}

int mg_batch_solve_bc(mg_batch b, const double* f, const double* g, const double* gN, double* u,
                      double tol, mg_batch_info* info) {
  if (!b || !f || !g || !u || !(tol >= 0.0)) return MG_ERR_INVALID_ARG;
  double* U = nullptr;
  TRY(batch_io(b, f, g, true, gN, u, &U));
  int worst = MG_OK;
  TRY(batch_run(b, tol, &worst));
  if (U != u) {
    MG_CUDA_TRY(cudaMemcpyAsync(u, b->u, b->total_nodes * sizeof(double), cudaMemcpyDefault,
                                b->st));
    MG_CUDA_TRY(cudaStreamSynchronize(b->st));
  }
  if (info)
    for (int p = 0; p < b->count; ++p) {
      const BatchResult& r = b->h_res[p];
      info[p].status = r.status;
      info[p].cycles = r.cycles;
      info[p].checks = r.checks;
      info[p].n_dof = b->mem[p]->lev[0].n_dof;
      info[p].rel_res = r.rel_res;
    }
  return worst;
}

int mg_batch_set_shape(mg_batch b, const mg_batch_shape* shape) {
  if (!b || !shape) return MG_ERR_INVALID_ARG;
  const mg_batch_shape& s = *shape;
  if ((s.threads != 256 && s.threads != 512 && s.threads != 1024) || s.first_group < 1 ||
      s.first_group > 8 || (s.cluster != 1 && s.cluster != 2 && s.cluster != 4 && s.cluster != 8) ||
      s.coop_min_dof < 0)
    return MG_ERR_INVALID_ARG;
  const BatchTune old = b->tune;
  b->tune = BatchTune{s.threads, s.first_group, s.cluster, s.coop_min_dof};
  const int rc = batch_capture(b);
  if (rc == MG_ERR_INVALID_ARG) {
    b->tune = old;
    TRY(batch_capture(b));
    return MG_ERR_INVALID_ARG;
  }
  return rc;
}

int mg_batch_get_shape(mg_batch b, mg_batch_shape* shape) {
  if (!b || !shape) return MG_ERR_INVALID_ARG;
  shape->threads = b->tune.threads;
  shape->first_group = b->tune.first_group;
  shape->cluster = b->tune.cluster;
  shape->coop_min_dof = b->tune.coop_min_dof;
  return MG_OK;
}

int mg_batch_tune(mg_batch b, const double* f, const double* g, double tol, int reps,
                  mg_batch_shape* best_out, float* ms_out) {
  if (!b || !f || !g || !(tol >= 0.0) || reps < 1) return MG_ERR_INVALID_ARG;
  double* U = nullptr;
  TRY(batch_io(b, f, g, true, nullptr, b->u, &U));
  const BatchTune start = b->tune;
  BatchTune best{0, 0, 0, 0};
  float best_ms = 0.f;
  auto consider = [&](const BatchTune& t) -> int {
    float ms = 0.f;
    bool ok = false;
    TRY(time_shape(b, t, tol, reps, &ms, &ok));
    if (ok && (best.threads == 0 || ms < best_ms)) {
      best = t;
      best_ms = ms;
    }
    return MG_OK;
  };
  // 1. block size and cluster size, with the first group and the sharing
  //    threshold as they are
  const int th[3] = {256, 512, 1024};
  const int cl[4] = {1, 2, 4, 8};
  for (int ti = 0; ti < 3; ++ti)
    for (int ci = 0; ci < 4; ++ci)
      TRY(consider(BatchTune{th[ti], start.first_group, cl[ci], start.coop_min_dof}));
  if (!best.threads) {
    b->tune = start;
    TRY(batch_capture(b));
    return MG_ERR_NOT_CONVERGED;
  }
  // 2. cluster size x which members a cluster shares (by fine-level DOFs):
  //    larger clusters pay only when few, large members share them
  {
    const int thr[5] = {0, 8192, 32768, 65536, 131072};
    const BatchTune base = best;
    for (int ci = 1; ci < 4; ++ci)
      for (int k = 0; k < 5; ++k) {
        const BatchTune t{base.threads, base.first_group, cl[ci], thr[k]};
        if (t.cluster == base.cluster && t.coop_min_dof == base.coop_min_dof) continue;
        TRY(consider(t));
      }
  }
  // 3. V-cycles before the first fp64 check (adaptive schedule only)
  if (b->stab.inner == 0) {
    const int fg[4] = {2, 3, 4, 6};
    const BatchTune base = best;
    for (int k = 0; k < 4; ++k)
      if (fg[k] != base.first_group)
        TRY(consider(BatchTune{base.threads, fg[k], base.cluster, base.coop_min_dof}));
  }
  b->tune = best;
  TRY(batch_capture(b));
  if (best_out) {
    best_out->threads = best.threads;
    best_out->first_group = best.first_group;
    best_out->cluster = best.cluster;
    best_out->coop_min_dof = best.coop_min_dof;
  }
  if (ms_out) *ms_out = best_ms;
  return MG_OK;
}

int mg_batch_timing(mg_batch b, float* setup_ms, float* solve_ms) {
  if (!b) return MG_ERR_INVALID_ARG;
  if (setup_ms) *setup_ms = b->setup_ms;
  if (solve_ms) *solve_ms = b->solve_ms;
  return MG_OK;
}

void mg_batch_destroy(mg_batch b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (mg_ctx* c : b->mem) mg_destroy(c);
  for (void* p : b->allocs) cudaFree(p);
  if (b->h_params) cudaFreeHost(b->h_params);
  if (b->h_res) cudaFreeHost(b->h_res);
  if (b->h_err) cudaFreeHost(b->h_err);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->st) cudaStreamDestroy(b->st);
  delete b;
}

}  // extern "C"

// binds the bounds-checked build's device error word (see common.cuh)
MG_BOUNDS_BINDER(bind_bounds_api)
