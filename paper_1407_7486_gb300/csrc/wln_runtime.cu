// Runtime around the Wilson kernel: reusable batches replayed from CUDA
// graphs, a continuous-batching request server with memory-based admission,
// and the tuning knobs the autotuner sets.  None of this comes from the
// paper (whose host loop made one launch per (rho_cm, T) point); it keeps
// the GPU fed with many profiles and uneven grids at once.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "wln_internal.cuh"

using namespace wln;

namespace {

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Four statistics per point: mean and group SEM of W_scal - 1 and W_ferm - 1.
constexpr int kStats = 4;

}  // namespace

// ------------------------------------------------------------------ batch

struct wln_batch {
  int device = 0;
  const wln_ensemble* ens = nullptr;
  wln_prec prec = WLN_PREC_FP32_COMP;
  int32_t n_groups = 0, lpg = 0, n_profiles = 0;
  int64_t n_points = 0;
  WilsonPlan plan{};
  void* mem = nullptr;
  Tile* tiles = nullptr;
  ProfileDev* profs = nullptr;
  double* rho = nullptr;
  double* T = nullptr;
  QuadProfile* quad = nullptr;
  double* partial = nullptr;
  double* sums = nullptr;     // [n_points][G][K]
  double* stats = nullptr;    // [4][n_points]
  double* gg = nullptr;       // [2][n_profiles][G]: spinor, scalar
  double* gamma = nullptr;    // [2][n_profiles][2]: spinor (mean, sem), scalar (mean, sem)
  bool has_action = false;
  cudaGraphExec_t graph = nullptr;
  int64_t kernels_per_run = 0;
  GuardBufs guard;            // precision guard (FP32 compensated, whole-block groups)
  void* guard_queue = nullptr;   // its queue (regrown to the first run's need, if larger)
  bool guard_checked = false;    // the first run has shown the queue holds what it selects
  int num_sms = 0;
  int* items = nullptr;       // the Wilson launch's item counter (the creating context's)
};

namespace {

// The float pass (with the guard's selection) of a batch run.
cudaError_t enqueue_wilson(wln_batch* b, cudaStream_t s, int* flag, int64_t* launches) {
  cudaError_t err = cudaSuccess;
  if (b->guard.on) err = cudaMemsetAsync(b->guard.counters, 0, 4 * sizeof(int), s);
  if (err != cudaSuccess) return err;
  return launch_wilson(s, b->plan, b->ens->e, b->tiles, b->profs, b->rho, b->n_groups, b->lpg,
                       b->prec, b->partial, b->n_points, flag, launches,
                       b->guard.on ? &b->guard : nullptr, b->items);
}

// The rest of a batch run: the guard's recomputation, the reduction, the
// statistics and the effective action.
cudaError_t enqueue_rest(wln_batch* b, cudaStream_t s, int64_t* launches) {
  cudaError_t err = launch_guard(s, b->guard, b->ens->e, b->tiles, b->profs, b->rho, b->partial,
                                 b->num_sms, launches);
  if (err != cudaSuccess) return err;
  err = launch_reduce_partials(s, b->plan, b->ens->e, b->partial, b->n_points, b->n_groups,
                               b->lpg, b->sums);
  ++*launches;
  if (err != cudaSuccess) return err;
  const int32_t P = static_cast<int32_t>(b->n_points);
  err = launch_jackknife(s, b->sums, P, b->n_groups, b->lpg, WLN_C_SCAL, b->stats, b->stats + P,
                         nullptr, nullptr, nullptr, launches);
  if (err != cudaSuccess) return err;
  err = launch_jackknife(s, b->sums, P, b->n_groups, b->lpg, WLN_C_FERM, b->stats + 2 * P,
                         b->stats + 3 * P, nullptr, nullptr, nullptr, launches);
  if (err != cudaSuccess || !b->has_action) return err;
  const size_t gstride = static_cast<size_t>(b->n_profiles) * b->n_groups;
  err = launch_effective_action(s, b->quad, b->n_profiles, b->rho, b->T, b->sums, b->n_groups,
                                b->lpg, 1, b->gg, b->gamma, launches);
  if (err != cudaSuccess) return err;
  return launch_effective_action(s, b->quad, b->n_profiles, b->rho, b->T, b->sums, b->n_groups,
                                 b->lpg, 0, b->gg + gstride, b->gamma + 2 * b->n_profiles,
                                 launches);
}

cudaError_t enqueue_batch(wln_batch* b, cudaStream_t s, int* flag, int64_t* launches) {
  cudaError_t err = enqueue_wilson(b, s, flag, launches);
  return err != cudaSuccess ? err : enqueue_rest(b, s, launches);
}

// A (re)allocated guard queue of cap entries, bound to the batch's guard.
cudaError_t bind_guard_queue(wln_batch* b, int64_t cap) {
  if (b->guard_queue) cudaFree(b->guard_queue);
  b->guard_queue = nullptr;
  cudaError_t err = cudaMalloc(&b->guard_queue, guard_queue_bytes(cap));
  if (err != cudaSuccess) return err;
  guard_bind(b->guard, b->guard.scratch, b->guard_queue, cap, b->guard.counters);
  return cudaSuccess;
}

}  // namespace

extern "C" {

wln_status wln_set_low_angle(wln_ctx* ctx, int32_t level) {
  if (!ctx) return WLN_EINVAL;
  if (level < 0 || level > 2) return fail(ctx, WLN_EINVAL, "low_angle: level must be 0, 1 or 2");
  ctx->low_angle = level;
  return WLN_OK;
}

wln_status wln_set_tuning(wln_ctx* ctx, int32_t points_per_lane, int32_t warps, int32_t rows,
                          int32_t stages, int32_t chain_blocks) {
  if (!ctx) return WLN_EINVAL;
  // instantiated shapes (radii per lane, warps per CTA): (2, 8), (4, 4), (4, 8), (8, 8)
  const int P = points_per_lane ? points_per_lane : 4;
  const bool p_ok = P == 2 || P == 4 || P == 8;
  const bool w_ok = warps == 0 || warps == 8 || (warps == 4 && P == 4);
  const bool r_ok = rows == 0 || (rows >= 2 && rows <= 256 && (rows & (rows - 1)) == 0);
  const bool s_ok = stages == 0 || (stages >= 2 && stages <= 8);
  if (!p_ok || !w_ok || !r_ok || !s_ok || chain_blocks < 0)
    return fail(ctx, WLN_EINVAL, "tuning: (P, warps) in (2, 8), (4, 4), (4, 8), (8, 8), rows a "
                                 "power of two <= 256, stages 2..8, chain >= 0 (0 = automatic)");
  ctx->tune_P = points_per_lane;
  ctx->tune_warps = warps;
  ctx->tune_rows = rows;
  ctx->tune_stages = stages;
  ctx->tune_chain = chain_blocks;
  return WLN_OK;
}

wln_status wln_batch_create(wln_ctx* ctx, const wln_ensemble* ens, const wln_profile* profiles,
                            int32_t n_profiles, const double* rho_cm, const int32_t* rho_off,
                            const double* T, const int32_t* T_off, int32_t n_groups,
                            wln_prec prec, wln_batch** out) {
  if (!ctx || !ens || !out) return fail(ctx, WLN_EINVAL, "null argument");
  *out = nullptr;
  if (prec != WLN_PREC_FP64 && prec != WLN_PREC_FP32_COMP && prec != WLN_PREC_FP32_NAIVE)
    return fail(ctx, WLN_EINVAL, "unknown precision");
  if (ens->device != ctx->device) return fail(ctx, WLN_EINVAL, "ensemble lives on another device");
  if (n_groups < 2 || ens->e.n_loops % n_groups != 0)
    return fail(ctx, WLN_EINVAL, "n_groups must be >= 2 and divide n_loops");
  wln_status st = check_batch(ctx, profiles, n_profiles, rho_cm, rho_off, T, T_off);
  if (st != WLN_OK) return st;
  DeviceGuard guard(ctx->device);
  wln_batch* b = new (std::nothrow) wln_batch();
  if (!b) return fail(ctx, WLN_ENOMEM, "host allocation");
  b->device = ctx->device;
  b->ens = ens;
  b->prec = prec;
  b->n_groups = n_groups;
  b->lpg = ens->e.n_loops / n_groups;
  b->n_profiles = n_profiles;
  Batch bt;
  build_batch(profiles, n_profiles, rho_cm, rho_off, T, T_off, ens->e.ppl,
              plan_points_per_lane(ctx, prec), bt);
  b->n_points = bt.n_points;
  const int64_t guard_pts =
      guard_applies(ctx, prec, kModeSums, ens->e.n_loops, n_groups, profiles, n_profiles)
          ? guard_points(profiles, n_profiles, rho_cm, rho_off, T, T_off, ens->e)
          : 0;
  const bool use_guard = guard_pts > 0;
  const int bpg = guard_layout_bpg(prec, kModeSums, ens->e.n_loops, n_groups);
  b->plan = make_plan(ctx, ens->e, static_cast<int>(bt.tiles.size()), prec, kModeSums, bpg);
  b->num_sms = ctx->num_sms;
  b->items = ctx->d_items;
  std::vector<QuadProfile> qp;
  b->has_action = build_quad(profiles, n_profiles, rho_cm, rho_off, T, T_off, qp, nullptr);

  const int32_t nr = rho_off[n_profiles], nt = T_off[n_profiles];
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t at = align256(off); off = at + bytes; return at; };
  const size_t o_tiles = take(sizeof(Tile) * bt.tiles.size());
  const size_t o_profs = take(sizeof(ProfileDev) * bt.profs.size());
  const size_t o_rho = take(sizeof(double) * nr);
  const size_t o_T = take(sizeof(double) * nt);
  const size_t o_quad = take(sizeof(QuadProfile) * n_profiles);
  const size_t upload = off;
  const size_t o_part = take(sizeof(double) * static_cast<size_t>(b->plan.n_chains + n_groups) *
                             b->n_points * WLN_K);
  const size_t o_sums = take(sizeof(double) * static_cast<size_t>(b->n_points) * n_groups * WLN_K);
  const size_t o_stats = take(sizeof(double) * kStats * static_cast<size_t>(b->n_points));
  const size_t o_gg = take(sizeof(double) * 2 * static_cast<size_t>(n_profiles) * n_groups);
  const size_t o_gamma = take(sizeof(double) * 4 * static_cast<size_t>(n_profiles));
  size_t o_gscr = 0, o_gcnt = 0;
  int64_t gcap = 0;
  if (use_guard) {
    b->guard.on = 1;
    b->guard.bpg = bpg;
    b->guard.warp_bytes = guard_warp_bytes(bpg, b->plan.P);
    gcap = guard_capacity(guard_pts, n_groups, kGuardPerPair);
    o_gscr = take(static_cast<size_t>(wilson_grid(b->plan, ens->e, prec)) * b->plan.warps *
                  b->guard.warp_bytes);
    o_gcnt = take(4 * sizeof(int));
  }
  cudaError_t err = cudaMalloc(&b->mem, off);
  if (err != cudaSuccess) {
    delete b;
    return cuda_fail(ctx, err, "cudaMalloc batch");
  }
  char* d = static_cast<char*>(b->mem);
  b->tiles = reinterpret_cast<Tile*>(d + o_tiles);
  b->profs = reinterpret_cast<ProfileDev*>(d + o_profs);
  b->rho = reinterpret_cast<double*>(d + o_rho);
  b->T = reinterpret_cast<double*>(d + o_T);
  b->quad = reinterpret_cast<QuadProfile*>(d + o_quad);
  b->partial = reinterpret_cast<double*>(d + o_part);
  b->sums = reinterpret_cast<double*>(d + o_sums);
  b->stats = reinterpret_cast<double*>(d + o_stats);
  b->gg = reinterpret_cast<double*>(d + o_gg);
  b->gamma = reinterpret_cast<double*>(d + o_gamma);
  if (use_guard) {
    b->guard.scratch = d + o_gscr;
    b->guard.counters = reinterpret_cast<int*>(d + o_gcnt);
    guard_attach(b->guard, ctx);   // mode and statistics of the creating context
    err = bind_guard_queue(b, gcap);
    if (err != cudaSuccess) {
      cudaFree(b->mem);
      delete b;
      return cuda_fail(ctx, err, "cudaMalloc batch guard queue");
    }
  }
  std::vector<char> h(upload, 0);
  std::memcpy(h.data() + o_tiles, bt.tiles.data(), sizeof(Tile) * bt.tiles.size());
  std::memcpy(h.data() + o_profs, bt.profs.data(), sizeof(ProfileDev) * bt.profs.size());
  std::memcpy(h.data() + o_rho, rho_cm, sizeof(double) * nr);
  std::memcpy(h.data() + o_T, T, sizeof(double) * nt);
  if (b->has_action) std::memcpy(h.data() + o_quad, qp.data(), sizeof(QuadProfile) * n_profiles);
  err = cudaMemcpy(d, h.data(), upload, cudaMemcpyHostToDevice);
  if (err != cudaSuccess) {
    if (b->guard_queue) cudaFree(b->guard_queue);
    cudaFree(b->mem);
    delete b;
    return cuda_fail(ctx, err, "upload batch");
  }
  *out = b;
  return WLN_OK;
}

wln_status wln_batch_run(wln_ctx* ctx, wln_batch* b, int32_t use_graph) {
  if (!ctx || !b) return fail(ctx, WLN_EINVAL, "null argument");
  if (b->device != ctx->device) return fail(ctx, WLN_EINVAL, "batch lives on another device");
  DeviceGuard guard(ctx->device);
  if (b->guard.on && !b->guard_checked) {
    // The first run goes direct and waits for its float pass: if the guard
    // selected more loops than its queue holds, the queue is regrown to that
    // number and the float pass runs again.  A batch's inputs are fixed, so
    // later runs (and their graph) select the same loops.
    int64_t launches = 0;
    cudaError_t err = enqueue_wilson(b, ctx->stream, ctx->d_flag, &launches);
    int selected = 0;
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(&selected, b->guard.counters, sizeof(int), cudaMemcpyDeviceToHost,
                            ctx->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
    if (err == cudaSuccess && selected > b->guard.cap) {
      err = bind_guard_queue(b, selected);
      if (err == cudaSuccess) err = enqueue_wilson(b, ctx->stream, ctx->d_flag, &launches);
    }
    if (err == cudaSuccess) err = enqueue_rest(b, ctx->stream, &launches);
    ctx->launches += launches;
    if (err != cudaSuccess) return cuda_fail(ctx, err, "batch run");
    b->guard_checked = true;
    return WLN_OK;
  }
  if (!use_graph) {
    int64_t launches = 0;
    cudaError_t err = enqueue_batch(b, ctx->stream, ctx->d_flag, &launches);
    ctx->launches += launches;
    if (err != cudaSuccess) return cuda_fail(ctx, err, "batch run");
    return WLN_OK;
  }
  if (!ctx->stream) return fail(ctx, WLN_EINVAL, "graph replay needs a non-default stream");
  if (!b->graph) {
    cudaError_t err = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed);
    if (err != cudaSuccess) return cuda_fail(ctx, err, "begin capture");
    int64_t launches = 0;
    cudaError_t err_enq = enqueue_batch(b, ctx->stream, ctx->d_flag, &launches);
    cudaGraph_t g = nullptr;
    err = cudaStreamEndCapture(ctx->stream, &g);
    if (err_enq != cudaSuccess || err != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(ctx, err_enq != cudaSuccess ? err_enq : err, "capture batch");
    }
    err = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (err != cudaSuccess) {
      b->graph = nullptr;
      return cuda_fail(ctx, err, "instantiate batch graph");
    }
    b->kernels_per_run = launches;
  }
  cudaError_t err = cudaGraphLaunch(b->graph, ctx->stream);
  if (err != cudaSuccess) return cuda_fail(ctx, err, "launch batch graph");
  ctx->launches += b->kernels_per_run;
  return WLN_OK;
}

wln_status wln_batch_results(wln_ctx* ctx, const wln_batch* b, double* group_sums, double* stats,
                             double* gamma) {
  if (!ctx || !b) return fail(ctx, WLN_EINVAL, "null argument");
  if (gamma && !b->has_action)
    return fail(ctx, WLN_EINVAL, "no effective action: a profile's grid is not evenly spaced in "
                                 "rho and geometric in T");
  DeviceGuard guard(ctx->device);
  cudaError_t err = cudaSuccess;
  bool host = false;
  auto copy = [&](double* dst, const double* src, size_t n) {
    if (!dst || err != cudaSuccess) return;
    host = host || !is_device_ptr(dst);
    err = cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, ctx->stream);
  };
  copy(group_sums, b->sums, static_cast<size_t>(b->n_points) * b->n_groups * WLN_K);
  copy(stats, b->stats, kStats * static_cast<size_t>(b->n_points));
  copy(gamma, b->gamma, 4 * static_cast<size_t>(b->n_profiles));
  if (err == cudaSuccess && host) err = cudaStreamSynchronize(ctx->stream);
  if (err != cudaSuccess) return cuda_fail(ctx, err, "batch results");
  if (host) return wln_synchronize(ctx);
  return WLN_OK;
}

wln_status wln_batch_info(const wln_batch* b, int64_t* n_points, int32_t* n_tiles,
                          int32_t* points_per_lane, int32_t* chain_blocks, int64_t* kernels_per_run) {
  if (!b) return WLN_EINVAL;
  if (n_points) *n_points = b->n_points;
  if (n_tiles) *n_tiles = b->plan.n_tiles;
  if (points_per_lane) *points_per_lane = b->plan.P;
  if (chain_blocks) *chain_blocks = b->plan.chain;
  if (kernels_per_run) *kernels_per_run = b->kernels_per_run;
  return WLN_OK;
}

wln_status wln_batch_free(wln_ctx* ctx, wln_batch* b) {
  if (!b) return fail(ctx, WLN_EINVAL, "null batch");
  DeviceGuard guard(b->device);
  if (ctx) cudaStreamSynchronize(ctx->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->guard_queue) cudaFree(b->guard_queue);
  if (b->mem) cudaFree(b->mem);
  delete b;
  return WLN_OK;
}

}  // extern "C"

// ----------------------------------------------------------------- server

namespace {

enum ReqState { kQueued = 0, kActive = 1, kFinalizing = 2, kDone = 3, kCancelled = 4 };

struct Request {
  int64_t id = 0;
  int state = kQueued;
  wln_profile prof{};
  std::vector<double> rho, T;
  int64_t n_points = 0;
  std::vector<Tile> tiles;          // p0 and rho0 within the request; profile set per step
  int32_t n_tile_groups = 0, next_tg = 0, done_tg = 0, inflight_tg = 0;
  bool has_action = false;
  bool allocated = false;           // holds an arena block
  QuadProfile quad{};
  // arena block
  size_t off = 0, bytes = 0;
  size_t o_part = 0, o_sums = 0, o_stats = 0, o_gg = 0, o_gamma = 0, o_quad = 0, o_rho = 0, o_T = 0;
  // results on the host (pinned), filled by the finalisation copy
  double* h_res = nullptr;
  cudaEvent_t done = nullptr;
};

// First-fit allocator over the server's device arena.
struct Arena {
  std::map<size_t, size_t> free_;   // offset -> size
  void init(size_t bytes) { free_.clear(); free_[0] = bytes; }
  bool alloc(size_t bytes, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t largest() const {
    size_t m = 0;
    for (auto& kv : free_) m = std::max(m, kv.second);
    return m;
  }
};

}  // namespace

struct wln_server {
  wln_ctx* ctx = nullptr;
  const wln_ensemble* ens = nullptr;
  wln_prec prec = WLN_PREC_FP32_COMP;
  int32_t G = 0, lpg = 0, P = 4, warps = 8;
  WilsonPlan base{};
  char* arena = nullptr;
  size_t arena_bytes = 0;
  Arena alloc;
  int32_t tg_per_step = 0;
  std::deque<int64_t> queue;
  std::vector<int64_t> active;      // admission order
  std::unordered_map<int64_t, Request> reqs;
  int64_t next_id = 1;
  cudaStream_t fin_stream = nullptr;
  // two step slots, so one step can be prepared while the other runs
  char* d_step[2] = {nullptr, nullptr};
  char* h_step[2] = {nullptr, nullptr};
  size_t step_bytes = 0;
  cudaEvent_t step_done[2] = {nullptr, nullptr};
  std::vector<std::pair<int64_t, int32_t>> inflight[2];
  int cur = 0;
  int64_t steps = 0;
  // precision guard: per-warp records shared by the steps (they run in stream
  // order), a queue and counters per step slot; a slot's queue is sized before
  // each step for everything its points could select (kGuardSel loops per
  // (point, group) that can reach the spin floor), grown when a step needs more
  GuardBufs guard[2];
  char* d_guard = nullptr;
  void* guard_queue[2] = {nullptr, nullptr};
};

namespace {

size_t request_bytes(const wln_server* sv, Request& r) {
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t at = align256(off); off = at + bytes; return at; };
  r.o_part = take(sizeof(double) * static_cast<size_t>(sv->base.n_chains + sv->G) * r.n_points * WLN_K);
  r.o_sums = take(sizeof(double) * static_cast<size_t>(r.n_points) * sv->G * WLN_K);
  r.o_stats = take(sizeof(double) * kStats * static_cast<size_t>(r.n_points));
  r.o_gg = take(sizeof(double) * 2 * static_cast<size_t>(sv->G));
  r.o_gamma = take(sizeof(double) * 4);
  r.o_quad = take(sizeof(QuadProfile));
  r.o_rho = take(sizeof(double) * r.rho.size());
  r.o_T = take(sizeof(double) * r.T.size());
  return align256(off);
}

size_t result_doubles(const wln_server* sv, const Request& r) {
  return static_cast<size_t>(r.n_points) * sv->G * WLN_K + kStats * static_cast<size_t>(r.n_points) + 4;
}

void release_request(wln_server* sv, Request& r) {
  if (r.allocated) sv->alloc.release(r.off, r.bytes);
  r.allocated = false;
  if (r.h_res) cudaFreeHost(r.h_res);
  r.h_res = nullptr;
}

// Admit queued requests, oldest first, while their blocks fit in the arena.
wln_status admit(wln_server* sv) {
  while (!sv->queue.empty()) {
    Request& r = sv->reqs[sv->queue.front()];
    if (!sv->alloc.alloc(r.bytes, &r.off)) break;
    r.allocated = true;
    char* base = sv->arena + r.off;
    cudaError_t err = cudaMallocHost(&r.h_res, sizeof(double) * result_doubles(sv, r));
    if (err == cudaSuccess && r.has_action) {
      QuadProfile q = r.quad;
      q.rho_base = 0; q.T_base = 0; q.p0 = 0;
      err = cudaMemcpyAsync(base + r.o_quad, &q, sizeof(q), cudaMemcpyHostToDevice, sv->fin_stream);
      if (err == cudaSuccess) err = cudaMemcpyAsync(base + r.o_rho, r.rho.data(), sizeof(double) * r.rho.size(), cudaMemcpyHostToDevice, sv->fin_stream);
      if (err == cudaSuccess) err = cudaMemcpyAsync(base + r.o_T, r.T.data(), sizeof(double) * r.T.size(), cudaMemcpyHostToDevice, sv->fin_stream);
      if (err == cudaSuccess) err = cudaStreamSynchronize(sv->fin_stream);
    }
    if (err != cudaSuccess) return cuda_fail(sv->ctx, err, "admit request");
    const int64_t part_base = static_cast<int64_t>((r.off + r.o_part) / sizeof(double));
    for (Tile& t : r.tiles) t.part_base = part_base;
    r.state = kActive;
    sv->active.push_back(r.id);
    sv->queue.pop_front();
  }
  return WLN_OK;
}

// Reduce, group statistics, effective action and copy-back of a request whose
// last tile group has finished, on the server's finalisation stream.
wln_status finalize(wln_server* sv, Request& r) {
  cudaStream_t s = sv->fin_stream;
  char* base = sv->arena + r.off;
  double* sums = reinterpret_cast<double*>(base + r.o_sums);
  double* stats = reinterpret_cast<double*>(base + r.o_stats);
  double* gg = reinterpret_cast<double*>(base + r.o_gg);
  double* gamma = reinterpret_cast<double*>(base + r.o_gamma);
  const int32_t np = static_cast<int32_t>(r.n_points);
  int64_t launches = 0;
  cudaError_t err = launch_reduce_partials(s, sv->base, sv->ens->e,
                                           reinterpret_cast<double*>(base + r.o_part), r.n_points,
                                           sv->G, sv->lpg, sums);
  ++launches;
  if (err == cudaSuccess)
    err = launch_jackknife(s, sums, np, sv->G, sv->lpg, WLN_C_SCAL, stats, stats + np, nullptr,
                           nullptr, nullptr, &launches);
  if (err == cudaSuccess)
    err = launch_jackknife(s, sums, np, sv->G, sv->lpg, WLN_C_FERM, stats + 2 * np, stats + 3 * np,
                           nullptr, nullptr, nullptr, &launches);
  if (err == cudaSuccess && r.has_action) {
    const QuadProfile* q = reinterpret_cast<const QuadProfile*>(base + r.o_quad);
    const double* rho = reinterpret_cast<const double*>(base + r.o_rho);
    const double* T = reinterpret_cast<const double*>(base + r.o_T);
    err = launch_effective_action(s, q, 1, rho, T, sums, sv->G, sv->lpg, 1, gg, gamma, &launches);
    if (err == cudaSuccess)
      err = launch_effective_action(s, q, 1, rho, T, sums, sv->G, sv->lpg, 0, gg + sv->G,
                                    gamma + 2, &launches);
  }
  sv->ctx->launches += launches;
  const size_t n_sums = static_cast<size_t>(r.n_points) * sv->G * WLN_K;
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(r.h_res, sums, n_sums * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(r.h_res + n_sums, stats, kStats * np * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(r.h_res + n_sums + kStats * np, gamma, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess && !r.done) err = cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming);
  if (err == cudaSuccess) err = cudaEventRecord(r.done, s);
  if (err != cudaSuccess) return cuda_fail(sv->ctx, err, "finalize request");
  r.state = kFinalizing;
  return WLN_OK;
}

// Account for a finished step: count its tile groups, finalize completed
// requests, release cancelled ones once nothing of theirs is in flight.
wln_status retire(wln_server* sv, int slot) {
  for (auto& [id, tg] : sv->inflight[slot]) {
    (void)tg;
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end()) continue;
    Request& r = it->second;
    r.inflight_tg--;
    r.done_tg++;
    if (r.state == kCancelled) {
      if (r.inflight_tg == 0) release_request(sv, r);
    } else if (r.done_tg == r.n_tile_groups) {
      sv->active.erase(std::find(sv->active.begin(), sv->active.end(), id));
      wln_status st = finalize(sv, r);
      if (st != WLN_OK) return st;
    }
  }
  sv->inflight[slot].clear();
  return WLN_OK;
}

wln_status launch_step(wln_server* sv, int slot) {
  // Pick up to tg_per_step tile groups, oldest request first.
  std::vector<std::pair<int64_t, int32_t>> pick;
  for (int64_t id : sv->active) {
    Request& r = sv->reqs[id];
    while (r.next_tg < r.n_tile_groups && static_cast<int32_t>(pick.size()) < sv->tg_per_step) {
      pick.emplace_back(id, r.next_tg++);
      r.inflight_tg++;
    }
    if (static_cast<int32_t>(pick.size()) >= sv->tg_per_step) break;
  }
  if (pick.empty()) return WLN_OK;
  // Work list of this step: tiles, one profile and radius set per request.
  std::vector<Tile> tiles;
  std::vector<ProfileDev> profs;
  std::vector<double> rho;
  std::unordered_map<int64_t, std::pair<int32_t, int32_t>> where;   // id -> (profile, rho base)
  for (auto& [id, tg] : pick) {
    Request& r = sv->reqs[id];
    auto w = where.find(id);
    if (w == where.end()) {
      w = where.emplace(id, std::make_pair(static_cast<int32_t>(profs.size()),
                                           static_cast<int32_t>(rho.size()))).first;
      profs.push_back(profile_constants(r.prof, sv->ens->e.ppl));
      rho.insert(rho.end(), r.rho.begin(), r.rho.end());
    }
    for (int j = 0; j < sv->warps; ++j) {
      Tile t = r.tiles[static_cast<size_t>(tg) * sv->warps + j];
      t.profile = w->second.first;
      t.rho0 += w->second.second;
      tiles.push_back(t);
    }
  }
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t at = align256(off); off = at + bytes; return at; };
  const size_t o_tiles = take(sizeof(Tile) * tiles.size());
  const size_t o_profs = take(sizeof(ProfileDev) * profs.size());
  const size_t o_rho = take(sizeof(double) * rho.size());
  if (off > sv->step_bytes) return fail(sv->ctx, WLN_EINVAL, "step work list exceeds its buffer");
  char* h = sv->h_step[slot];
  std::memcpy(h + o_tiles, tiles.data(), sizeof(Tile) * tiles.size());
  std::memcpy(h + o_profs, profs.data(), sizeof(ProfileDev) * profs.size());
  std::memcpy(h + o_rho, rho.data(), sizeof(double) * rho.size());
  char* d = sv->d_step[slot];
  cudaStream_t s = sv->ctx->stream;
  cudaError_t err = cudaMemcpyAsync(d, h, off, cudaMemcpyHostToDevice, s);
  WilsonPlan plan = sv->base;
  plan.n_tiles = static_cast<int>(tiles.size());
  plan.n_tile_groups = static_cast<int>(pick.size());
  plan.n_items = static_cast<int64_t>(plan.n_chains) * plan.n_tile_groups;
  int64_t launches = 0;
  GuardBufs& gb = sv->guard[slot];
  if (err == cudaSuccess && gb.on) {
    int64_t reach = 0;
    for (auto& [id, tg] : pick) {
      const Request& r = sv->reqs[id];
      for (int j = 0; j < sv->warps; ++j) {
        const Tile& tl = r.tiles[static_cast<size_t>(tg) * sv->warps + j];
        for (int p = 0; p < tl.n_valid; ++p)
          reach += guard_point_reaches(r.prof, r.rho[tl.rho0 + p], tl.T, sv->ens->e);
      }
    }
    const int64_t need = guard_capacity(reach, sv->G, kGuardSel);
    if (need > gb.cap) {
      // this slot's previous step has retired, so its queue is idle
      if (sv->guard_queue[slot]) cudaFree(sv->guard_queue[slot]);
      sv->guard_queue[slot] = nullptr;
      err = cudaMalloc(&sv->guard_queue[slot], guard_queue_bytes(need));
      if (err == cudaSuccess) guard_bind(gb, gb.scratch, sv->guard_queue[slot], need, gb.counters);
    }
    if (err == cudaSuccess) err = cudaMemsetAsync(gb.counters, 0, 4 * sizeof(int), s);
  }
  if (err == cudaSuccess)
    err = launch_wilson(s, plan, sv->ens->e, reinterpret_cast<Tile*>(d + o_tiles),
                        reinterpret_cast<ProfileDev*>(d + o_profs),
                        reinterpret_cast<double*>(d + o_rho), sv->G, sv->lpg, sv->prec,
                        reinterpret_cast<double*>(sv->arena), 0, sv->ctx->d_flag, &launches,
                        gb.on ? &gb : nullptr, sv->ctx->d_items);
  if (err == cudaSuccess)
    err = launch_guard(s, gb, sv->ens->e, reinterpret_cast<Tile*>(d + o_tiles),
                       reinterpret_cast<ProfileDev*>(d + o_profs),
                       reinterpret_cast<double*>(d + o_rho), reinterpret_cast<double*>(sv->arena),
                       sv->ctx->num_sms, &launches);
  sv->ctx->launches += launches;
  if (err == cudaSuccess) err = cudaEventRecord(sv->step_done[slot], s);
  if (err != cudaSuccess) return cuda_fail(sv->ctx, err, "server step");
  sv->inflight[slot] = std::move(pick);
  sv->steps++;
  return WLN_OK;
}

}  // namespace

extern "C" {

wln_status wln_server_create(wln_ctx* ctx, const wln_ensemble* ens, int32_t n_groups,
                             wln_prec prec, int64_t arena_bytes, int32_t tile_groups_per_step,
                             wln_server** out) {
  if (!ctx || !ens || !out) return fail(ctx, WLN_EINVAL, "null argument");
  *out = nullptr;
  if (prec != WLN_PREC_FP64 && prec != WLN_PREC_FP32_COMP && prec != WLN_PREC_FP32_NAIVE)
    return fail(ctx, WLN_EINVAL, "unknown precision");
  if (n_groups < 2 || ens->e.n_loops % n_groups != 0)
    return fail(ctx, WLN_EINVAL, "n_groups must be >= 2 and divide n_loops");
  if (arena_bytes < (1 << 20) || tile_groups_per_step < 1)
    return fail(ctx, WLN_EINVAL, "arena >= 1 MiB and at least one tile group per step");
  DeviceGuard guard(ctx->device);
  wln_server* sv = new (std::nothrow) wln_server();
  if (!sv) return fail(ctx, WLN_ENOMEM, "host allocation");
  sv->ctx = ctx;
  sv->ens = ens;
  sv->prec = prec;
  sv->G = n_groups;
  sv->lpg = ens->e.n_loops / n_groups;
  sv->tg_per_step = tile_groups_per_step;
  // One fixed work decomposition (chain length) for every step, so a request's
  // sums are accumulated in the same order whatever it is batched with.
  const wln_profile tube{WLN_PROFILE_FLUX_TUBE, 0, 1.0, 1.0, 0.0};
  const bool use_guard = guard_applies(ctx, prec, kModeSums, ens->e.n_loops, n_groups, &tube, 1);
  const int bpg = guard_layout_bpg(prec, kModeSums, ens->e.n_loops, n_groups);
  sv->base = make_plan(ctx, ens->e, tile_groups_per_step * 8, prec, kModeSums, bpg);
  sv->P = sv->base.P;
  sv->warps = sv->base.warps;
  sv->arena_bytes = static_cast<size_t>(arena_bytes);
  sv->step_bytes = align256(sizeof(Tile) * tile_groups_per_step * sv->warps) +
                   align256(sizeof(ProfileDev) * tile_groups_per_step * sv->warps) +
                   align256(sizeof(double) * tile_groups_per_step * sv->warps * sv->P) + 1024;
  cudaError_t err = cudaMalloc(reinterpret_cast<void**>(&sv->arena), sv->arena_bytes);
  for (int i = 0; i < 2 && err == cudaSuccess; ++i) {
    err = cudaMalloc(reinterpret_cast<void**>(&sv->d_step[i]), sv->step_bytes);
    if (err == cudaSuccess) err = cudaMallocHost(reinterpret_cast<void**>(&sv->h_step[i]), sv->step_bytes);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&sv->step_done[i], cudaEventDisableTiming);
  }
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&sv->fin_stream, cudaStreamNonBlocking);
  if (err == cudaSuccess && use_guard) {
    const size_t scr = align256(static_cast<size_t>(wilson_grid(sv->base, ens->e, prec)) *
                                sv->base.warps * guard_warp_bytes(bpg, sv->P));
    const size_t cnt = 256;
    err = cudaMalloc(reinterpret_cast<void**>(&sv->d_guard), scr + 2 * cnt);
    for (int i = 0; i < 2 && err == cudaSuccess; ++i) {
      GuardBufs& g = sv->guard[i];
      g.on = 1;
      g.bpg = bpg;
      g.warp_bytes = guard_warp_bytes(bpg, sv->P);
      // the queue comes with the first step that needs one
      guard_bind(g, sv->d_guard, nullptr, 0, reinterpret_cast<int*>(sv->d_guard + scr + i * cnt));
      guard_attach(g, ctx);
    }
  }
  if (err != cudaSuccess) {
    wln_server_free(sv);
    return cuda_fail(ctx, err, "server allocation");
  }
  sv->alloc.init(sv->arena_bytes);
  *out = sv;
  return WLN_OK;
}

wln_status wln_server_submit(wln_server* sv, const wln_profile* profile, const double* rho,
                             int32_t n_rho, const double* T, int32_t n_T, int64_t* id) {
  if (!sv || !profile || !rho || !T || !id) return WLN_EINVAL;
  const int32_t roff[2] = {0, n_rho}, toff[2] = {0, n_T};
  if (n_rho < 1 || n_T < 1) return fail(sv->ctx, WLN_EINVAL, "a request needs rho and T values");
  wln_status st = check_batch(sv->ctx, profile, 1, rho, roff, T, toff);
  if (st != WLN_OK) return st;
  Request r;
  r.id = sv->next_id++;
  r.prof = *profile;
  r.rho.assign(rho, rho + n_rho);
  r.T.assign(T, T + n_T);
  r.n_points = static_cast<int64_t>(n_rho) * n_T;
  Batch bt;
  build_batch(profile, 1, rho, roff, T, toff, sv->ens->e.ppl, sv->P, bt);
  r.tiles = bt.tiles;
  // pad to whole tile groups with inactive tiles
  while (r.tiles.size() % sv->warps) {
    Tile pad{};
    pad.T = 1.0;
    pad.part_stride = static_cast<int32_t>(r.n_points);
    r.tiles.push_back(pad);
  }
  r.n_tile_groups = static_cast<int32_t>(r.tiles.size() / sv->warps);
  std::vector<QuadProfile> qp;
  r.has_action = build_quad(profile, 1, rho, roff, T, toff, qp, nullptr);
  if (r.has_action) r.quad = qp[0];
  r.bytes = request_bytes(sv, r);
  if (r.bytes > sv->arena_bytes)
    return fail(sv->ctx, WLN_EINVAL,
                "request needs " + std::to_string(r.bytes >> 20) + " MiB; the arena holds " +
                std::to_string(sv->arena_bytes >> 20) + " MiB");
  *id = r.id;
  sv->queue.push_back(r.id);
  sv->reqs.emplace(r.id, std::move(r));
  return WLN_OK;
}

wln_status wln_server_step(wln_server* sv, int32_t* n_active, int32_t* n_queued) {
  if (!sv) return WLN_EINVAL;
  DeviceGuard guard(sv->ctx->device);
  // Retire finished steps (without waiting).
  for (int slot = 0; slot < 2; ++slot) {
    if (sv->inflight[slot].empty()) continue;
    if (cudaEventQuery(sv->step_done[slot]) == cudaSuccess) {
      wln_status st = retire(sv, slot);
      if (st != WLN_OK) return st;
    } else {
      (void)cudaGetLastError();
    }
  }
  // Finished finalisations free their arena blocks.
  for (auto& kv : sv->reqs) {
    Request& r = kv.second;
    if (r.state == kFinalizing && cudaEventQuery(r.done) == cudaSuccess) {
      r.state = kDone;
      sv->alloc.release(r.off, r.bytes);
      r.allocated = false;
    }
  }
  (void)cudaGetLastError();
  wln_status st = admit(sv);
  if (st != WLN_OK) return st;
  // Keep up to two steps in flight: when both slots are busy, wait for the older.
  const int slot = sv->cur;
  if (!sv->inflight[slot].empty()) {
    cudaError_t err = cudaEventSynchronize(sv->step_done[slot]);
    if (err != cudaSuccess) return cuda_fail(sv->ctx, err, "wait for step");
    if ((st = retire(sv, slot)) != WLN_OK) return st;
  }
  if ((st = launch_step(sv, slot)) != WLN_OK) return st;
  if (!sv->inflight[slot].empty()) sv->cur ^= 1;
  if (n_active) *n_active = static_cast<int32_t>(sv->active.size());
  if (n_queued) *n_queued = static_cast<int32_t>(sv->queue.size());
  return WLN_OK;
}

wln_status wln_server_poll(wln_server* sv, int64_t id, int32_t* state, double* group_sums,
                           double* stats, double* gamma) {
  if (!sv || !state) return WLN_EINVAL;
  auto it = sv->reqs.find(id);
  if (it == sv->reqs.end()) return fail(sv->ctx, WLN_EINVAL, "unknown request");
  Request& r = it->second;
  if (r.state == kFinalizing && cudaEventQuery(r.done) == cudaSuccess) {
    r.state = kDone;
    sv->alloc.release(r.off, r.bytes);
    r.allocated = false;
  }
  (void)cudaGetLastError();
  *state = r.state;
  if (r.state != kDone) return WLN_OK;
  const size_t n_sums = static_cast<size_t>(r.n_points) * sv->G * WLN_K;
  if (group_sums) std::memcpy(group_sums, r.h_res, n_sums * sizeof(double));
  if (stats) std::memcpy(stats, r.h_res + n_sums, kStats * r.n_points * sizeof(double));
  if (gamma) std::memcpy(gamma, r.h_res + n_sums + kStats * r.n_points, 4 * sizeof(double));
  return WLN_OK;
}

wln_status wln_server_release(wln_server* sv, int64_t id) {
  if (!sv) return WLN_EINVAL;
  auto it = sv->reqs.find(id);
  if (it == sv->reqs.end()) return fail(sv->ctx, WLN_EINVAL, "unknown request");
  Request& r = it->second;
  if (r.state != kDone && r.state != kCancelled) return fail(sv->ctx, WLN_EBUSY, "request not finished");
  if (r.state == kCancelled && r.inflight_tg > 0) return fail(sv->ctx, WLN_EBUSY, "work in flight");
  release_request(sv, r);
  if (r.done) cudaEventDestroy(r.done);
  sv->reqs.erase(it);
  return WLN_OK;
}

wln_status wln_server_cancel(wln_server* sv, int64_t id) {
  if (!sv) return WLN_EINVAL;
  auto it = sv->reqs.find(id);
  if (it == sv->reqs.end()) return fail(sv->ctx, WLN_EINVAL, "unknown request");
  Request& r = it->second;
  if (r.state == kQueued) {
    sv->queue.erase(std::find(sv->queue.begin(), sv->queue.end(), id));
    r.state = kCancelled;
  } else if (r.state == kActive) {
    sv->active.erase(std::find(sv->active.begin(), sv->active.end(), id));
    r.state = kCancelled;
    if (r.inflight_tg == 0) release_request(sv, r);
  } else {
    return fail(sv->ctx, WLN_EBUSY, "request already finishing");
  }
  return WLN_OK;
}

wln_status wln_server_info(const wln_server* sv, int64_t* steps, int64_t* arena_free_bytes,
                           int32_t* n_active, int32_t* n_queued) {
  if (!sv) return WLN_EINVAL;
  if (steps) *steps = sv->steps;
  if (arena_free_bytes) {
    size_t f = 0;
    for (auto& kv : sv->alloc.free_) f += kv.second;
    *arena_free_bytes = static_cast<int64_t>(f);
  }
  if (n_active) *n_active = static_cast<int32_t>(sv->active.size());
  if (n_queued) *n_queued = static_cast<int32_t>(sv->queue.size());
  return WLN_OK;
}

wln_status wln_server_free(wln_server* sv) {
  if (!sv) return WLN_EINVAL;
  DeviceGuard guard(sv->ctx->device);
  cudaStreamSynchronize(sv->ctx->stream);
  if (sv->fin_stream) {
    cudaStreamSynchronize(sv->fin_stream);
    cudaStreamDestroy(sv->fin_stream);
  }
  for (auto& kv : sv->reqs) {
    if (kv.second.h_res) cudaFreeHost(kv.second.h_res);
    if (kv.second.done) cudaEventDestroy(kv.second.done);
  }
  for (int i = 0; i < 2; ++i) {
    if (sv->d_step[i]) cudaFree(sv->d_step[i]);
  }
  if (sv->d_guard) cudaFree(sv->d_guard);
  for (void* q : sv->guard_queue)
    if (q) cudaFree(q);
  for (int i = 0; i < 2; ++i) {
    if (sv->h_step[i]) cudaFreeHost(sv->h_step[i]);
    if (sv->step_done[i]) cudaEventDestroy(sv->step_done[i]);
  }
  if (sv->arena) cudaFree(sv->arena);
  delete sv;
  return WLN_OK;
}

}  // extern "C"
