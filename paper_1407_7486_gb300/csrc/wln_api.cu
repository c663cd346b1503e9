// C ABI of libwln: argument checks, device buffers and launch sequencing.
// The arithmetic lives in wln_gen.cu, wln_wilson.cu and wln_stats.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "wln_internal.cuh"

namespace wln {

wln_status fail(wln_ctx* ctx, wln_status st, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return st;
}

wln_status cuda_fail(wln_ctx* ctx, cudaError_t err, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(err);
  (void)cudaGetLastError();
  return fail(ctx, err == cudaErrorMemoryAllocation ? WLN_ENOMEM : WLN_ECUDA, m);
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

wln_status ensure_scratch(wln_ctx* ctx, size_t bytes) {
  if (ctx->scratch.bytes >= bytes) return WLN_OK;
  cudaError_t err = cudaStreamSynchronize(ctx->stream);
  if (err != cudaSuccess) return cuda_fail(ctx, err, "synchronize before growing scratch");
  if (ctx->scratch.ptr) cudaFree(ctx->scratch.ptr);
  ctx->scratch.ptr = nullptr;
  ctx->scratch.bytes = 0;
  const size_t want = bytes + bytes / 4;
  err = cudaMalloc(&ctx->scratch.ptr, want);
  if (err != cudaSuccess) return cuda_fail(ctx, err, "cudaMalloc scratch");
  ctx->scratch.bytes = want;
  return WLN_OK;
}

wln_status ensure_pinned(wln_ctx* ctx, size_t bytes) {
  // The previous upload from the staging buffer must have finished.
  cudaError_t err = cudaEventSynchronize(ctx->staging_done);
  if (err != cudaSuccess) return cuda_fail(ctx, err, "wait for staging buffer");
  if (ctx->pinned_bytes >= bytes) return WLN_OK;
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  ctx->pinned = nullptr;
  ctx->pinned_bytes = 0;
  const size_t want = bytes + bytes / 4 + 4096;
  err = cudaMallocHost(&ctx->pinned, want);
  if (err != cudaSuccess) return cuda_fail(ctx, err, "cudaMallocHost staging");
  ctx->pinned_bytes = want;
  return WLN_OK;
}

// Restores the caller's current device on scope exit.
DeviceGuard::DeviceGuard(int dev) {
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  if (prev != dev) cudaSetDevice(dev);
}

DeviceGuard::~DeviceGuard() {
  int cur = -1;
  if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
}

// Reads (and clears) the device error flag after the stream's work is done.
wln_status check_flag(wln_ctx* ctx) {
  int h = 0;
  cudaError_t err = cudaMemcpyAsync(&h, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
  if (err != cudaSuccess) return cuda_fail(ctx, err, "synchronize");
  if (h != 0) {
    cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    if (h == kErrGuardQueue)
      return fail(ctx, WLN_ENOMEM,
                  "the precision guard's queue was full: some loops it selected kept float "
                  "precision (see wln_precision_guard_stats)");
    return fail(ctx, WLN_ETIMEOUT,
                h == kErrTimeoutFull    ? "a staged-copy wait ran out (device)"
                : h == kErrTimeoutEmpty ? "a buffer-release wait ran out (device)"
                                        : "the self-test wait ran out (device), as intended");
  }
  return WLN_OK;
}

namespace {


size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Bump allocator over the context's scratch buffer for one call.
struct Carve {
  size_t off = 0;
  template <class T>
  size_t take(size_t n) {
    const size_t at = align_up(off);
    off = at + n * sizeof(T);
    return at;
  }
};

template <class T>
T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

wln_status check_loops(wln_ctx* ctx, int32_t n_loops, int32_t ppl) {
  if (!is_pow2(ppl) || ppl < 4 || ppl > 16384)
    return fail(ctx, WLN_EINVAL, "ppl must be a power of two in [4, 16384]");
  if (n_loops < 1 || n_loops > (1 << 24))
    return fail(ctx, WLN_EINVAL, "n_loops must be in [1, 2^24]");
  return WLN_OK;
}

wln_status alloc_ensemble(wln_ctx* ctx, int32_t n_loops, int32_t ppl, bool fp64, wln_ensemble** out) {
  wln_ensemble* en = new (std::nothrow) wln_ensemble();
  if (!en) return fail(ctx, WLN_ENOMEM, "host allocation");
  en->device = ctx->device;
  en->e.n_loops = n_loops;
  en->e.ppl = ppl;
  en->e.n_blocks = (n_loops + 31) / 32;
  const size_t n4 = static_cast<size_t>(en->e.n_blocks) * (ppl / 2) * 32;
  const size_t n64 = fp64 ? static_cast<size_t>(n_loops) * 2 * ppl : 0;
  for (size_t i = 0; i < ctx->ens_cache.size(); ++i) {
    const wln_ctx::EnsembleMem m = ctx->ens_cache[i];
    if (m.n4 == n4 && m.n_blocks == static_cast<size_t>(en->e.n_blocks) && m.n64 == n64) {
      en->e.blocks = m.blocks;
      en->e.stats = m.stats;
      bind_ensemble_stats(en->e);
      en->e.xy64 = m.xy64;
      ctx->ens_cache.erase(ctx->ens_cache.begin() + static_cast<std::ptrdiff_t>(i));
      *out = en;
      return WLN_OK;
    }
  }
  cudaError_t err = cudaMalloc(&en->e.blocks, n4 * sizeof(float4));
  if (err == cudaSuccess)
    err = cudaMalloc(&en->e.stats, ensemble_stats_bytes(en->e.n_blocks, ppl));
  if (err == cudaSuccess) bind_ensemble_stats(en->e);
  if (err == cudaSuccess && fp64) err = cudaMalloc(&en->e.xy64, n64 * sizeof(double));
  if (err != cudaSuccess) {
    if (en->e.blocks) cudaFree(en->e.blocks);
    if (en->e.stats) cudaFree(en->e.stats);
    delete en;
    return cuda_fail(ctx, err, "cudaMalloc ensemble");
  }
  *out = en;
  return WLN_OK;
}

wln_status finish_ensemble(wln_ctx* ctx, wln_ensemble* en, int* d_deg, wln_ensemble** out) {
  // the degeneracy flag, and the block statistics for the largest |y| of any
  // loop (kept on the host for the precision guard's bound on which points
  // can reach its spin floor), read back with one wait
  int deg = 0;
  std::vector<float2> st(static_cast<size_t>(en->e.n_blocks));
  cudaError_t err = cudaMemcpyAsync(&deg, d_deg, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(st.data(), en->e.stats, st.size() * sizeof(float2),
                          cudaMemcpyDeviceToHost, ctx->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
  if (err != cudaSuccess) {
    wln_free_ensemble(ctx, en);
    return cuda_fail(ctx, err, "loop generation");
  }
  if (deg) {
    wln_free_ensemble(ctx, en);
    return fail(ctx, WLN_EINVAL, "two consecutive loop points coincide (zero-length segment)");
  }
  for (const float2& s : st) en->e.ymax = std::fmax(en->e.ymax, s.y);
  *out = en;
  return WLN_OK;
}

// A caller's output array: written directly when on the device, through a
// scratch buffer and a copy back when on the host.
struct Out {
  void* user = nullptr;
  void* dev = nullptr;
  size_t bytes = 0;
  size_t off = 0;
  bool host = false;
};

template <class T>
Out plan_out(Carve& cv, T* user, size_t n) {
  Out o;
  o.user = user;
  o.bytes = n * sizeof(T);
  o.host = user && !is_device_ptr(user);
  if (o.host) o.off = cv.take<T>(n);
  return o;
}

void bind_out(Out& o, void* base) { o.dev = o.host ? at<void>(base, o.off) : o.user; }

cudaError_t copy_back(const Out& o, cudaStream_t s) {
  if (!o.host || !o.user) return cudaSuccess;
  return cudaMemcpyAsync(o.user, o.dev, o.bytes, cudaMemcpyDeviceToHost, s);
}

}  // namespace


wln_status check_batch(wln_ctx* ctx, const wln_profile* profiles, int32_t n_profiles,
                       const double* rho_cm, const int32_t* rho_off, const double* T,
                       const int32_t* T_off) {
  if (n_profiles < 1 || !profiles || !rho_cm || !rho_off || !T || !T_off)
    return fail(ctx, WLN_EINVAL, "profiles, grids and offsets are required");
  if (rho_off[0] != 0 || T_off[0] != 0) return fail(ctx, WLN_EINVAL, "offsets must start at 0");
  for (int q = 0; q < n_profiles; ++q) {
    const wln_profile& pr = profiles[q];
    if (pr.kind != WLN_PROFILE_FLUX_TUBE && pr.kind != WLN_PROFILE_CONST_B)
      return fail(ctx, WLN_EINVAL, "unknown profile kind");
    if (pr.kind == WLN_PROFILE_FLUX_TUBE && !(pr.lambda > 0.0 && std::isfinite(pr.lambda) && std::isfinite(pr.F)))
      return fail(ctx, WLN_EINVAL, "flux tube needs finite F and lambda > 0");
    if (pr.kind == WLN_PROFILE_CONST_B && !std::isfinite(pr.B))
      return fail(ctx, WLN_EINVAL, "constant field needs finite B");
    if (rho_off[q + 1] <= rho_off[q] || T_off[q + 1] <= T_off[q])
      return fail(ctx, WLN_EINVAL, "every profile needs at least one rho and one T");
    for (int i = rho_off[q]; i < rho_off[q + 1]; ++i)
      if (!(rho_cm[i] >= 0.0 && std::isfinite(rho_cm[i]))) return fail(ctx, WLN_EINVAL, "rho_cm must be finite and >= 0");
    for (int i = T_off[q]; i < T_off[q + 1]; ++i)
      if (!(T[i] > 0.0 && std::isfinite(T[i]))) return fail(ctx, WLN_EINVAL, "T must be finite and > 0");
  }
  return WLN_OK;
}

namespace {

// Mapped-grid node i of n: scale (1/x_i - 1), x_i = x0 (n - i)/n.
double mapped_node(int i, int n, double scale, double start, double* x0_out) {
  const double x0 = 1.0 / (1.0 + start / scale);
  if (x0_out) *x0_out = x0;
  if (i == 0) return start;
  const double x = x0 * static_cast<double>(n - i) / n;
  return scale * (1.0 / x - 1.0);
}

bool check_mapped(const double* v, int n, double scale, const char* what, std::string* why) {
  if (!(scale > 0.0 && std::isfinite(scale))) {
    if (why) *why = std::string(what) + ": mapped grid needs a finite scale > 0";
    return false;
  }
  for (int i = 1; i < n; ++i) {
    const double want = mapped_node(i, n, scale, v[0], nullptr);
    if (std::fabs(v[i] - want) > 1e-9 * std::fabs(want)) {
      if (why) *why = std::string(what) + " do not follow the mapped grid (wln_mapped_grid)";
      return false;
    }
  }
  return true;
}

}  // namespace

bool build_quad(const wln_profile* profiles, int32_t n_profiles, const double* rho_cm,
                const int32_t* rho_off, const double* T, const int32_t* T_off,
                std::vector<QuadProfile>& qp, std::string* why, const wln_quad* quad) {
  qp.assign(n_profiles, QuadProfile{});
  int64_t base = 0;
  for (int q = 0; q < n_profiles; ++q) {
    const int nr = rho_off[q + 1] - rho_off[q], nt = T_off[q + 1] - T_off[q];
    const double* r = rho_cm + rho_off[q];
    const double* t = T + T_off[q];
    QuadProfile& x = qp[q];
    x.kind = profiles[q].kind;
    x.n_rho = nr; x.n_T = nt; x.rho_base = rho_off[q]; x.T_base = T_off[q];
    x.p0 = base;
    if (quad) {
      x.rho_kind = quad[q].rho_kind;
      x.T_kind = quad[q].T_kind;
      x.rho_scale = quad[q].rho_scale;
      x.T_scale = quad[q].T_scale;
      x.small_T = quad[q].small_T != 0;
      if ((x.rho_kind != WLN_GRID_LINEAR && x.rho_kind != WLN_GRID_MAPPED) ||
          (x.T_kind != WLN_GRID_LOG && x.T_kind != WLN_GRID_MAPPED)) {
        if (why) *why = "unknown grid kind (radii: LINEAR or MAPPED; times: LOG or MAPPED)";
        return false;
      }
    }
    if (x.rho_kind == WLN_GRID_LINEAR) {
      x.h_rho = nr > 1 ? (r[nr - 1] - r[0]) / (nr - 1) : 0.0;
      for (int i = 1; i < nr; ++i)
        if (std::fabs((r[i] - r[i - 1]) - x.h_rho) > 1e-9 * (std::fabs(x.h_rho) + std::fabs(r[i]))) {
          if (why) *why = "rho_cm must be evenly spaced";
          return false;
        }
    } else {
      if (!check_mapped(r, nr, x.rho_scale, "rho_cm", why)) return false;
      mapped_node(0, nr, x.rho_scale, r[0], &x.rho_x0);
    }
    if (x.T_kind == WLN_GRID_LOG) {
      x.h_u = nt > 1 ? std::log(t[nt - 1] / t[0]) / (nt - 1) : 0.0;
      for (int i = 1; i < nt; ++i)
        if (std::fabs(std::log(t[i] / t[i - 1]) - x.h_u) > 1e-9 * (std::fabs(x.h_u) + 1.0)) {
          if (why) *why = "T must be geometrically spaced";
          return false;
        }
    } else {
      if (!check_mapped(t, nt, x.T_scale, "T", why)) return false;
      mapped_node(0, nt, x.T_scale, t[0], &x.T_x0);
    }
    if (x.kind == WLN_PROFILE_FLUX_TUBE) {
      x.l2 = profiles[q].lambda * profiles[q].lambda;
      x.eB_scale = profiles[q].F * x.l2 / 3.14159265358979323846;   // 2 calF lambda^2
    } else {
      x.l2 = 1.0;
      x.eB_scale = profiles[q].B;
    }
    base += static_cast<int64_t>(nr) * nt;
  }
  return true;
}

ProfileDev profile_constants(const wln_profile& pr, int ppl) {
  const double pi = 3.14159265358979323846;
  ProfileDev pd{};
  pd.kind = pr.kind;
  if (pr.kind == WLN_PROFILE_FLUX_TUBE) {
    pd.l2 = pr.lambda * pr.lambda;
    pd.turns_per = pr.F / (4.0 * pi * pi);                        // calF / (2 pi)
    pd.spin_per = (pr.F / (2.0 * pi)) * pd.l2 / ppl;               // calF lambda^2 / N
  } else {
    pd.l2 = 1.0;
    pd.turns_per = pr.B / (4.0 * pi);
    pd.spin_per = pr.B;
  }
  return pd;
}

void build_batch(const wln_profile* profiles, int32_t n_profiles, const double* rho_cm,
                 const int32_t* rho_off, const double* T, const int32_t* T_off, int ppl, int P,
                 Batch& bt) {
  bt.rho.assign(rho_cm, rho_cm + rho_off[n_profiles]);
  int64_t base = 0;
  for (int q = 0; q < n_profiles; ++q) {
    bt.profs.push_back(profile_constants(profiles[q], ppl));
    const int nr = rho_off[q + 1] - rho_off[q], nt = T_off[q + 1] - T_off[q];
    for (int it = 0; it < nt; ++it)
      for (int a = 0; a < nr; a += P) {
        Tile t{};
        t.profile = q;
        t.n_valid = nr - a < P ? nr - a : P;
        t.rho0 = rho_off[q] + a;
        t.p0 = static_cast<int32_t>(base + static_cast<int64_t>(it) * nr + a);
        t.T = T[T_off[q] + it];
        bt.tiles.push_back(t);
      }
    base += static_cast<int64_t>(nr) * nt;
  }
  bt.n_points = base;
  for (Tile& t : bt.tiles) {
    t.part_base = 0;
    t.part_stride = static_cast<int32_t>(base);
  }
}

}  // namespace wln

using namespace wln;

extern "C" {

wln_status wln_create(wln_ctx** out, int device, void* cuda_stream) {
  if (!out) return WLN_EINVAL;
  *out = nullptr;
  int n = 0;
  cudaError_t err = cudaGetDeviceCount(&n);
  if (err != cudaSuccess || n == 0) {
    (void)cudaGetLastError();
    return WLN_ECUDA;
  }
  if (device < 0 || device >= n) return WLN_EINVAL;
  wln_ctx* ctx = new (std::nothrow) wln_ctx();
  if (!ctx) return WLN_ENOMEM;
  DeviceGuard guard(device);
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  // the device error flag and the precision guard's running totals
  err = cudaMalloc(&ctx->d_flag, 64);
  if (err == cudaSuccess) err = cudaMemset(ctx->d_flag, 0, 64);
  if (err == cudaSuccess) {
    ctx->d_guard_totals = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(ctx->d_flag) + 8);
    ctx->d_items = reinterpret_cast<int*>(reinterpret_cast<char*>(ctx->d_flag) + 48);
  }
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&ctx->staging_done, cudaEventDisableTiming);
  if (err != cudaSuccess) {
    (void)cudaGetLastError();
    if (ctx->d_flag) cudaFree(ctx->d_flag);
    delete ctx;
    return WLN_ECUDA;
  }
  *out = ctx;
  return WLN_OK;
}

wln_status wln_destroy(wln_ctx* ctx) {
  if (!ctx) return WLN_EINVAL;
  DeviceGuard guard(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (const wln_ctx::EnsembleMem& m : ctx->ens_cache) {
    cudaFree(m.blocks);
    cudaFree(m.stats);
    if (m.xy64) cudaFree(m.xy64);
  }
  if (ctx->scratch.ptr) cudaFree(ctx->scratch.ptr);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->d_flag) cudaFree(ctx->d_flag);
  if (ctx->staging_done) cudaEventDestroy(ctx->staging_done);
  delete ctx;
  return WLN_OK;
}

wln_status wln_set_stream(wln_ctx* ctx, void* cuda_stream) {
  if (!ctx) return WLN_EINVAL;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return WLN_OK;
}

wln_status wln_synchronize(wln_ctx* ctx) {
  if (!ctx) return WLN_EINVAL;
  DeviceGuard guard(ctx->device);
  return check_flag(ctx);
}

const char* wln_last_error(const wln_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

int64_t wln_launch_count(const wln_ctx* ctx) { return ctx ? ctx->launches : 0; }

wln_status wln_selftest_wait(wln_ctx* ctx, int32_t timeout_ms) {
  if (!ctx) return WLN_EINVAL;
  if (timeout_ms < 1 || timeout_ms > 2000)
    return fail(ctx, WLN_EINVAL, "timeout_ms must be in [1, 2000]");
  DeviceGuard guard(ctx->device);
  cudaError_t err = launch_selftest_wait(ctx->stream, ctx->d_flag,
                                         static_cast<uint64_t>(timeout_ms) * 1000000ull);
  ++ctx->launches;
  if (err != cudaSuccess) return cuda_fail(ctx, err, "self-test launch");
  return check_flag(ctx);
}

wln_status wln_set_precision_guard(wln_ctx* ctx, int32_t enabled) {
  if (!ctx) return WLN_EINVAL;
  if (enabled < 0 || enabled > 2) return fail(ctx, WLN_EINVAL, "precision guard: 0, 1 or 2");
  ctx->guard = enabled;
  return WLN_OK;
}

wln_status wln_precision_guard_stats(wln_ctx* ctx, int64_t* escalated_loops, int64_t* launches,
                                     int64_t* overflows, int64_t* saturated, int32_t reset) {
  if (!ctx) return WLN_EINVAL;
  DeviceGuard guard(ctx->device);
  unsigned long long h[4] = {0, 0, 0, 0};
  cudaError_t err = cudaMemcpyAsync(h, ctx->d_guard_totals, sizeof(h), cudaMemcpyDeviceToHost,
                                    ctx->stream);
  if (err == cudaSuccess && reset)
    err = cudaMemsetAsync(ctx->d_guard_totals, 0, sizeof(h), ctx->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
  if (err != cudaSuccess) return cuda_fail(ctx, err, "precision guard statistics");
  if (escalated_loops) *escalated_loops = static_cast<int64_t>(h[0]);
  if (overflows) *overflows = static_cast<int64_t>(h[1]);
  if (saturated) *saturated = static_cast<int64_t>(h[2]);
  if (launches) *launches = static_cast<int64_t>(h[3]);
  return WLN_OK;
}

wln_status wln_gen_loops(wln_ctx* ctx, uint64_t seed, int64_t loop0, int32_t n_loops,
                         int32_t ppl, int32_t keep_fp64, wln_ensemble** out) {
  if (!ctx || !out) return fail(ctx, WLN_EINVAL, "null argument");
  *out = nullptr;
  wln_status st = check_loops(ctx, n_loops, ppl);
  if (st != WLN_OK) return st;
  if (loop0 < 0 || loop0 + ((n_loops + 31) / 32) * 32 > (int64_t(1) << 32))
    return fail(ctx, WLN_EINVAL, "loop0 + n_loops must stay below 2^32 (the Philox counter word)");
  DeviceGuard guard(ctx->device);
  wln_ensemble* en = nullptr;
  if ((st = alloc_ensemble(ctx, n_loops, ppl, keep_fp64 != 0, &en)) != WLN_OK) return st;
  en->e.loop0 = loop0;
  Carve cv;
  const size_t o_deg = cv.take<int>(1);
  const size_t o_work = cv.take<char>(gen_loops_work_bytes(en->e.n_blocks, ppl));
  if ((st = ensure_scratch(ctx, cv.off)) != WLN_OK) { wln_free_ensemble(ctx, en); return st; }
  int* d_deg = at<int>(ctx->scratch.ptr, o_deg);
  cudaError_t err = cudaMemsetAsync(d_deg, 0, sizeof(int), ctx->stream);
  if (err == cudaSuccess)
    err = launch_gen_loops(ctx->stream, seed, en->e, at<char>(ctx->scratch.ptr, o_work), d_deg);
  ctx->launches += gen_loops_launches(en->e.n_blocks, ppl);
  if (err != cudaSuccess) {
    wln_free_ensemble(ctx, en);
    return cuda_fail(ctx, err, "launch loop generation");
  }
  return finish_ensemble(ctx, en, d_deg, out);
}

wln_status wln_gen_dloops(wln_ctx* ctx, uint64_t seed, int64_t loop0, int32_t n_loops,
                          int32_t ppl, int32_t keep_fp64, wln_ensemble** out) {
  if (!ctx || !out) return fail(ctx, WLN_EINVAL, "null argument");
  *out = nullptr;
  wln_status st = check_loops(ctx, n_loops, ppl);
  if (st != WLN_OK) return st;
  if (loop0 < 0 || loop0 + ((n_loops + 31) / 32) * 32 > (int64_t(1) << 32))
    return fail(ctx, WLN_EINVAL, "loop0 + n_loops must stay below 2^32 (the Philox counter word)");
  DeviceGuard guard(ctx->device);
  wln_ensemble* en = nullptr;
  if ((st = alloc_ensemble(ctx, n_loops, ppl, keep_fp64 != 0, &en)) != WLN_OK) return st;
  en->e.loop0 = loop0;
  Carve cv;
  const size_t o_deg = cv.take<int>(1);
  const size_t o_work = cv.take<char>(gen_dloops_work_bytes(en->e.n_blocks, ppl));
  if ((st = ensure_scratch(ctx, cv.off)) != WLN_OK) { wln_free_ensemble(ctx, en); return st; }
  int* d_deg = at<int>(ctx->scratch.ptr, o_deg);
  cudaError_t err = cudaMemsetAsync(d_deg, 0, sizeof(int), ctx->stream);
  if (err == cudaSuccess)
    err = launch_gen_dloops(ctx->stream, seed, en->e, at<char>(ctx->scratch.ptr, o_work), d_deg);
  ctx->launches += gen_dloops_launches(en->e.n_blocks, ppl);
  if (err != cudaSuccess) {
    wln_free_ensemble(ctx, en);
    return cuda_fail(ctx, err, "launch d-loop generation");
  }
  return finish_ensemble(ctx, en, d_deg, out);
}

wln_status wln_ensemble_from_host(wln_ctx* ctx, const float* xy, int32_t n_loops, int32_t ppl,
                                  wln_ensemble** out) {
  if (!ctx || !out || !xy) return fail(ctx, WLN_EINVAL, "null argument");
  *out = nullptr;
  wln_status st = check_loops(ctx, n_loops, ppl);
  if (st != WLN_OK) return st;
  DeviceGuard guard(ctx->device);
  wln_ensemble* en = nullptr;
  if ((st = alloc_ensemble(ctx, n_loops, ppl, false, &en)) != WLN_OK) return st;
  const size_t n = static_cast<size_t>(n_loops) * 2 * ppl;
  const bool dev = is_device_ptr(xy);
  Carve cv;
  const size_t o_deg = cv.take<int>(1);
  const size_t o_xy = dev ? 0 : cv.take<float>(n);
  if ((st = ensure_scratch(ctx, cv.off)) != WLN_OK) { wln_free_ensemble(ctx, en); return st; }
  int* d_deg = at<int>(ctx->scratch.ptr, o_deg);
  const float* src = xy;
  cudaError_t err = cudaMemsetAsync(d_deg, 0, sizeof(int), ctx->stream);
  if (!dev && err == cudaSuccess) {
    float* d_xy = at<float>(ctx->scratch.ptr, o_xy);
    err = cudaMemcpyAsync(d_xy, xy, n * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    src = d_xy;
  }
  if (err == cudaSuccess) err = launch_pack_loops(ctx->stream, src, en->e, d_deg);
  ctx->launches += 4;   // pack, degeneracy check, block and sub-block statistics
  if (err != cudaSuccess) {
    wln_free_ensemble(ctx, en);
    return cuda_fail(ctx, err, "pack loops");
  }
  return finish_ensemble(ctx, en, d_deg, out);
}

wln_status wln_free_ensemble(wln_ctx* ctx, wln_ensemble* ens) {
  if (!ens) return fail(ctx, WLN_EINVAL, "null ensemble");
  DeviceGuard guard(ens->device);
  if (ctx) cudaStreamSynchronize(ctx->stream);
  if (ctx && ctx->device == ens->device && ens->e.blocks && ens->e.stats &&
      ctx->ens_cache.size() < kEnsembleCache) {
    // kept for the next ensemble of this shape (wln_destroy frees it)
    ctx->ens_cache.push_back(wln_ctx::EnsembleMem{
        ens->e.blocks, ens->e.stats, ens->e.xy64,
        static_cast<size_t>(ens->e.n_blocks) * (ens->e.ppl / 2) * 32,
        static_cast<size_t>(ens->e.n_blocks),
        ens->e.xy64 ? static_cast<size_t>(ens->e.n_loops) * 2 * ens->e.ppl : 0});
    delete ens;
    return WLN_OK;
  }
  if (ens->e.blocks) cudaFree(ens->e.blocks);
  if (ens->e.stats) cudaFree(ens->e.stats);
  if (ens->e.xy64) cudaFree(ens->e.xy64);
  delete ens;
  return WLN_OK;
}

wln_status wln_ensemble_info(const wln_ensemble* ens, int32_t* n_loops, int32_t* ppl,
                             int32_t* has_fp64) {
  if (!ens) return WLN_EINVAL;
  if (n_loops) *n_loops = ens->e.n_loops;
  if (ppl) *ppl = ens->e.ppl;
  if (has_fp64) *has_fp64 = ens->e.xy64 != nullptr;
  return WLN_OK;
}

wln_status wln_loops_copy(wln_ctx* ctx, const wln_ensemble* ens, float* xy_f32, double* xy_f64) {
  if (!ctx || !ens) return fail(ctx, WLN_EINVAL, "null argument");
  if (xy_f64 && !ens->e.xy64) return fail(ctx, WLN_EINVAL, "ensemble has no double copy");
  DeviceGuard guard(ctx->device);
  const size_t n = static_cast<size_t>(ens->e.n_loops) * 2 * ens->e.ppl;
  cudaError_t err = cudaSuccess;
  if (xy_f32) {
    Carve cv;
    Out o = plan_out(cv, xy_f32, n);
    wln_status st = ensure_scratch(ctx, cv.off + 256);
    if (st != WLN_OK) return st;
    bind_out(o, ctx->scratch.ptr);
    err = launch_unpack_loops(ctx->stream, ens->e, static_cast<float*>(o.dev));
    ++ctx->launches;
    if (err == cudaSuccess) err = copy_back(o, ctx->stream);
  }
  if (err == cudaSuccess && xy_f64)
    err = cudaMemcpyAsync(xy_f64, ens->e.xy64, n * sizeof(double), cudaMemcpyDefault, ctx->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
  if (err != cudaSuccess) return cuda_fail(ctx, err, "copy loops");
  return WLN_OK;
}

wln_status wln_philox_stream(wln_ctx* ctx, uint64_t seed, int64_t loop0, int32_t n_loops,
                             int32_t n_calls, uint32_t* out) {
  if (!ctx || !out || n_loops < 0 || n_calls < 0 || loop0 < 0 ||
      loop0 + n_loops > (int64_t(1) << 32))
    return fail(ctx, WLN_EINVAL, "bad Philox stream arguments");
  DeviceGuard guard(ctx->device);
  const size_t n = static_cast<size_t>(n_loops) * n_calls * 4;
  Carve cv;
  Out o = plan_out(cv, out, n);
  wln_status st = ensure_scratch(ctx, cv.off + 256);
  if (st != WLN_OK) return st;
  bind_out(o, ctx->scratch.ptr);
  cudaError_t err = launch_philox_stream(ctx->stream, seed, loop0, n_loops, n_calls,
                                         static_cast<uint32_t*>(o.dev));
  ++ctx->launches;
  if (err == cudaSuccess) err = copy_back(o, ctx->stream);
  if (err == cudaSuccess && o.host) err = cudaStreamSynchronize(ctx->stream);
  if (err != cudaSuccess) return cuda_fail(ctx, err, "Philox stream");
  return WLN_OK;
}

}  // extern "C"

namespace wln {
namespace {

// Group sums of one Wilson pass: the plain sums (WLN_K components) or the
// discretisation levels (WLN_KL components).
wln_status wilson_pass(wln_ctx* ctx, const wln_ensemble* ens, const wln_profile* profiles,
                       int32_t n_profiles, const double* rho_cm, const int32_t* rho_off,
                       const double* T, const int32_t* T_off, int32_t n_groups,
                       wln_prec prec, double* group_sums, int mode) {
  if (!ctx || !ens || !group_sums) return fail(ctx, WLN_EINVAL, "null argument");
  if (prec != WLN_PREC_FP64 && prec != WLN_PREC_FP32_COMP && prec != WLN_PREC_FP32_NAIVE)
    return fail(ctx, WLN_EINVAL, "unknown precision");
  if (ens->device != ctx->device) return fail(ctx, WLN_EINVAL, "ensemble lives on another device");
  const bool per_loop = mode == kModeLoops;
  if (per_loop) n_groups = 1;
  else if (n_groups < 2 || ens->e.n_loops % n_groups != 0)
    return fail(ctx, WLN_EINVAL, "n_groups must be >= 2 and divide n_loops");
  if (level_mode(mode) && (ens->e.ppl % 4 != 0 || ens->e.ppl < 8))
    return fail(ctx, WLN_EINVAL, "discretisation levels need ppl a multiple of 4 and >= 8");
  wln_status st = check_batch(ctx, profiles, n_profiles, rho_cm, rho_off, T, T_off);
  if (st != WLN_OK) return st;
  DeviceGuard guard(ctx->device);
  const int K = level_mode(mode) ? WLN_KL : WLN_K;

  Batch bt;
  const int P = plan_points_per_lane(ctx, prec, mode);
  build_batch(profiles, n_profiles, rho_cm, rho_off, T, T_off, ens->e.ppl, P, bt);
  if (bt.n_points > (int64_t(1) << 31) - 1) return fail(ctx, WLN_EINVAL, "too many points");
  // the precision guard runs where some point's spin can reach its floor; its
  // queue first gets kGuardPerPair entries per such (point, group)
  const int64_t guard_pts =
      guard_applies(ctx, prec, mode, ens->e.n_loops, n_groups, profiles, n_profiles)
          ? guard_points(profiles, n_profiles, rho_cm, rho_off, T, T_off, ens->e)
          : 0;
  const bool use_guard = guard_pts > 0;
  const int bpg = guard_layout_bpg(prec, mode, ens->e.n_loops, n_groups);
  const WilsonPlan plan =
      make_plan(ctx, ens->e, static_cast<int>(bt.tiles.size()), prec, mode, bpg);
  // A queue of kGuardSel entries per such (point, group) holds anything a
  // pass can select; up to 2^22 entries (192 MiB) the call takes that and need
  // not wait.  Otherwise a launch whose guard selected more loops than the
  // queue holds is run again with the queue sized to exactly what it
  // selected (the selection depends only on the float walk, so the second
  // launch selects the same loops).
  const int64_t worst = use_guard ? guard_capacity(guard_pts, n_groups, kGuardSel) : 0;
  int64_t gcap = worst <= (int64_t(1) << 22) ? worst
                                              : guard_capacity(guard_pts, n_groups, kGuardPerPair);
  for (int attempt = 0;; ++attempt) {
    // Device layout of this call: work list | profiles | radii | partials |
    // (precision guard: per-warp records, queue, counters) | (host output)
    Carve cv;
    const size_t o_tiles = cv.take<Tile>(bt.tiles.size());
    const size_t o_profs = cv.take<ProfileDev>(bt.profs.size());
    const size_t o_rho = cv.take<double>(bt.rho.size());
    const size_t upload = cv.off;
    const size_t n_partial =
        per_loop ? 0 : static_cast<size_t>(plan.n_chains + n_groups) * bt.n_points * K;
    const size_t o_part = cv.take<double>(n_partial);
    GuardBufs gb;
    size_t o_gscr = 0, o_gq = 0, o_gcnt = 0;
    if (use_guard) {
      gb.on = 1;
      gb.bpg = bpg;
      gb.warp_bytes = guard_warp_bytes(bpg, plan.P);
      o_gscr = cv.take<char>(static_cast<size_t>(wilson_grid(plan, ens->e, prec)) * plan.warps *
                             gb.warp_bytes);
      o_gq = cv.take<char>(guard_queue_bytes(gcap));
      o_gcnt = cv.take<int>(4);
    }
    const size_t n_out = per_loop ? static_cast<size_t>(bt.n_points) * ens->e.n_loops * 2
                                  : static_cast<size_t>(bt.n_points) * n_groups * K;
    Out out = plan_out(cv, group_sums, n_out);
    if ((st = ensure_scratch(ctx, cv.off)) != WLN_OK) return st;
    if ((st = ensure_pinned(ctx, upload)) != WLN_OK) return st;
    bind_out(out, ctx->scratch.ptr);

    char* h = static_cast<char*>(ctx->pinned);
    std::memcpy(h + o_tiles, bt.tiles.data(), bt.tiles.size() * sizeof(Tile));
    std::memcpy(h + o_profs, bt.profs.data(), bt.profs.size() * sizeof(ProfileDev));
    std::memcpy(h + o_rho, bt.rho.data(), bt.rho.size() * sizeof(double));
    char* d = static_cast<char*>(ctx->scratch.ptr);
    cudaError_t err = cudaMemcpyAsync(d, h, upload, cudaMemcpyHostToDevice, ctx->stream);
    if (err == cudaSuccess) err = cudaEventRecord(ctx->staging_done, ctx->stream);
    if (err != cudaSuccess) return cuda_fail(ctx, err, "upload work list");

    int64_t launches = 0;
    if (per_loop) {
      err = launch_wilson_loops(ctx->stream, plan, ens->e, at<Tile>(d, o_tiles),
                                at<ProfileDev>(d, o_profs), at<double>(d, o_rho), prec,
                                static_cast<double*>(out.dev), ctx->d_flag, &launches, ctx->d_items);
      ctx->launches += launches;
      if (err != cudaSuccess) return cuda_fail(ctx, err, "Wilson kernel");
    } else {
      const int32_t lpg = ens->e.n_loops / n_groups;
      if (use_guard) {
        guard_bind(gb, d + o_gscr, d + o_gq, gcap, at<int>(d, o_gcnt));
        guard_attach(gb, ctx);
        err = cudaMemsetAsync(gb.counters, 0, 4 * sizeof(int), ctx->stream);
        if (err != cudaSuccess) return cuda_fail(ctx, err, "precision guard counters");
      }
      err = launch_wilson(ctx->stream, plan, ens->e, at<Tile>(d, o_tiles),
                          at<ProfileDev>(d, o_profs), at<double>(d, o_rho), n_groups, lpg, prec,
                          at<double>(d, o_part), bt.n_points, ctx->d_flag, &launches,
                          use_guard ? &gb : nullptr, ctx->d_items);
      if (err != cudaSuccess) return cuda_fail(ctx, err, "Wilson kernel");
      if (use_guard && gcap < worst) {
        // the loops the float pass selected (the call waits for it here)
        int selected = 0;
        err = cudaMemcpyAsync(&selected, gb.counters, sizeof(int), cudaMemcpyDeviceToHost,
                              ctx->stream);
        if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
        if (err != cudaSuccess) return cuda_fail(ctx, err, "precision guard queue");
        if (selected > gcap && attempt == 0) {
          ctx->launches += launches;
          gcap = selected;
          continue;
        }
      }
      if (use_guard) {
        err = launch_guard(ctx->stream, gb, ens->e, at<Tile>(d, o_tiles),
                           at<ProfileDev>(d, o_profs), at<double>(d, o_rho), at<double>(d, o_part),
                           ctx->num_sms, &launches);
        if (err != cudaSuccess) return cuda_fail(ctx, err, "precision guard");
      }
      err = launch_reduce_partials(ctx->stream, plan, ens->e, at<double>(d, o_part), bt.n_points,
                                   n_groups, lpg, static_cast<double*>(out.dev));
      ++launches;
      ctx->launches += launches;
      if (err != cudaSuccess) return cuda_fail(ctx, err, "group reduction");
    }
    if (out.host) {
      if ((err = copy_back(out, ctx->stream)) != cudaSuccess) return cuda_fail(ctx, err, "copy results");
      return check_flag(ctx);
    }
    return WLN_OK;
  }
}

}  // namespace
}  // namespace wln

extern "C" {

wln_status wln_wilson_avg(wln_ctx* ctx, const wln_ensemble* ens, const wln_profile* profiles,
                          int32_t n_profiles, const double* rho_cm, const int32_t* rho_off,
                          const double* T, const int32_t* T_off, int32_t n_groups,
                          wln_prec prec, double* group_sums) {
  return wilson_pass(ctx, ens, profiles, n_profiles, rho_cm, rho_off, T, T_off, n_groups, prec,
                     group_sums, kModeSums);
}

wln_status wln_wilson_levels(wln_ctx* ctx, const wln_ensemble* ens, const wln_profile* profiles,
                             int32_t n_profiles, const double* rho_cm, const int32_t* rho_off,
                             const double* T, const int32_t* T_off, int32_t n_groups,
                             wln_prec prec, double* group_sums) {
  return wilson_pass(ctx, ens, profiles, n_profiles, rho_cm, rho_off, T, T_off, n_groups, prec,
                     group_sums, kModeLevels);
}

wln_status wln_wilson_levels_nested(wln_ctx* ctx, const wln_ensemble* ens,
                                    const wln_profile* profiles, int32_t n_profiles,
                                    const double* rho_cm, const int32_t* rho_off, const double* T,
                                    const int32_t* T_off, int32_t n_groups, wln_prec prec,
                                    double* group_sums) {
  return wilson_pass(ctx, ens, profiles, n_profiles, rho_cm, rho_off, T, T_off, n_groups, prec,
                     group_sums, kModeNested);
}

wln_status wln_wilson_loops(wln_ctx* ctx, const wln_ensemble* ens, const wln_profile* profiles,
                            int32_t n_profiles, const double* rho_cm, const int32_t* rho_off,
                            const double* T, const int32_t* T_off, wln_prec prec,
                            double* loop_values) {
  return wilson_pass(ctx, ens, profiles, n_profiles, rho_cm, rho_off, T, T_off, 0, prec,
                     loop_values, kModeLoops);
}

wln_status wln_group_sums_loops(wln_ctx* ctx, const double* loop_values, int64_t n_points,
                                int32_t n_loops, int32_t n_groups, int32_t shuffle, uint64_t seed,
                                double* group_sums, int32_t* perm) {
  if (!ctx || !loop_values || !group_sums) return fail(ctx, WLN_EINVAL, "null argument");
  if (n_points < 1 || n_loops < 1 || n_groups < 2 || n_loops % n_groups != 0)
    return fail(ctx, WLN_EINVAL, "n_groups must be >= 2 and divide n_loops");
  if (n_points > (int64_t(1) << 32)) return fail(ctx, WLN_EINVAL, "too many points");
  DeviceGuard guard(ctx->device);
  const size_t nW = static_cast<size_t>(n_points) * n_loops * 2;
  const bool w_dev = is_device_ptr(loop_values);
  Carve cv;
  const size_t o_W = w_dev ? 0 : cv.take<double>(nW);
  const bool need_perm = shuffle != 0;
  const size_t o_perm = need_perm && !perm ? cv.take<int32_t>(static_cast<size_t>(n_points) * n_loops) : 0;
  Out os = plan_out(cv, group_sums, static_cast<size_t>(n_points) * n_groups * WLN_K);
  Out op = plan_out(cv, need_perm ? perm : static_cast<int32_t*>(nullptr),
                    static_cast<size_t>(n_points) * n_loops);
  wln_status st = ensure_scratch(ctx, cv.off + 256);
  if (st != WLN_OK) return st;
  bind_out(os, ctx->scratch.ptr);
  bind_out(op, ctx->scratch.ptr);
  const double* W = loop_values;
  cudaError_t err = cudaSuccess;
  if (!w_dev) {
    double* dW = at<double>(ctx->scratch.ptr, o_W);
    err = cudaMemcpyAsync(dW, loop_values, nW * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    W = dW;
  }
  int32_t* dperm = nullptr;
  if (need_perm) dperm = perm ? static_cast<int32_t*>(op.dev) : at<int32_t>(ctx->scratch.ptr, o_perm);
  int64_t launches = 0;
  if (err == cudaSuccess)
    err = launch_group_sums_loops(ctx->stream, W, n_points, n_loops, n_groups, need_perm, seed,
                                  dperm, static_cast<double*>(os.dev), &launches);
  ctx->launches += launches;
  if (err == cudaSuccess) err = copy_back(os, ctx->stream);
  if (err == cudaSuccess && need_perm) err = copy_back(op, ctx->stream);
  if (err != cudaSuccess) return cuda_fail(ctx, err, "group sums of loop values");
  if (os.host || op.host || !w_dev) return check_flag(ctx);
  return WLN_OK;
}

wln_status wln_corrcoef(wln_ctx* ctx, const double* x, int32_t n_rows, int32_t n_samples,
                        int32_t stride, int32_t comp, int32_t ref, double* out) {
  if (!ctx || !x || !out) return fail(ctx, WLN_EINVAL, "null argument");
  if (n_rows < 1 || n_samples < 2 || stride < 1 || comp < 0 || comp >= stride || ref < 0 ||
      ref >= n_rows)
    return fail(ctx, WLN_EINVAL, "bad correlation sizes");
  DeviceGuard guard(ctx->device);
  const size_t nX = static_cast<size_t>(n_rows) * n_samples * stride;
  const bool x_dev = is_device_ptr(x);
  Carve cv;
  const size_t o_X = x_dev ? 0 : cv.take<double>(nX);
  Out oo = plan_out(cv, out, static_cast<size_t>(n_rows));
  wln_status st = ensure_scratch(ctx, cv.off + 256);
  if (st != WLN_OK) return st;
  bind_out(oo, ctx->scratch.ptr);
  const double* X = x;
  cudaError_t err = cudaSuccess;
  if (!x_dev) {
    double* dX = at<double>(ctx->scratch.ptr, o_X);
    err = cudaMemcpyAsync(dX, x, nX * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    X = dX;
  }
  if (err == cudaSuccess)
    err = launch_corrcoef(ctx->stream, X, n_rows, n_samples, stride, comp, ref,
                          static_cast<double*>(oo.dev));
  ++ctx->launches;
  if (err == cudaSuccess) err = copy_back(oo, ctx->stream);
  if (err != cudaSuccess) return cuda_fail(ctx, err, "correlation coefficients");
  if (oo.host || !x_dev) return check_flag(ctx);
  return WLN_OK;
}

wln_status wln_extrapolate(wln_ctx* ctx, const double* level_sums, int32_t n_points,
                           int32_t n_groups, int32_t loops_per_group, double* out) {
  if (!ctx || !level_sums || !out) return fail(ctx, WLN_EINVAL, "null argument");
  if (n_points < 1 || n_groups < 2 || loops_per_group < 1)
    return fail(ctx, WLN_EINVAL, "bad extrapolation sizes");
  DeviceGuard guard(ctx->device);
  const size_t nS = static_cast<size_t>(n_points) * n_groups * WLN_KL;
  const bool s_dev = is_device_ptr(level_sums);
  Carve cv;
  const size_t o_S = s_dev ? 0 : cv.take<double>(nS);
  Out oo = plan_out(cv, out, static_cast<size_t>(n_points) * 12);
  wln_status st = ensure_scratch(ctx, cv.off + 256);
  if (st != WLN_OK) return st;
  bind_out(oo, ctx->scratch.ptr);
  const double* S = level_sums;
  cudaError_t err = cudaSuccess;
  if (!s_dev) {
    double* dS = at<double>(ctx->scratch.ptr, o_S);
    err = cudaMemcpyAsync(dS, level_sums, nS * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    S = dS;
  }
  if (err == cudaSuccess)
    err = launch_extrapolate(ctx->stream, S, n_points, n_groups, loops_per_group,
                             static_cast<double*>(oo.dev));
  ++ctx->launches;
  if (err == cudaSuccess) err = copy_back(oo, ctx->stream);
  if (err != cudaSuccess) return cuda_fail(ctx, err, "extrapolation");
  if (oo.host || !s_dev) return check_flag(ctx);
  return WLN_OK;
}

}  // extern "C"

namespace wln {
namespace {
wln_status jackknife_impl(wln_ctx* ctx, const double* group_sums, int32_t n_points,
                          int32_t n_groups, int32_t loops_per_group, int32_t comp, double* mean,
                          double* sem, double* jk_var, double* cov, bool packed) {
  if (!ctx || !group_sums || !mean || !sem) return fail(ctx, WLN_EINVAL, "null argument");
  if (n_points < 1 || n_groups < 2 || loops_per_group < 1 || comp < 0 || comp >= WLN_K)
    return fail(ctx, WLN_EINVAL, "bad jackknife sizes");
  if (cov && static_cast<int64_t>(n_points) * n_points > (int64_t(1) << 33))
    return fail(ctx, WLN_EINVAL, "covariance too large");
  DeviceGuard guard(ctx->device);
  const size_t nS = static_cast<size_t>(n_points) * n_groups * WLN_K;
  const bool s_dev = is_device_ptr(group_sums);
  Carve cv;
  const size_t o_S = s_dev ? 0 : cv.take<double>(nS);
  const size_t o_dev = cov ? cv.take<double>(static_cast<size_t>(n_groups) * n_points) : 0;
  Out om = plan_out(cv, mean, n_points), os = plan_out(cv, sem, n_points);
  Out oj = plan_out(cv, jk_var, n_points);
  const size_t n_cov = !cov ? 0
                      : packed ? static_cast<size_t>(n_points) * (n_points + 1) / 2
                               : static_cast<size_t>(n_points) * n_points;
  Out oc = plan_out(cv, cov, n_cov);
  wln_status st = ensure_scratch(ctx, cv.off + 256);
  if (st != WLN_OK) return st;
  bind_out(om, ctx->scratch.ptr); bind_out(os, ctx->scratch.ptr);
  bind_out(oj, ctx->scratch.ptr); bind_out(oc, ctx->scratch.ptr);
  const double* S = group_sums;
  cudaError_t err = cudaSuccess;
  if (!s_dev) {
    double* dS = at<double>(ctx->scratch.ptr, o_S);
    err = cudaMemcpyAsync(dS, group_sums, nS * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    S = dS;
  }
  int64_t launches = 0;
  if (err == cudaSuccess)
    err = launch_jackknife(ctx->stream, S, n_points, n_groups, loops_per_group, comp,
                           static_cast<double*>(om.dev), static_cast<double*>(os.dev),
                           static_cast<double*>(oj.dev),
                           cov ? at<double>(ctx->scratch.ptr, o_dev) : nullptr,
                           static_cast<double*>(oc.dev), &launches, packed);
  ctx->launches += launches;
  for (const Out* o : {&om, &os, &oj, &oc})
    if (err == cudaSuccess) err = copy_back(*o, ctx->stream);
  if (err != cudaSuccess) return cuda_fail(ctx, err, "jackknife");
  if (om.host || os.host || oj.host || oc.host || !s_dev) return check_flag(ctx);
  return WLN_OK;
}
}  // namespace
}  // namespace wln

extern "C" {

wln_status wln_jackknife(wln_ctx* ctx, const double* group_sums, int32_t n_points,
                         int32_t n_groups, int32_t loops_per_group, int32_t comp, double* mean,
                         double* sem, double* jk_var, double* cov) {
  return wln::jackknife_impl(ctx, group_sums, n_points, n_groups, loops_per_group, comp, mean,
                             sem, jk_var, cov, false);
}

wln_status wln_jackknife_packed(wln_ctx* ctx, const double* group_sums, int32_t n_points,
                                int32_t n_groups, int32_t loops_per_group, int32_t comp,
                                double* mean, double* sem, double* jk_var, double* cov_packed) {
  return wln::jackknife_impl(ctx, group_sums, n_points, n_groups, loops_per_group, comp, mean,
                             sem, jk_var, cov_packed, true);
}

wln_status wln_loop_sem(wln_ctx* ctx, const double* group_sums, int32_t n_points,
                        int32_t n_groups, int32_t n_loops, int32_t comp_sum, int32_t comp_sq,
                        double* out) {
  if (!ctx || !group_sums || !out) return fail(ctx, WLN_EINVAL, "null argument");
  if (n_points < 1 || n_groups < 1 || n_loops < 2 || comp_sum < 0 || comp_sum >= WLN_K ||
      comp_sq < 0 || comp_sq >= WLN_K)
    return fail(ctx, WLN_EINVAL, "bad loop-SEM sizes");
  DeviceGuard guard(ctx->device);
  const size_t nS = static_cast<size_t>(n_points) * n_groups * WLN_K;
  const bool s_dev = is_device_ptr(group_sums);
  Carve cv;
  const size_t o_S = s_dev ? 0 : cv.take<double>(nS);
  Out o = plan_out(cv, out, n_points);
  wln_status st = ensure_scratch(ctx, cv.off + 256);
  if (st != WLN_OK) return st;
  bind_out(o, ctx->scratch.ptr);
  const double* S = group_sums;
  cudaError_t err = cudaSuccess;
  if (!s_dev) {
    double* dS = at<double>(ctx->scratch.ptr, o_S);
    err = cudaMemcpyAsync(dS, group_sums, nS * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    S = dS;
  }
  if (err == cudaSuccess)
    err = launch_loop_sem(ctx->stream, S, n_points, n_groups, n_loops, comp_sum, comp_sq,
                          static_cast<double*>(o.dev));
  ++ctx->launches;
  if (err == cudaSuccess) err = copy_back(o, ctx->stream);
  if (err != cudaSuccess) return cuda_fail(ctx, err, "loop SEM");
  if (o.host || !s_dev) return check_flag(ctx);
  return WLN_OK;
}

wln_status wln_effective_action(wln_ctx* ctx, const wln_profile* profiles, int32_t n_profiles,
                                const double* rho_cm, const int32_t* rho_off, const double* T,
                                const int32_t* T_off, const double* group_sums, int32_t n_groups,
                                int32_t loops_per_group, int32_t spinor, double* gamma_groups,
                                double* gamma_mean_sem) {
  if (!ctx || !group_sums || !gamma_mean_sem) return fail(ctx, WLN_EINVAL, "null argument");
  if (n_groups < 2 || loops_per_group < 1) return fail(ctx, WLN_EINVAL, "bad group sizes");
  wln_status st = check_batch(ctx, profiles, n_profiles, rho_cm, rho_off, T, T_off);
  if (st != WLN_OK) return st;
  std::vector<QuadProfile> qp;
  std::string why;
  if (!build_quad(profiles, n_profiles, rho_cm, rho_off, T, T_off, qp, &why))
    return fail(ctx, WLN_EINVAL, why);
  const int64_t base = qp.back().p0 + static_cast<int64_t>(qp.back().n_rho) * qp.back().n_T;
  DeviceGuard guard(ctx->device);
  const size_t nS = static_cast<size_t>(base) * n_groups * WLN_K;
  const bool s_dev = is_device_ptr(group_sums);
  Carve cv;
  const size_t o_qp = cv.take<QuadProfile>(qp.size());
  const size_t o_r = cv.take<double>(rho_off[n_profiles]);
  const size_t o_t = cv.take<double>(T_off[n_profiles]);
  const size_t upload = cv.off;
  const size_t o_S = s_dev ? 0 : cv.take<double>(nS);
  const size_t o_gg = cv.take<double>(static_cast<size_t>(n_profiles) * n_groups);
  Out og = plan_out(cv, gamma_groups, static_cast<size_t>(n_profiles) * n_groups);
  Out om = plan_out(cv, gamma_mean_sem, static_cast<size_t>(n_profiles) * 2);
  if ((st = ensure_scratch(ctx, cv.off + 256)) != WLN_OK) return st;
  if ((st = ensure_pinned(ctx, upload)) != WLN_OK) return st;
  bind_out(og, ctx->scratch.ptr);
  bind_out(om, ctx->scratch.ptr);
  char* h = static_cast<char*>(ctx->pinned);
  std::memcpy(h + o_qp, qp.data(), qp.size() * sizeof(QuadProfile));
  std::memcpy(h + o_r, rho_cm, rho_off[n_profiles] * sizeof(double));
  std::memcpy(h + o_t, T, T_off[n_profiles] * sizeof(double));
  char* d = static_cast<char*>(ctx->scratch.ptr);
  cudaError_t err = cudaMemcpyAsync(d, h, upload, cudaMemcpyHostToDevice, ctx->stream);
  if (err == cudaSuccess) err = cudaEventRecord(ctx->staging_done, ctx->stream);
  const double* S = group_sums;
  if (err == cudaSuccess && !s_dev) {
    err = cudaMemcpyAsync(d + o_S, group_sums, nS * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    S = at<double>(d, o_S);
  }
  double* gg = gamma_groups ? static_cast<double*>(og.dev) : at<double>(d, o_gg);
  int64_t launches = 0;
  if (err == cudaSuccess)
    err = launch_effective_action(ctx->stream, at<QuadProfile>(d, o_qp), n_profiles,
                                  at<double>(d, o_r), at<double>(d, o_t), S, n_groups,
                                  loops_per_group, spinor, gg, static_cast<double*>(om.dev),
                                  &launches);
  ctx->launches += launches;
  if (err == cudaSuccess) err = copy_back(og, ctx->stream);
  if (err == cudaSuccess) err = copy_back(om, ctx->stream);
  if (err != cudaSuccess) return cuda_fail(ctx, err, "effective action");
  if (og.host || om.host || !s_dev) return check_flag(ctx);
  return WLN_OK;
}

wln_status wln_mapped_grid(int32_t n, double scale, double start, double* out) {
  if (n < 1 || !out || !(scale > 0.0 && std::isfinite(scale)) || !(start >= 0.0 && std::isfinite(start)))
    return WLN_EINVAL;
  for (int i = 0; i < n; ++i) out[i] = mapped_node(i, n, scale, start, nullptr);
  return WLN_OK;
}

wln_status wln_effective_action_full(wln_ctx* ctx, const wln_profile* profiles, int32_t n_profiles,
                                     const double* rho_cm, const int32_t* rho_off, const double* T,
                                     const int32_t* T_off, const wln_quad* quad,
                                     const double* group_sums, int32_t n_groups,
                                     int32_t loops_per_group, int32_t spinor, double* gamma_groups,
                                     double* gamma, double* density, double* integrand) {
  if (!ctx || !group_sums || !gamma) return fail(ctx, WLN_EINVAL, "null argument");
  if (n_groups < 2 || loops_per_group < 1) return fail(ctx, WLN_EINVAL, "bad group sizes");
  wln_status st = check_batch(ctx, profiles, n_profiles, rho_cm, rho_off, T, T_off);
  if (st != WLN_OK) return st;
  std::vector<QuadProfile> qp;
  std::string why;
  if (!build_quad(profiles, n_profiles, rho_cm, rho_off, T, T_off, qp, &why, quad))
    return fail(ctx, WLN_EINVAL, why);
  const int64_t n_points = qp.back().p0 + static_cast<int64_t>(qp.back().n_rho) * qp.back().n_T;
  const int32_t n_rho_total = rho_off[n_profiles];
  int32_t max_rho = 0;
  std::vector<int32_t> point_profile(static_cast<size_t>(n_points));
  for (int q = 0; q < n_profiles; ++q) {
    max_rho = std::max(max_rho, qp[q].n_rho);
    for (int64_t p = 0; p < static_cast<int64_t>(qp[q].n_rho) * qp[q].n_T; ++p)
      point_profile[static_cast<size_t>(qp[q].p0 + p)] = q;
  }
  DeviceGuard guard(ctx->device);
  const size_t nS = static_cast<size_t>(n_points) * n_groups * WLN_K;
  const bool s_dev = is_device_ptr(group_sums);
  Carve cv;
  const size_t o_qp = cv.take<QuadProfile>(qp.size());
  const size_t o_r = cv.take<double>(n_rho_total);
  const size_t o_t = cv.take<double>(T_off[n_profiles]);
  const size_t o_pp = cv.take<int32_t>(point_profile.size());
  const size_t upload = cv.off;
  const size_t o_S = s_dev ? 0 : cv.take<double>(nS);
  const size_t o_dg = cv.take<double>(static_cast<size_t>(n_rho_total) * n_groups);
  const size_t o_gg = cv.take<double>(static_cast<size_t>(n_profiles) * n_groups);
  const size_t o_den = cv.take<double>(static_cast<size_t>(n_rho_total) * 3);
  Out og = plan_out(cv, gamma_groups, static_cast<size_t>(n_profiles) * n_groups);
  Out om = plan_out(cv, gamma, static_cast<size_t>(n_profiles) * 3);
  Out od = plan_out(cv, density, static_cast<size_t>(n_rho_total) * 3);
  Out oi = plan_out(cv, integrand, static_cast<size_t>(n_points) * 3);
  if ((st = ensure_scratch(ctx, cv.off + 256)) != WLN_OK) return st;
  if ((st = ensure_pinned(ctx, upload)) != WLN_OK) return st;
  for (Out* o : {&og, &om, &od, &oi}) bind_out(*o, ctx->scratch.ptr);
  char* h = static_cast<char*>(ctx->pinned);
  std::memcpy(h + o_qp, qp.data(), qp.size() * sizeof(QuadProfile));
  std::memcpy(h + o_r, rho_cm, n_rho_total * sizeof(double));
  std::memcpy(h + o_t, T, T_off[n_profiles] * sizeof(double));
  std::memcpy(h + o_pp, point_profile.data(), point_profile.size() * sizeof(int32_t));
  char* d = static_cast<char*>(ctx->scratch.ptr);
  cudaError_t err = cudaMemcpyAsync(d, h, upload, cudaMemcpyHostToDevice, ctx->stream);
  if (err == cudaSuccess) err = cudaEventRecord(ctx->staging_done, ctx->stream);
  const double* S = group_sums;
  if (err == cudaSuccess && !s_dev) {
    err = cudaMemcpyAsync(d + o_S, group_sums, nS * sizeof(double), cudaMemcpyHostToDevice,
                          ctx->stream);
    S = at<double>(d, o_S);
  }
  int64_t launches = 0;
  if (err == cudaSuccess)
    err = launch_effective_action_full(
        ctx->stream, at<QuadProfile>(d, o_qp), n_profiles, max_rho, n_rho_total, n_points,
        at<int32_t>(d, o_pp), at<double>(d, o_r), at<double>(d, o_t), S, n_groups,
        loops_per_group, spinor, at<double>(d, o_dg),
        gamma_groups ? static_cast<double*>(og.dev) : at<double>(d, o_gg),
        static_cast<double*>(om.dev),
        density ? static_cast<double*>(od.dev) : at<double>(d, o_den),
        static_cast<double*>(oi.dev), &launches);
  ctx->launches += launches;
  for (const Out* o : {&og, &om, &od, &oi})
    if (err == cudaSuccess) err = copy_back(*o, ctx->stream);
  if (err != cudaSuccess) return cuda_fail(ctx, err, "full effective action");
  if (og.host || om.host || od.host || oi.host || !s_dev) return check_flag(ctx);
  return WLN_OK;
}

}  // extern "C"
