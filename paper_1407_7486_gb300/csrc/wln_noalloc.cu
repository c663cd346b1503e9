// wln_wilson_avg_noalloc: the Wilson group sums of wln_wilson_avg with every
// piece of working memory taken from one fixed array compiled into the
// library, so the call never allocates device (or pinned host) memory.
//
// Some callers cannot allocate: code that runs where the device memory is
// owned by another allocator (a framework's caching pool that forbids direct
// cudaMalloc), latency-bound loops that must not take cudaMalloc's implicit
// device synchronisation, and long-running services that have reserved all
// device memory up front.  They pass their inputs and outputs and the library
// works inside the array below.
//
// The array lives for as long as the library is loaded, on every GPU the
// process touches with it.  All calls share it: two calls whose GPU work
// overlaps in time (different streams, or different host threads) race on
// it.  The arithmetic is exactly that of wln_wilson_avg (same kernels, same
// work decomposition), so the results are identical.
#include <cmath>

#include "wln_internal.cuh"

namespace wln {
namespace {

constexpr size_t kNoAllocBytes = size_t(64) << 20;   // 64 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch, looked up once per device.
void* g_scratch_addr[kMaxDevices] = {};

wln_status scratch_address(wln_ctx* ctx, void** out) {
  if (ctx->device < 0 || ctx->device >= kMaxDevices)
    return fail(ctx, WLN_EINVAL, "device index beyond the no-alloc table");
  if (!g_scratch_addr[ctx->device]) {
    void* p = nullptr;
    cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (err != cudaSuccess) return cuda_fail(ctx, err, "cudaGetSymbolAddress(no-alloc scratch)");
    g_scratch_addr[ctx->device] = p;
  }
  *out = g_scratch_addr[ctx->device];
  return WLN_OK;
}

size_t align_up(size_t x) { return (x + 255) / 256 * 256; }

bool is_pinned_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

// Per-profile constants and tile / point offsets (one thread: few profiles).
// Same formulas and tile order as the host-side batch of wln_wilson_avg.
__global__ void noalloc_profiles_kernel(const wln_profile* prof, int32_t n_profiles,
                                        const int32_t* rho_off, const int32_t* T_off, int32_t P,
                                        int32_t ppl, ProfileDev* pd, int32_t* tile_base,
                                        int64_t* point_base) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const double pi = 3.14159265358979323846;
  int32_t tb = 0;
  int64_t pb = 0;
  for (int q = 0; q < n_profiles; ++q) {
    ProfileDev d{};
    d.kind = prof[q].kind;
    if (prof[q].kind == WLN_PROFILE_FLUX_TUBE) {
      d.l2 = prof[q].lambda * prof[q].lambda;
      d.turns_per = prof[q].F / (4.0 * pi * pi);
      d.spin_per = (prof[q].F / (2.0 * pi)) * d.l2 / ppl;
    } else {
      d.l2 = 1.0;
      d.turns_per = prof[q].B / (4.0 * pi);
      d.spin_per = prof[q].B;
    }
    pd[q] = d;
    const int nr = rho_off[q + 1] - rho_off[q], nt = T_off[q + 1] - T_off[q];
    tile_base[q] = tb;
    point_base[q] = pb;
    tb += nt * ((nr + P - 1) / P);
    pb += static_cast<int64_t>(nr) * nt;
  }
  tile_base[n_profiles] = tb;
  point_base[n_profiles] = pb;
}

__global__ void noalloc_tiles_kernel(int32_t n_tiles, int32_t n_profiles, const int32_t* rho_off,
                                     const int32_t* T_off, const double* T, int32_t P,
                                     const int32_t* tile_base, const int64_t* point_base,
                                     Tile* tiles) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  int lo = 0, hi = n_profiles - 1;   // last q with tile_base[q] <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (tile_base[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const int q = lo;
  const int nr = rho_off[q + 1] - rho_off[q];
  const int per_row = (nr + P - 1) / P;
  const int k = t - tile_base[q];
  const int it = k / per_row, a = (k % per_row) * P;
  Tile x{};
  x.profile = q;
  x.n_valid = nr - a < P ? nr - a : P;
  x.rho0 = rho_off[q] + a;
  x.p0 = static_cast<int32_t>(point_base[q] + static_cast<int64_t>(it) * nr + a);
  x.T = T[T_off[q] + it];
  x.part_base = 0;
  x.part_stride = static_cast<int32_t>(point_base[n_profiles]);
  tiles[t] = x;
}

}  // namespace
}  // namespace wln

using namespace wln;

extern "C" wln_status wln_wilson_avg_noalloc(wln_ctx* ctx, const wln_ensemble* ens,
                                             const wln_profile* profiles, int32_t n_profiles,
                                             const double* rho_cm, const int32_t* rho_off,
                                             const double* T, const int32_t* T_off,
                                             int32_t n_groups, wln_prec prec,
                                             double* group_sums) {
  if (!ctx || !ens || !group_sums) return fail(ctx, WLN_EINVAL, "null argument");
  if (prec != WLN_PREC_FP64 && prec != WLN_PREC_FP32_COMP && prec != WLN_PREC_FP32_NAIVE)
    return fail(ctx, WLN_EINVAL, "unknown precision");
  if (ens->device != ctx->device) return fail(ctx, WLN_EINVAL, "ensemble lives on another device");
  if (n_groups < 2 || ens->e.n_loops % n_groups != 0)
    return fail(ctx, WLN_EINVAL, "n_groups must be >= 2 and divide n_loops");
  wln_status st = check_batch(ctx, profiles, n_profiles, rho_cm, rho_off, T, T_off);
  if (st != WLN_OK) return st;
  const int P = plan_points_per_lane(ctx, prec);
  int64_t n_tiles = 0, n_points = 0;
  for (int q = 0; q < n_profiles; ++q) {
    const int nr = rho_off[q + 1] - rho_off[q], nt = T_off[q + 1] - T_off[q];
    n_tiles += static_cast<int64_t>(nt) * ((nr + P - 1) / P);
    n_points += static_cast<int64_t>(nr) * nt;
  }
  if (n_tiles > (int64_t(1) << 30) || n_points > (int64_t(1) << 30))
    return fail(ctx, WLN_EINVAL, "too many points");
  const int32_t n_rho = rho_off[n_profiles], n_T = T_off[n_profiles];
  const int64_t guard_pts =
      guard_applies(ctx, prec, kModeSums, ens->e.n_loops, n_groups, profiles, n_profiles)
          ? guard_points(profiles, n_profiles, rho_cm, rho_off, T, T_off, ens->e)
          : 0;
  const bool use_guard = guard_pts > 0;
  const int bpg = guard_layout_bpg(prec, kModeSums, ens->e.n_loops, n_groups);
  const WilsonPlan plan =
      make_plan(ctx, ens->e, static_cast<int>(n_tiles), prec, kModeSums, bpg);
  const bool host_out = !is_device_ptr(group_sums);

  // Layout inside the array: inputs copied from the host, the work list built
  // on the device, the partial sums and (for a host output) the group sums.
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t at = align_up(off); off = at + bytes; return at; };
  const size_t o_prof = take(sizeof(wln_profile) * n_profiles);
  const size_t o_roff = take(sizeof(int32_t) * (n_profiles + 1));
  const size_t o_toff = take(sizeof(int32_t) * (n_profiles + 1));
  const size_t o_rho = take(sizeof(double) * n_rho);
  const size_t o_T = take(sizeof(double) * n_T);
  const size_t o_pd = take(sizeof(ProfileDev) * n_profiles);
  const size_t o_tb = take(sizeof(int32_t) * (n_profiles + 1));
  const size_t o_pb = take(sizeof(int64_t) * (n_profiles + 1));
  const size_t o_tiles = take(sizeof(Tile) * n_tiles);
  const size_t o_part = take(sizeof(double) * static_cast<size_t>(plan.n_chains + n_groups) *
                             n_points * WLN_K);
  const size_t out_bytes = sizeof(double) * static_cast<size_t>(n_points) * n_groups * WLN_K;
  const size_t o_out = host_out ? take(out_bytes) : 0;
  // the precision guard's per-warp records, queue and counters
  GuardBufs gb;
  size_t o_gscr = 0, o_gq = 0, o_gcnt = 0;
  int64_t gcap = 0;
  if (use_guard) {
    gb.on = 1;
    gb.bpg = bpg;
    gb.warp_bytes = guard_warp_bytes(bpg, plan.P);
    gcap = guard_capacity(guard_pts, n_groups, kGuardPerPair);
    o_gscr = take(static_cast<size_t>(wilson_grid(plan, ens->e, prec)) * plan.warps *
                  gb.warp_bytes);
    o_gq = take(guard_queue_bytes(gcap));
    o_gcnt = take(4 * sizeof(int));
  }
  if (off > kNoAllocBytes)
    return fail(ctx, WLN_EINVAL,
                "problem needs " + std::to_string(off >> 20) + " MiB of working memory; the "
                "no-alloc entry point has " + std::to_string(kNoAllocBytes >> 20) + " MiB "
                "(use wln_wilson_avg, or fewer points or groups)");

  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device) cudaSetDevice(ctx->device);
  void* base = nullptr;
  st = scratch_address(ctx, &base);
  if (st != WLN_OK) {
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return st;
  }
  char* d = static_cast<char*>(base);
  cudaStream_t s = ctx->stream;
  cudaError_t err = cudaMemcpyAsync(d + o_prof, profiles, sizeof(wln_profile) * n_profiles,
                                    cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(d + o_roff, rho_off, sizeof(int32_t) * (n_profiles + 1), cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(d + o_toff, T_off, sizeof(int32_t) * (n_profiles + 1), cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(d + o_rho, rho_cm, sizeof(double) * n_rho, cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(d + o_T, T, sizeof(double) * n_T, cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) {
    noalloc_profiles_kernel<<<1, 1, 0, s>>>(reinterpret_cast<const wln_profile*>(d + o_prof),
                                            n_profiles, reinterpret_cast<const int32_t*>(d + o_roff),
                                            reinterpret_cast<const int32_t*>(d + o_toff), P,
                                            ens->e.ppl, reinterpret_cast<ProfileDev*>(d + o_pd),
                                            reinterpret_cast<int32_t*>(d + o_tb),
                                            reinterpret_cast<int64_t*>(d + o_pb));
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) {
    noalloc_tiles_kernel<<<static_cast<unsigned>((n_tiles + 255) / 256), 256, 0, s>>>(
        static_cast<int32_t>(n_tiles), n_profiles, reinterpret_cast<const int32_t*>(d + o_roff),
        reinterpret_cast<const int32_t*>(d + o_toff), reinterpret_cast<const double*>(d + o_T), P,
        reinterpret_cast<const int32_t*>(d + o_tb), reinterpret_cast<const int64_t*>(d + o_pb),
        reinterpret_cast<Tile*>(d + o_tiles));
    err = cudaGetLastError();
  }
  const int32_t lpg = ens->e.n_loops / n_groups;
  double* out = host_out ? reinterpret_cast<double*>(d + o_out) : group_sums;
  int64_t launches = 2;
  if (use_guard) {
    guard_bind(gb, d + o_gscr, d + o_gq, gcap, reinterpret_cast<int*>(d + o_gcnt));
    guard_attach(gb, ctx);
    if (err == cudaSuccess) err = cudaMemsetAsync(gb.counters, 0, 4 * sizeof(int), s);
  }
  if (err == cudaSuccess)
    err = launch_wilson(s, plan, ens->e, reinterpret_cast<const Tile*>(d + o_tiles),
                        reinterpret_cast<const ProfileDev*>(d + o_pd),
                        reinterpret_cast<const double*>(d + o_rho), n_groups, lpg, prec,
                        reinterpret_cast<double*>(d + o_part), n_points, ctx->d_flag, &launches,
                        use_guard ? &gb : nullptr, ctx->d_items);
  if (err == cudaSuccess)
    err = launch_guard(s, gb, ens->e, reinterpret_cast<const Tile*>(d + o_tiles),
                       reinterpret_cast<const ProfileDev*>(d + o_pd),
                       reinterpret_cast<const double*>(d + o_rho),
                       reinterpret_cast<double*>(d + o_part), ctx->num_sms, &launches);
  if (err == cudaSuccess) {
    err = launch_reduce_partials(s, plan, ens->e, reinterpret_cast<const double*>(d + o_part),
                                 n_points, n_groups, lpg, out);
    ++launches;
  }
  ctx->launches += launches;
  // Inputs in page-locked host memory are read by the stream later, not
  // during the copy call: wait until the stream has read them, so that the
  // caller may reuse them on return (pageable inputs are staged by the copy
  // call itself).  The context's staging event is recorded, not created.
  bool pinned_inputs = false;
  for (const void* q : {static_cast<const void*>(profiles), static_cast<const void*>(rho_off),
                        static_cast<const void*>(T_off), static_cast<const void*>(rho_cm),
                        static_cast<const void*>(T)})
    pinned_inputs = pinned_inputs || is_pinned_host(q);
  if (err == cudaSuccess && host_out)
    err = cudaMemcpyAsync(group_sums, out, out_bytes, cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess && !host_out && pinned_inputs) {
    err = cudaEventRecord(ctx->staging_done, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(ctx->staging_done);
  }
  if (err != cudaSuccess) {
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return cuda_fail(ctx, err, "no-alloc Wilson group sums");
  }
  // A host output waits for the stream and reads (and clears) the device
  // error flag, as wln_wilson_avg does; with a device output the flag is read
  // by the next synchronising call (wln_synchronize).
  st = host_out ? check_flag(ctx) : WLN_OK;
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  return st;
}
