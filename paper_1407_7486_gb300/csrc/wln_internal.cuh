// Internal declarations shared by the CUDA translation units of libwln.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "wln.h"

namespace wln {

// Loops are stored in blocks of 32 (one loop per warp lane).  Within a block,
// row i2 holds points 2*i2 and 2*i2+1 of each loop as one float4
// (x0, y0, x1, y1); lane l of the block is loop 32*b + l.  A block is
// therefore ppl/2 rows of 32 float4 (512 bytes per row), contiguous, so a
// range of rows is one bulk (TMA) copy and a warp reads a row with one
// conflict-free 16-byte load per lane.
constexpr int kLanes = 32;

// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit multiplies with the round keys bumped by the Weyl
// constants.  Streams in use: counter (j, loop, 0, 0) increments of
// wln_gen_loops; (m/2, loop, 1, 0) Gaussians of wln_gen_dloops; (t/4, point,
// 2, 0) the Fisher-Yates draws of the randomised groups.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Device error flag values: bounded waits that ran out, and a precision-guard
// queue that could not hold every loop its launch selected.
constexpr int kErrTimeoutFull = 1;
constexpr int kErrTimeoutEmpty = 2;
constexpr int kErrTimeoutSelfTest = 3;
constexpr int kErrGuardQueue = 4;

struct Ensemble {
  int64_t loop0 = 0;          // global index of the first loop (Philox counter word 1)
  int32_t n_loops = 0;
  int32_t ppl = 0;
  int32_t n_blocks = 0;       // ceil(n_loops / 32)
  float4* blocks = nullptr;   // [n_blocks][ppl/2][32]
  double* xy64 = nullptr;     // optional [n_loops][2][ppl]
  float2* stats = nullptr;    // [n_blocks]: longest segment, largest |y| of the block's loops
  float2* sub_stats = nullptr;  // [n_blocks][n_sub]: the same over kSubRows rows (their
                                // segments, the next row's first point included)
  float* maxlen = nullptr;    // [n_blocks]: longest loop (sum of its segment lengths)
  int32_t n_sub = 0;          // ceil(ppl / 2 / kSubRows); stats, sub_stats and maxlen
                              // share one allocation (ensemble_stats_bytes)
  float ymax = 0.0f;          // host copy of the largest |y| of any loop (host-side bounds)
};

constexpr int kSubRows = 64;   // rows (point pairs) per sub-block of the statistics
inline int32_t ensemble_n_sub(int32_t ppl) { return (ppl / 2 + kSubRows - 1) / kSubRows; }
inline size_t ensemble_stats_bytes(int32_t n_blocks, int32_t ppl) {
  return static_cast<size_t>(n_blocks) * (1 + ensemble_n_sub(ppl)) * sizeof(float2) +
         static_cast<size_t>(n_blocks) * sizeof(float);
}
// The views into the statistics allocation at e.stats.
inline void bind_ensemble_stats(Ensemble& e) {
  e.n_sub = ensemble_n_sub(e.ppl);
  e.sub_stats = e.stats + e.n_blocks;
  e.maxlen = reinterpret_cast<float*>(e.sub_stats + static_cast<size_t>(e.n_blocks) * e.n_sub);
}

// Per-profile constants used by the Wilson kernels.
struct ProfileDev {
  int32_t kind;
  int32_t pad;
  double l2;          // lambda^2
  double turns_per;   // flux tube: calF/(2 pi) = F/(4 pi^2), phase in turns per unit sum X*J1
                      // constant field: B/(4 pi), turns per unit sum of X (twice the area)
  double spin_per;    // flux tube: calF lambda^2 / N per unit T per unit sum of j2;
                      // constant field: B (spin = B T)
};

// A tile: P consecutive radii of one profile at one proper time.  Its
// partial sums go to partial[part_base + ((c + g) * part_stride + p0 + i) * K]:
// one launch can serve several independent batches (requests), each with its
// own partial buffer and point count.
struct Tile {
  int32_t profile;
  int32_t n_valid;    // radii in this tile (1..P)
  int32_t rho0;       // index of the first radius in the flattened rho array
  int32_t p0;         // point index of the first radius within its batch
  double T;
  int64_t part_base;  // offset (in doubles) of its batch's partial buffer
  int32_t part_stride;  // points in its batch
  int32_t pad;
};

// What a Wilson launch produces: group sums (WLN_K per point and group), the
// discretisation levels (WLN_KL), or every loop's W - 1 (scalar, spinor).
// kModeNested: levels from the nested loops (all points, even points, points
// 0 mod 4), WLN_KL components like kModeLevels.
constexpr int kModeSums = 0, kModeLevels = 1, kModeLoops = 2, kModeNested = 3;
__host__ __device__ constexpr bool level_mode(int mode) {
  return mode == kModeLevels || mode == kModeNested;
}

// Geometry of one Wilson launch.
struct WilsonPlan {
  int P;              // points (radii) per lane
  int warps;          // warps (tiles) per CTA
  int rows;           // float4 rows per staged chunk
  int stages;         // staged chunks in flight
  int chain;          // 32-loop blocks per work item
  int n_tiles;
  int n_tile_groups;  // ceil(n_tiles / warps)
  int n_chains;       // ceil(n_blocks / chain)
  int64_t n_items;    // n_chains * n_tile_groups
  int grid;           // persistent CTAs
  int mode;           // kModeSums, kModeLevels, kModeLoops or kModeNested
  int low_angle;      // highest cheaper form of theta a block may take (0, 1 or 2)
};

// Precision guard of the FP32-compensated group sums (wln_guard.cu): a
// queued loop to recompute in double-float, the partial sum its correction
// belongs to, and the buffers of one Wilson launch.
struct GuardItem {
  int32_t tile;     // tile index in the launch's work list; -1: not filled
  int32_t p_loop;   // radius within the tile << 24 | loop index
  double f1;        // the float pass's W_ferm - 1 of this loop and radius
};
struct GuardSlot {
  int64_t dst;      // index (in doubles) of the partial's first component
  int32_t item0;    // its queued loops: items [item0, item0 + n)
  int32_t n;
};
constexpr int kGuardSel = 64;   // loops a warp may select per (group, radius)
constexpr float kGuardFloor = 2.0f;   // blocks whose largest spin stays below are not recorded
constexpr int kGuardPerPair = 8;      // queue entries provided per (point, group) that can
                                      // reach the floor, before a launch shows its need
struct GuardBufs {
  int on = 0;
  int all = 0;                  // select every recorded loop (a check of the double-float walk)
  int bpg = 0;                  // 32-loop blocks per group
  char* scratch = nullptr;      // per warp (guard_warp_bytes): block maxima, per-lane
                                // |spin|, sin(phase), float W_ferm - 1, selection list
  size_t warp_bytes = 0;
  GuardItem* items = nullptr;
  double2* out = nullptr;       // per item: corrections of W_ferm - 1 and of its square
  GuardSlot* slots = nullptr;
  int64_t cap = 0;              // items (and slots) the queue holds
  int* counters = nullptr;      // this launch: items, slots, overflows, saturated selections
  unsigned long long* totals = nullptr;   // the context's running totals (wln_precision_guard_stats)
  int* flag = nullptr;          // the context's device error flag (kErrGuardQueue on overflow)
};

struct Scratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace wln

struct wln_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string last_error;
  int num_sms = 0;
  int64_t launches = 0;
  int* d_flag = nullptr;          // device error flag
  wln::Scratch scratch;           // partial sums, work lists (device)
  void* pinned = nullptr;         // host staging for work lists
  size_t pinned_bytes = 0;
  cudaEvent_t staging_done = nullptr;
  // tuning overrides (0 = automatic)
  int tune_P = 0, tune_warps = 0, tune_rows = 0, tune_stages = 0, tune_chain = 0;
  int low_angle = 2;    // highest cheaper form of theta the float walks may take
  int guard = 1;        // precision guard of the FP32-compensated group sums (2: every
                        // recorded loop, a check of the double-float walk)
  unsigned long long* d_guard_totals = nullptr;   // escalated loops, overflows, saturated, launches
  int* d_items = nullptr;   // a Wilson launch's item counter (dynamic schedule), zeroed per launch
  // Device memory of the last freed ensembles, reused by the next ensemble of
  // the same shape: a loop that draws and frees an ensemble every step then
  // makes no cudaMalloc / cudaFree, which would wait for the whole device.
  struct EnsembleMem {
    float4* blocks;
    float2* stats;
    double* xy64;
    size_t n4, n_blocks, n64;
  };
  std::vector<EnsembleMem> ens_cache;
};
constexpr size_t kEnsembleCache = 2;   // freed ensembles a context keeps

struct wln_ensemble {
  wln::Ensemble e;
  int device = 0;
};

namespace wln {

// Status helpers (wln_api.cu).
wln_status fail(wln_ctx* ctx, wln_status st, const std::string& msg);
wln_status cuda_fail(wln_ctx* ctx, cudaError_t err, const char* what);
bool is_device_ptr(const void* p);
// Waits for the context's stream, then reads and clears the device error
// flag: WLN_ETIMEOUT when a bounded device wait ran out since the last check.
wln_status check_flag(wln_ctx* ctx);
wln_status ensure_scratch(wln_ctx* ctx, size_t bytes);
wln_status ensure_pinned(wln_ctx* ctx, size_t bytes);

// Restores the caller's current device on scope exit (wln_api.cu).
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev);
  ~DeviceGuard();
};

// Host-side work list of one batch of profiles (wln_api.cu).
struct Batch {
  std::vector<Tile> tiles;
  std::vector<ProfileDev> profs;
  std::vector<double> rho;
  int64_t n_points = 0;
};
wln_status check_batch(wln_ctx* ctx, const wln_profile* profiles, int32_t n_profiles,
                       const double* rho_cm, const int32_t* rho_off, const double* T,
                       const int32_t* T_off);
void build_batch(const wln_profile* profiles, int32_t n_profiles, const double* rho_cm,
                 const int32_t* rho_off, const double* T, const int32_t* T_off, int ppl, int P,
                 Batch& bt);
ProfileDev profile_constants(const wln_profile& pr, int ppl);

// Generation (wln_gen.cu).
cudaError_t launch_philox_stream(cudaStream_t s, uint64_t seed, int64_t loop0, int32_t n_loops,
                                 int32_t n_calls, uint32_t* out);
// Unit loops: increments drawn once into `work` (gen_loops_work_bytes of
// it), then closed and centred; blocks are taken in slices so that `work`
// stays within kGenWorkBytes.  gen_loops_launches counts the kernels.
constexpr int kGenChunk = 32;                       // points per warp drawing increments
constexpr int kGenWarps = 4;                        // warps per CTA drawing increments
constexpr size_t kGenWorkBytes = size_t(1) << 30;   // increments and chunk sums of a slice
int gen_warps(int32_t ppl);
int gen_chunk(int32_t ppl);
int gen_slice_blocks(int32_t n_blocks, int32_t ppl);
size_t gen_loops_work_bytes(int32_t n_blocks, int32_t ppl);
int gen_loops_launches(int32_t n_blocks, int32_t ppl);
cudaError_t launch_gen_loops(cudaStream_t s, uint64_t seed, const Ensemble& e, void* work,
                             int* d_degenerate);
// d-loops: Gaussians drawn into `work` (gen_dloops_work_bytes of it), then
// the bisection levels built in place, in slices of blocks within
// kGenWorkBytes.
int gen_dslice_blocks(int32_t n_blocks, int32_t ppl);
size_t gen_dloops_work_bytes(int32_t n_blocks, int32_t ppl);
int gen_dloops_launches(int32_t n_blocks, int32_t ppl);
cudaError_t launch_gen_dloops(cudaStream_t s, uint64_t seed, const Ensemble& e, void* work,
                              int* d_degenerate);
cudaError_t launch_pack_loops(cudaStream_t s, const float* xy, const Ensemble& e, int* d_degenerate);
cudaError_t launch_unpack_loops(cudaStream_t s, const Ensemble& e, float* xy);

// Wilson loops (wln_wilson.cu).  A launch given an item counter (device int,
// zeroed by the launch on its stream) schedules items dynamically: each CTA
// starts with its own index and claims the next free item when it starts
// staging one, so CTAs that finish early take more (results do not depend
// on which CTA walks an item).  guard_bpg > 0 aligns the chains of blocks to
// groups of that many blocks, as the precision guard needs.
WilsonPlan make_plan(const wln_ctx* ctx, const Ensemble& e, int n_tiles, wln_prec prec,
                     int mode = kModeSums, int guard_bpg = 0);
// The persistent grid a Wilson launch of this plan uses.
int wilson_grid(const WilsonPlan& plan, const Ensemble& e, wln_prec prec);
int plan_points_per_lane(const wln_ctx* ctx, wln_prec prec, int mode = kModeSums);
cudaError_t launch_wilson(cudaStream_t s, const WilsonPlan& plan, const Ensemble& e,
                          const Tile* tiles, const ProfileDev* profs, const double* rho,
                          int32_t n_groups, int32_t loops_per_group, wln_prec prec,
                          double* partial, int64_t n_points, int* d_flag, int64_t* launches,
                          const GuardBufs* guard = nullptr, int* item_counter = nullptr);

// Precision guard (wln_guard.cu).  The blocks per group when the pass's
// layout admits it (FP32-compensated group sums, groups of a whole number of
// 32-loop blocks, at most 64), else 0: the plan aligns its chains to them
// whether or not the guard runs, so the guard changes only the loops it
// recomputes.  Whether a pass takes it: that layout, the context's setting,
// and some flux-tube profile.
int guard_layout_bpg(wln_prec prec, int mode, int32_t n_loops, int32_t n_groups);
bool guard_applies(const wln_ctx* ctx, wln_prec prec, int mode, int32_t n_loops,
                   int32_t n_groups, const wln_profile* profiles, int32_t n_profiles);
size_t guard_warp_bytes(int bpg, int P);
// Points whose spin can reach kGuardFloor at all: spin <= T eB(gap), eB(r) =
// 2 calF lambda^2 / (lambda^2 + r^2)^2 the tube's field, gap = max(0, rho -
// sqrt(T) ymax) the closest any loop comes to the axis (a 1% margin on ymax
// and 10% on the floor).  Only these can put loops in the guard's queue.
bool guard_point_reaches(const wln_profile& pr, double rho, double T, const Ensemble& e);
int64_t guard_points(const wln_profile* profiles, int32_t n_profiles, const double* rho_cm,
                     const int32_t* rho_off, const double* T, const int32_t* T_off,
                     const Ensemble& e);
// Queue entries for n_points such points: per_pair per (point, group), at
// least 65536; 0 when no point can reach the floor.
int64_t guard_capacity(int64_t n_points, int32_t n_groups, int per_pair);
size_t guard_queue_bytes(int64_t cap);
void guard_bind(GuardBufs& g, void* scratch, void* queue, int64_t cap, int* counters);
// The context's mode and running totals into g.
void guard_attach(GuardBufs& g, const wln_ctx* ctx);
// Recomputes the queued loops and adds the corrections to their partials.
cudaError_t launch_guard(cudaStream_t s, const GuardBufs& g, const Ensemble& e,
                         const Tile* tiles, const ProfileDev* profs, const double* rho,
                         double* partial, int num_sms, int64_t* launches);
// Per-loop values: out[p][loop][2] = (W_scal - 1, W_ferm - 1), p the point.
cudaError_t launch_wilson_loops(cudaStream_t s, const WilsonPlan& plan, const Ensemble& e,
                                const Tile* tiles, const ProfileDev* profs, const double* rho,
                                wln_prec prec, double* out, int* d_flag, int64_t* launches,
                                int* item_counter = nullptr);
// Group sums [n_points][G][WLN_K] of per-loop values [n_points][n_loops][2],
// contiguous groups or (shuffle) a Fisher-Yates permutation per point;
// perm: [n_points][n_loops] scratch (and output) for the shuffled order.
cudaError_t launch_group_sums_loops(cudaStream_t s, const double* W, int64_t n_points,
                                    int32_t n_loops, int32_t G, bool shuffle, uint64_t seed,
                                    int32_t* perm, double* S, int64_t* launches);
cudaError_t launch_corrcoef(cudaStream_t s, const double* X, int32_t n_rows, int32_t n_samples,
                            int32_t stride, int32_t comp, int32_t ref, double* out);
cudaError_t launch_selftest_wait(cudaStream_t s, int* d_flag, uint64_t limit_ns);
cudaError_t launch_reduce_partials(cudaStream_t s, const WilsonPlan& plan, const Ensemble& e,
                                   const double* partial, int64_t n_points, int32_t n_groups,
                                   int32_t loops_per_group, double* group_sums);

// Statistics (wln_stats.cu).
// cov_packed: the covariance as its upper triangle, row by row
// (n (n + 1) / 2 doubles), else the full n x n matrix.
cudaError_t launch_jackknife(cudaStream_t s, const double* S, int32_t n_points, int32_t G,
                             int32_t lpg, int32_t comp, double* mean, double* sem,
                             double* jk_var, double* dev_scratch, double* cov, int64_t* launches,
                             bool cov_packed = false);
cudaError_t launch_extrapolate(cudaStream_t s, const double* level_sums, int32_t n_points,
                               int32_t G, int32_t lpg, double* out);
cudaError_t launch_loop_sem(cudaStream_t s, const double* S, int32_t n_points, int32_t G,
                            int32_t n_loops, int32_t comp_sum, int32_t comp_sq, double* out);

struct QuadProfile {
  int32_t kind;
  int32_t n_rho, n_T;
  int32_t rho_base;  // first radius in the flattened radii
  int32_t T_base;    // first proper time in the flattened times
  int32_t pad;
  int64_t p0;        // first point of the profile
  double h_rho;      // radius spacing
  double h_u;        // spacing of ln T
  double eB_scale;   // flux tube: 2 calF lambda^2 = F lambda^2 / pi; constant: B
  double l2;
  // axis kinds (WLN_GRID_*) and mapped-grid parameters
  int32_t rho_kind = WLN_GRID_LINEAR, T_kind = WLN_GRID_LOG;
  int32_t small_T = 0, pad2 = 0;
  double rho_scale = 0.0, T_scale = 0.0;
  double rho_x0 = 1.0, T_x0 = 1.0;   // x at the first node of a mapped axis
};
// Quadrature tables of a batch of profiles; false (with a reason) when a
// profile's radii are not evenly spaced or its times not geometric (wln_api.cu).
// quad: per-profile grid kinds (nullptr: linear radii, geometric times).
bool build_quad(const wln_profile* profiles, int32_t n_profiles, const double* rho_cm,
                const int32_t* rho_off, const double* T, const int32_t* T_off,
                std::vector<QuadProfile>& qp, std::string* why,
                const wln_quad* quad = nullptr);
// Full effective action (wln_effective_action_full): d_groups is scratch of
// n_rho_total * G doubles; rho_profile maps a flattened radius to its profile.
cudaError_t launch_effective_action_full(cudaStream_t s, const QuadProfile* qp,
                                         int32_t n_profiles, int32_t max_rho,
                                         int32_t n_rho_total, int64_t n_points,
                                         const int32_t* point_profile, const double* rho,
                                         const double* T, const double* S, int32_t G,
                                         int32_t lpg, int32_t spinor, double* d_groups,
                                         double* gamma_groups, double* gamma, double* density,
                                         double* integrand, int64_t* launches);
cudaError_t launch_effective_action(cudaStream_t s, const QuadProfile* qp, int32_t n_profiles,
                                    const double* rho, const double* T, const double* S,
                                    int32_t G, int32_t lpg, int32_t spinor, double* gamma_groups,
                                    double* gamma_mean_sem, int64_t* launches);

}  // namespace wln
