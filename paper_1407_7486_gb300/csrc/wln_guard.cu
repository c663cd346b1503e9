// Precision guard of the FP32-compensated group sums (paper Sec.
// "Uncertainties and the Fermion Problem": the spinor factor cosh(spin)
// magnifies every error of the phase and spin, so a group mean carries the
// errors of the few loops with the largest spins, undiluted).
//
// The float pass (wln_wilson.cu) keeps, for every block of 32 loops whose
// largest spin reaches kGuardFloor, each loop's spin, sin(phase) and float
// W_ferm - 1.  At the end of every group it estimates the rounding error of
// the group's spinor sum from a model of the float walk and, while the
// estimate exceeds half of the 1e-6 bar (relative to max(1, <cosh spin>)),
// selects the loop with the largest error share, up to 64 loops.  Selected
// (point, loop) pairs go to a queue; a slot entry names the partial sum they
// belong to.
//
// This file recomputes each queued loop with a double-float walk (each value
// an unevaluated sum hi + lo of two floats, ~2^-44 relative), forms W_ferm - 1
// in double, and adds W_df - W_float (and the same for the square) to the
// loop's partial sum, summing the corrections of one slot in queue order: the
// result does not depend on scheduling.  Double-float keeps the work on the
// FP32 pipe, 64 times as wide as GB300's FP64 pipe.
//
// Double-float arithmetic: error-free transformations of Knuth (two-sum),
// Dekker (fast two-sum) and the FMA two-product; addition, multiplication,
// reciprocal and reciprocal square root as in Joldes, Muller and Popescu,
// "Tight and rigorous error bounds for basic building blocks of double-word
// arithmetic" (ACM TOMS 2017), the last two by one Newton-Raphson step from
// the float approximation.  The arctangent reduces its argument with a table
// of atan(j/16) and sums five terms of the Taylor series.  Intrinsics with
// explicit rounding keep the compiler from fusing the transformations.
#include <cmath>

#include "wln_internal.cuh"

namespace wln {
namespace {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return ff{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_of(double x) {
  const float h = static_cast<float>(x);
  return ff{h, static_cast<float>(x - static_cast<double>(h))};
}

__device__ __forceinline__ ff neg(ff a) { return ff{-a.hi, -a.lo}; }

// Sum without cancellation between the operands (error ~2^-46 (|a| + |b|)).
__device__ __forceinline__ ff add(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

// Sum accurate relative to the result, also under cancellation (running sums).
__device__ __forceinline__ ff add_acc(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  const ff t = two_sum(a.lo, b.lo);
  const ff v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}

__device__ __forceinline__ ff mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ ff mul_f(ff a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// 1/a: r = approx(1/a.hi), then r + r (1 - a r) with the residual exact to
// first order (two FMAs); the error of r squares.
__device__ __forceinline__ ff rcp(ff a) {
  const float r = rcp_approx(a.hi);
  float e = __fmaf_rn(-a.hi, r, 1.0f);
  e = __fmaf_rn(-a.lo, r, e);
  return fast_two_sum(r, __fmul_rn(r, e));
}

// 1/sqrt(a), a > 0: y + y (1 - a y^2) / 2 from the float approximation y.
__device__ __forceinline__ ff rsqrt(ff a) {
  const float y = rsqrt_approx(a.hi);
  const float y2 = __fmul_rn(y, y);
  const ff ay2 = mul(a, ff{y2, __fmaf_rn(y, y, -y2)});
  const float e = __fsub_rn(__fsub_rn(1.0f, ay2.hi), ay2.lo);   // 1 - a y^2, exact to 2^-46
  return fast_two_sum(y, __fmul_rn(__fmul_rn(0.5f, y), e));
}

// atan(j/16), j = 0..16, and pi, pi/2, 1/3 as hi + lo (gen_ff_consts.py).
__constant__ float2 kAtanTable[17] = {
    {0.0f, 0.0f},
    {6.241881102e-02f, -1.027277929e-09f},
    {1.243549958e-01f, -1.240382241e-09f},
    {1.853479445e-01f, 5.497632571e-09f},
    {2.449786663e-01f, -3.178677765e-09f},
    {3.028848767e-01f, -8.353086223e-09f},
    {3.587706685e-01f, 1.763949875e-09f},
    {4.124104381e-01f, 3.536626769e-09f},
    {4.636476040e-01f, 5.012158688e-09f},
    {5.123894811e-01f, -2.075691974e-08f},
    {5.585992932e-01f, 2.211159789e-08f},
    {6.022873521e-01f, -5.950149262e-09f},
    {6.435011029e-01f, 5.868937336e-09f},
    {6.823165417e-01f, 1.320299514e-08f},
    {7.188299894e-01f, 1.018833551e-08f},
    {7.531512976e-01f, -1.660708016e-08f},
    {7.853981853e-01f, -2.185569414e-08f},
};
constexpr float kPI_HI = 3.141592741e+00f, kPI_LO = -8.742277657e-08f;
constexpr float kPI_2_HI = 1.570796371e+00f, kPI_2_LO = -4.371138829e-08f;
constexpr float kTHIRD_HI = 3.333333433e-01f, kTHIRD_LO = -9.934107759e-09f;

// atan(u) for 0 <= u <= 1 (u.hi may exceed 1 by a rounding): with c = j/16
// the nearest table point, atan u = atan c + atan v, v = (u - c)/(1 + u c),
// |v| <= 1/32 + rounding; atan v / v = 1 - v^2/3 + v^4/5 - v^6/7 + v^8/9
// (the next term, v^10/11 < 1e-16, is dropped), the head 1 - v^2/3 in
// double-float and the rest (< 2e-7) in float.  tab: the table in shared memory.
__device__ __forceinline__ ff atan_unit(ff u, const float2* tab) {
  const int j = min(16, max(0, __float2int_rn(__fmul_rn(u.hi, 16.0f))));
  const float c = __fmul_rn(static_cast<float>(j), 0.0625f);
  const ff num = add(u, ff{-c, 0.0f});                  // exact: u and c are close
  const ff den = add(ff{1.0f, 0.0f}, mul_f(u, c));
  const ff v = mul(num, rcp(den));
  const ff v2 = mul(v, v);
  const float t = v2.hi;
  const float tail = __fmul_rn(__fmul_rn(t, t),
                               __fmaf_rn(t, __fmaf_rn(t, 1.0f / 9.0f, -1.0f / 7.0f), 0.2f));
  const ff third = mul(v2, ff{kTHIRD_HI, kTHIRD_LO});
  const ff q = add(add(ff{1.0f, 0.0f}, neg(third)), ff{tail, 0.0f});
  const float2 a = tab[j];
  return add(ff{a.x, a.y}, mul(v, q));
}

// The angle of (x, y), y > 0, in (0, pi): fold to [0, 1], then unfold the
// octant (pi/2 - a above the diagonal, pi - a for x < 0).
__device__ __forceinline__ ff atan2_pos(ff y, ff x, const float2* tab) {
  const bool xneg = x.hi < 0.0f;
  const ff ax = xneg ? neg(x) : x;
  const bool up = y.hi > ax.hi;
  const ff u = up ? mul(ax, rcp(y)) : mul(y, rcp(ax));
  ff a = atan_unit(u, tab);
  if (up) a = add(ff{kPI_2_HI, kPI_2_LO}, neg(a));
  if (xneg) a = add(ff{kPI_HI, kPI_LO}, neg(a));
  return a;
}

// One loop at one point in double-float: the same closed forms as the float
// walk and the oracle (segment phase calF X int dt/Q, spin 2 calF lambda^2
// (T/N) int dt/Q^2; Eqs. rhoi-Ci and the spin integral of Eq. Wfermfpl),
// with theta = atan2(sqrt(D), Q0 + B) and the spin bracket
// (D - B (B + C)) / (Q0 Q1) + C int dt/Q.
struct FFWalk {
  ff s, rho, l2;        // sqrt(T), rho_cm, lambda^2
  ff rx, ry, q, rq;     // position, Q and 1/Q at the current point
  ff ph, sp;            // sums of X int dt/Q and of the spin bracket / D

  __device__ __forceinline__ void start(float x0, float y0) {
    rx = add(rho, mul_f(s, x0));
    ry = mul_f(s, y0);
    q = add(l2, add(mul(rx, rx), mul(ry, ry)));
    rq = rcp(q);
    ph = ff{0.0f, 0.0f};
    sp = ff{0.0f, 0.0f};
  }

  __device__ __forceinline__ void step(float x1, float y1, const float2* tab) {
    const ff rx1 = add(rho, mul_f(s, x1));
    const ff ry1 = mul_f(s, y1);
    const ff dx = add(rx1, neg(rx)), dy = add(ry1, neg(ry));
    const ff C = add(mul(dx, dx), mul(dy, dy));
    const ff B = add(mul(rx, dx), mul(ry, dy));
    const ff X = add(mul(rx, dy), neg(mul(ry, dx)));
    const ff D = add(mul(l2, C), mul(X, X));
    const ff q1 = add(l2, add(mul(rx1, rx1), mul(ry1, ry1)));
    const ff rq1 = rcp(q1);
    const ff rsD = rsqrt(D);
    const ff theta = atan2_pos(mul(D, rsD), add(q, B), tab);
    const ff J1 = mul(theta, rsD);
    ph = add_acc(ph, mul(X, J1));
    const ff bc = add(B, C);
    const ff br = add(mul(mul(add(D, neg(mul(B, bc))), rq), rq1), mul(C, J1));
    sp = add_acc(sp, mul(br, mul(rsD, rsD)));
    rx = rx1; ry = ry1; q = q1; rq = rq1;
  }
};

// cosh(x) - 1 = 2 sinh^2(x/2)
__device__ __forceinline__ double cosh_m1(double x) {
  const double h = sinh(0.5 * x);
  return 2.0 * h * h;
}

// One thread per queued (point, loop): the loop's W_ferm - 1 in double-float,
// and its difference from the float value the float pass summed.
__global__ void __launch_bounds__(128) guard_walk_kernel(GuardBufs g, const float4* blocks,
                                                         int32_t ppl, const Tile* tiles,
                                                         const ProfileDev* profs,
                                                         const double* rho) {
  __shared__ float2 tab[17];
  if (threadIdx.x < 17) tab[threadIdx.x] = kAtanTable[threadIdx.x];
  __syncthreads();
  const int64_t n = min(static_cast<int64_t>(g.counters[0]), g.cap);
  const int rows = ppl / 2;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const GuardItem it = g.items[i];
    if (it.tile < 0) continue;   // a reservation past the queue's end
    const Tile tile = tiles[it.tile];
    const int p = it.p_loop >> 24, loop = it.p_loop & 0xFFFFFF;
    const ProfileDev prof = profs[tile.profile];
    FFWalk w;
    w.s = ff_of(sqrt(tile.T));
    w.rho = ff_of(rho[tile.rho0 + p]);
    w.l2 = ff_of(prof.l2);
    const float4* src = blocks + static_cast<size_t>(loop >> 5) * rows * 32 + (loop & 31);
    const float4 v0 = src[0];
    w.start(v0.x, v0.y);
    w.step(v0.z, v0.w, tab);
    for (int r = 1; r < rows; ++r) {
      const float4 v = src[static_cast<size_t>(r) * 32];
      w.step(v.x, v.y, tab);
      w.step(v.z, v.w, tab);
    }
    w.step(v0.x, v0.y, tab);   // closing segment
    const double turns =
        (static_cast<double>(w.ph.hi) + static_cast<double>(w.ph.lo)) * prof.turns_per;
    const double fr = turns - rint(turns);
    const double h = sinpi(fr);
    const double scal_m1 = -2.0 * h * h;
    const double spin = (static_cast<double>(w.sp.hi) + static_cast<double>(w.sp.lo)) *
                        (prof.spin_per * tile.T);
    const double ferm_m1 = cospi(2.0 * fr) * cosh_m1(spin) + scal_m1;
    // Past the double range (spins above ~710, squares above ~355) both the
    // float pass and the oracle hold +-inf: the float value stays.
    const double d1 = ferm_m1 - it.f1, d2 = ferm_m1 * ferm_m1 - it.f1 * it.f1;
    g.out[i] = make_double2(isfinite(d1) ? d1 : 0.0, isfinite(d2) ? d2 : 0.0);
  }
}

// Adds each slot's corrections, in queue order, to the spinor components of
// its partial sum; then counts the launch into the context totals, and raises
// the context's error flag if the queue could not hold every selected loop
// (those selections kept float precision).
__global__ void guard_fixup_kernel(GuardBufs g, double* partial) {
  const int64_t n = g.counters[1];
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const GuardSlot sl = g.slots[i];
    double a = 0.0, b = 0.0;
    for (int j = 0; j < sl.n; ++j) {
      const double2 d = g.out[sl.item0 + j];
      a += d.x;
      b += d.y;
    }
    partial[sl.dst + WLN_C_FERM] += a;
    partial[sl.dst + WLN_C_FERM_SQ] += b;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && g.totals) {
    atomicAdd(&g.totals[0], static_cast<unsigned long long>(
                                min(static_cast<int64_t>(g.counters[0]), g.cap)));
    atomicAdd(&g.totals[1], static_cast<unsigned long long>(g.counters[2]));
    atomicAdd(&g.totals[2], static_cast<unsigned long long>(g.counters[3]));
    atomicAdd(&g.totals[3], 1ull);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && g.flag && g.counters[2] > 0)
    atomicExch(g.flag, kErrGuardQueue);
}

}  // namespace

size_t guard_warp_bytes(int bpg, int P) {
  const size_t recs = static_cast<size_t>(bpg) * P;
  size_t off = (recs * sizeof(float) + 15) / 16 * 16;          // block maxima
  off += 2 * recs * 32 * sizeof(float);                        // |spin|, sin(phase) per lane
  off += recs * 32 * sizeof(double);                           // float W_ferm - 1 per lane
  off += kGuardSel * sizeof(int32_t);                          // selection list
  return (off + 255) / 256 * 256;
}

size_t guard_queue_bytes(int64_t cap) {
  return static_cast<size_t>(cap) * (sizeof(GuardItem) + sizeof(double2) + sizeof(GuardSlot));
}

void guard_bind(GuardBufs& g, void* scratch, void* queue, int64_t cap, int* counters) {
  g.scratch = static_cast<char*>(scratch);
  char* q = static_cast<char*>(queue);
  g.items = reinterpret_cast<GuardItem*>(q);
  g.out = reinterpret_cast<double2*>(q + static_cast<size_t>(cap) * sizeof(GuardItem));
  g.slots = reinterpret_cast<GuardSlot*>(q + static_cast<size_t>(cap) *
                                                 (sizeof(GuardItem) + sizeof(double2)));
  g.cap = cap;
  g.counters = counters;
}

void guard_attach(GuardBufs& g, const wln_ctx* ctx) {
  g.all = ctx->guard == 2;
  g.totals = ctx->d_guard_totals;
  g.flag = ctx->d_flag;
}

bool guard_point_reaches(const wln_profile& pr, double rho, double T, const Ensemble& e) {
  if (pr.kind != WLN_PROFILE_FLUX_TUBE) return false;
  const double pi = 3.14159265358979323846;
  const double l2 = pr.lambda * pr.lambda;
  const double gap = std::fmax(0.0, rho - std::sqrt(T) * 1.01 * static_cast<double>(e.ymax));
  const double den = l2 + gap * gap;
  return T * 2.0 * std::fabs(pr.F) / (2.0 * pi) * l2 / (den * den) >= 0.9 * kGuardFloor;
}

int64_t guard_points(const wln_profile* profiles, int32_t n_profiles, const double* rho_cm,
                     const int32_t* rho_off, const double* T, const int32_t* T_off,
                     const Ensemble& e) {
  int64_t n = 0;
  for (int q = 0; q < n_profiles; ++q)
    for (int32_t it = T_off[q]; it < T_off[q + 1]; ++it)
      for (int32_t ir = rho_off[q]; ir < rho_off[q + 1]; ++ir)
        n += guard_point_reaches(profiles[q], rho_cm[ir], T[it], e);
  return n;
}

int64_t guard_capacity(int64_t n_points, int32_t n_groups, int per_pair) {
  if (n_points <= 0) return 0;
  const int64_t c = n_points * n_groups * static_cast<int64_t>(per_pair);
  return c < 65536 ? 65536 : c;
}

cudaError_t launch_guard(cudaStream_t s, const GuardBufs& g, const Ensemble& e,
                         const Tile* tiles, const ProfileDev* profs, const double* rho,
                         double* partial, int num_sms, int64_t* launches) {
  if (!g.on) return cudaSuccess;
  guard_walk_kernel<<<num_sms * 4, 128, 0, s>>>(g, e.blocks, e.ppl, tiles, profs, rho);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  guard_fixup_kernel<<<num_sms, 128, 0, s>>>(g, partial);
  *launches += 2;
  return cudaGetLastError();
}

}  // namespace wln

namespace wln {

int guard_layout_bpg(wln_prec prec, int mode, int32_t n_loops, int32_t n_groups) {
  if (prec != WLN_PREC_FP32_COMP || mode != kModeSums) return 0;
  if (n_groups < 1 || n_loops % n_groups != 0) return 0;
  const int32_t lpg = n_loops / n_groups;
  return (lpg % 32 == 0 && lpg / 32 <= 64) ? lpg / 32 : 0;
}

bool guard_applies(const wln_ctx* ctx, wln_prec prec, int mode, int32_t n_loops,
                   int32_t n_groups, const wln_profile* profiles, int32_t n_profiles) {
  if (!ctx->guard || !guard_layout_bpg(prec, mode, n_loops, n_groups)) return false;
  for (int q = 0; q < n_profiles; ++q)
    if (profiles[q].kind == WLN_PROFILE_FLUX_TUBE) return true;
  return false;
}

}  // namespace wln
