// Wilson-loop kernel: for every (loop, point) the phase e * closed line
// integral of A and the spin integral e int B dtau of the scaled, shifted loop
// (paper Sec. "Wilson Loop", Eqs. rhoi-Ci; Sec. "Fermion Part", Eq.
// Wfermfpl), then W and its group sums (Sec. "Grouping Worldlines").
//
// Segment k of a loop runs from r_k to r_{k+1}, r = (rho_cm, 0) + sqrt(T) y.
// With d = r_{k+1} - r_k, Q(t) = lambda^2 + |r + t d|^2 = C t^2 + 2 B t + Q0:
//   C = |d|^2, B = r.d, X = r x d, D = lambda^2 C + X^2 (the discriminant,
//   by the Lagrange identity |r|^2 |d|^2 - (r.d)^2 = X^2),
//   int_0^1 dt/Q   = theta / sqrt(D),  theta = atan2(C sqrt(D), D + B (B + C))
//                  = atan2(sqrt(D), Q0 + B)  (Q0 C = D + B^2),
//   int_0^1 dt/Q^2 = [(C + B)/Q1 - B/Q0 + C int dt/Q] / (2 D), where
//   (C + B)/Q1 - B/Q0 = (D - B (B + C)) / (Q0 Q1) since Q1 = Q0 + 2B + C.
// The flux tube f = rho^2/(lambda^2 + rho^2) has f/rho^2 = 1/Q, so the phase
// of the segment is calF X int dt/Q, and e B = 2 calF lambda^2 / Q^2, so the
// segment's spin integral is (T/N) 2 calF lambda^2 int dt/Q^2.  Both are
// exact along the straight segment.  A constant field B gives phase B * area
// (half the sum of X) and spin B T.
//
// Work decomposition (GB300): a warp owns P radii at one T ("tile") and its
// 32 lanes are 32 loops (one "block" of the blocked ensemble).  A CTA of
// `warps` warps shares each staged block: TMA bulk copies bring chunks of
// the block's rows into a shared-memory ring guarded by mbarriers, and every
// warp walks them for its own tile, so each staged byte is used by
// warps * P points.  A work item is (chain of consecutive blocks, group of
// tiles); persistent CTAs take items round-robin so concurrent CTAs share a
// chain in L2.  W terms are reduced over lanes (and blocks) in FP64 in a
// fixed order into per-(chain, group) partials; a second kernel sums the
// partials of each group in chain order.
//
// Low-angle forms: with u = |d| / sqrt(Q0), tan(theta) <= u / (1 - u)
// (D <= Q0 C and B >= -sqrt(Q0) |d|).  Every ensemble carries, per 32-loop
// block, its longest segment and largest |y|, which bound u for every
// segment of the block at the warp's tile (T, rho, lambda).  For u <= 0.45
// (theta <= pi/4) the warp walks the block with the arctangent's low form,
// without the range fold and the octant unfolding (6 of the 17 operations of
// theta; the same bits); for u <= 0.045 (tan(theta) < 0.05) it takes
// int dt/Q = theta / sqrt(D) from three terms of the series of atan(t)/t,
// without 1/sqrt(D) (the spin then takes 1/D; the result moves by rounding
// only).  The choice is per block and the same on every
// lane, so the walk has no branch per segment: the row loop exists once per
// form (twice for the nested levels, whose long loop pays more for a third
// copy in instruction fetch than the series saves).
//
// Discretisation levels (Sec. "Estimating the Discretization Uncertainties"):
// the same pass can instead walk the three interleaved sub-loops of every
// loop -- circle (even points, N/2 of them), square (points 1 mod 4) and
// triangle (points 3 mod 4), N/4 each -- as closed polygons with proper time
// T/N' per segment, and combine their phases and spins into W at the levels
// N, N/2 and N/4.  A staged row (points 2i, 2i+1) feeds the circle with its
// even point and the square (i even) or the triangle (i odd) with its odd
// point, so the levels cost the same N segments per loop and radius.
#include <cfloat>

#include "wln_internal.cuh"

namespace wln {
namespace {

constexpr int kComps = WLN_K;
constexpr int kLevelComps = WLN_KL;

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on an mbarrier phase: gives up after limit_ns of wall time
// (2 s by default), or after 2^26 polls whatever the clock says.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          uint64_t limit_ns = 2000000000ull) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// ------------------------------------------------------ arithmetic flavours
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

// Angle of the point (x, y) with y > 0, in (0, pi).  With t = min(y,|x|) /
// max(y,|x|) in [0, 1], atan(t) = t + t^3 Q(t^2), Q the degree-7 minimax
// polynomial of gen_atan_poly.py (Remez exchange on the relative error:
// 1.7e-8 in exact arithmetic, within 1.3 float ulps as evaluated here);
// then the octant is unfolded: pi/2 - atan for y > |x|, pi - angle for x < 0.
// Inputs are finite with y > 0, so no special cases are needed.
__device__ __forceinline__ float atan_unit(float t) {
  const float s = t * t;
  float q = 0.002920693f;
  q = fmaf(q, s, -0.01636793f);
  q = fmaf(q, s, 0.043211866f);
  q = fmaf(q, s, -0.07552215f);
  q = fmaf(q, s, 0.106660046f);
  q = fmaf(q, s, -0.14211056f);
  q = fmaf(q, s, 0.19993773f);
  q = fmaf(q, s, -0.33333153f);
  return fmaf(t * s, q, t);
}

__device__ __forceinline__ float atan2_pos(float y, float x) {
  const float ax = fabsf(x);
  float r = atan_unit(fminf(y, ax) * rcp_approx(fmaxf(y, ax)));
  r = y > ax ? 1.5707963267948966f - r : r;
  return x < 0.0f ? 3.14159265358979323846f - r : r;
}

// The same angle when 0 < y <= x (at most pi/4): no octant to unfold, and
// bitwise equal to atan2_pos there.
__device__ __forceinline__ float atan2_low(float y, float x) {
  return atan_unit(y * rcp_approx(x));
}

// The angle when 0 < y <= 0.05 x: the Taylor series t - t^3/3 + t^5/5 of
// atan t, whose remainder (below t^7/7) is under 2.2e-9 of atan t there.
// (The walk's short-series form uses the same series for theta / sqrt(D)
// directly; this one serves walks that do not carry Q.)
__device__ __forceinline__ float atan2_tiny(float y, float x) {
  const float t = y * rcp_approx(x);
  const float s = t * t;
  return fmaf(t * s, fmaf(s, 0.2f, -0.333333343f), t);
}

// at2_form<1>: the angle when every segment of a block is known to subtend
// at most pi/4 at the field axis; at2_form<2>: at most atan(0.05) (kLowAngle:
// the flavour has these cheaper forms); at2_form<0> is the general angle.
struct F32Comp {
  using F = float;
  static constexpr bool kCompensated = true;
  static constexpr bool kLowAngle = true;
  __device__ static float rcp(float x) { return rcp_approx(x); }
  __device__ static float rsq(float x) { return rsqrt_approx(x); }
  template <int FORM>
  __device__ static float at2_form(float y, float x) {
    return FORM == 2 ? atan2_tiny(y, x) : (FORM == 1 ? atan2_low(y, x) : atan2_pos(y, x));
  }
};
struct F32Naive {
  using F = float;
  static constexpr bool kCompensated = false;
  static constexpr bool kLowAngle = true;
  __device__ static float rcp(float x) { return rcp_approx(x); }
  __device__ static float rsq(float x) { return rsqrt_approx(x); }
  template <int FORM>
  __device__ static float at2_form(float y, float x) {
    return FORM == 2 ? atan2_tiny(y, x) : (FORM == 1 ? atan2_low(y, x) : atan2_pos(y, x));
  }
};
struct F64 {
  using F = double;
  static constexpr bool kCompensated = false;
  static constexpr bool kLowAngle = false;
  __device__ static double rcp(double x) { return 1.0 / x; }
  __device__ static double rsq(double x) { return rsqrt(x); }
  template <int FORM>
  __device__ static double at2_form(double y, double x) { return atan2(y, x); }
};

// Sum of segment terms: terms are added plainly into `part`, and every few
// segments `fold` adds the partial into the running sum, with Kahan
// compensation in the compensated flavour (c holds the amount by which s
// exceeds the true sum).
template <class F, bool kComp>
struct Acc {
  F s, c, part;
  __device__ __forceinline__ void zero() { s = F(0); c = F(0); part = F(0); }
  __device__ __forceinline__ void add(F x) { part += x; }
  __device__ __forceinline__ void fold() {
    if (kComp) {
      const F y = part - c;
      const F t = s + y;
      c = (t - s) - y;
      s = t;
    } else {
      s += part;
    }
    part = F(0);
  }
};

// ----------------------------------------------------------- kernel params
struct KParams {
  const float4* blocks;
  int32_t n_blocks, ppl, n_loops;
  const Tile* tiles;
  int32_t n_tiles;
  const ProfileDev* profs;
  const double* rho;
  int32_t lpg, G;
  double* partial;       // [(n_chains + G)][n_points][K]
  int64_t n_points;
  int32_t rows;          // float4 rows per chunk
  int32_t stages;
  int32_t chain;
  int32_t n_tile_groups, n_chains;
  int64_t n_items;
  int* flag;
  double* loops_out;     // per-loop mode: [n_points][n_loops][2]
  const float2* stats;   // per block: longest segment, largest |y|
  int32_t low_angle;     // highest form of theta a block may take (0: general everywhere)
};

// Whether every segment of block b subtends at most pi/4 at the field axis
// for the warp's tile, i.e. theta <= pi/4, i.e. sqrt(D) <= Q0 + B.  With |d|
// the segment, D <= Q0 C = Q0 |d|^2 (Lagrange) and B >= -|r| |d| >= -sqrt(Q0)
// |d|, so 2 |d| <= sqrt(Q0) is enough, and Q0 >= lambda^2 + (rho -
// sqrt(T) |y|_max)^2 for rho > sqrt(T) |y|_max.  The segments are sqrt(T)
// times the unit loop's (up to span of them for a sub-loop), and a margin of
// 0.9 keeps the float comparison of the two sides on the same side.  Every
// lane computes the same answer from the same block statistics.
// The same bound gives t = tan(theta) <= u / (1 - u), u = |d| / sqrt(Q0);
// for u <= 0.045, t < 0.05 and three terms of the series of atan t suffice.
// Returns the form of theta for the block: 2, 1 or 0 (general).  (In float:
// the margins are far above its rounding.)
struct LowAngle {
  float two_span_sT, sT, rho_min, l2;
  __device__ __forceinline__ int block(const KParams& k, int b) const {
    const float2 st = k.stats[b];
    const float gap = fmaxf(0.0f, rho_min - sT * st.y);
    const float lhs = two_span_sT * st.x, rhs = sqrtf(l2 + gap * gap);
    return lhs <= 0.09f * rhs ? 2 : (lhs <= 0.9f * rhs ? 1 : 0);
  }
};

// Per-lane walk of one loop for the P radii of a tile (flux tube).  CQ
// carries Q at the current point so that theta = atan2(sqrt(D), Q0 + B)
// (one multiply fewer per segment and radius, one register more per radius);
// without it theta = atan2(C sqrt(D), D + B (B + C)).  step_<1> may be used
// when every segment subtends at most pi/4 at the axis, step_<2> when at most
// atan(0.05) (the caller has checked): theta then needs no octant unfolding,
// and in the second case only three terms of its series.
template <class A, int P, bool CQ = true>
struct Walk {
  using F = typename A::F;
  F s, l2;           // sqrt(T), lambda^2
  F rho[P];
  // state at the current point
  F ux, uy;          // unit-loop point
  F ry;              // scaled y (shared by the radii)
  F rx[P];           // shifted, scaled x
  F q[P], rq[P];     // Q and 1/Q at the current point
  Acc<F, A::kCompensated> ph[P], sp[P];

  __device__ __forceinline__ void start(F x0, F y0) {
    ux = x0; uy = y0;
    ry = s * y0;
    const F e0 = fma(ry, ry, l2);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      rx[p] = fma(s, x0, rho[p]);
      const F q0 = fma(rx[p], rx[p], e0);
      if (CQ) q[p] = q0;
      rq[p] = A::rcp(q0);
      ph[p].zero();
      sp[p].zero();
    }
  }

  // Advance along the straight segment to unit-loop point (x1, y1).
  __device__ __forceinline__ void step(F x1, F y1) { step_<0>(x1, y1); }

  template <int FORM>
  __device__ __forceinline__ void step_(F x1, F y1) {
    const F dx = s * (x1 - ux), dy = s * (y1 - uy);
    const F C = fma(dx, dx, dy * dy);
    const F l2C = l2 * C;
    const F ry1 = s * y1;
    const F e1 = fma(ry1, ry1, l2);
    const F rydy = ry * dy, rydx = ry * dx;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const F rx1 = fma(s, x1, rho[p]);
      const F q1 = fma(rx1, rx1, e1);
      const F rq1 = A::rcp(q1);
      const F B = fma(rx[p], dx, rydy);
      const F X = fma(rx[p], dy, -rydx);
      const F D = fma(X, X, l2C);
      const F BC = B + C;
      if constexpr (FORM == 2 && CQ) {
        // tan(theta) = t < 0.05 with t^2 = D r^2, r = 1/(Q0 + B): int dt/Q =
        // theta / sqrt(D) = r atan(t) / t = r (1 - t^2/3 + t^4/5), without
        // 1/sqrt(D); the spin takes 1/D instead.
        const F r = A::rcp(q[p] + B);
        const F t2 = D * (r * r);
        const F J1 = r * fma(t2, fma(t2, F(0.2), F(-0.333333343)), F(1));
        ph[p].add(X * J1);
        const F br = fma(fma(-B, BC, D) * rq[p], rq1, C * J1);
        sp[p].add(br * A::rcp(D));
      } else {
        const F rsD = A::rsq(D);
        // atan2(C sqrt(D), D + B (B + C)) with the common factor C removed:
        // Q0 C = D + B^2 (Lagrange), so D + B (B + C) = C (Q0 + B).
        const F ya = CQ ? D * rsD : C * (D * rsD);
        const F xa = CQ ? q[p] + B : fma(B, BC, D);
        const F theta = A::template at2_form<FORM>(ya, xa);
        const F J1 = theta * rsD;
        ph[p].add(X * J1);
        // (C + B)/Q1 - B/Q0 = (D - B (B + C)) / (Q0 Q1), free of the
        // cancellation between the two quotients.
        const F br = fma(fma(-B, BC, D) * rq[p], rq1, C * J1);
        sp[p].add(br * (rsD * rsD));
      }
      rx[p] = rx1;
      if (CQ) q[p] = q1;
      rq[p] = rq1;
    }
    ux = x1; uy = y1; ry = ry1;
  }

  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int p = 0; p < P; ++p) { ph[p].fold(); sp[p].fold(); }
  }

  // Raw phase and spin sums of radius p (sum and compensation terms).
  __device__ __forceinline__ void raw(int p, double& ps, double& pc, double& ss,
                                      double& sc) const {
    ps = ph[p].s; pc = ph[p].c; ss = sp[p].s; sc = sp[p].c;
  }
};

// Constant field: only the area is needed, half the sum of X = r x d.
template <class A, int P>
struct WalkB {
  using F = typename A::F;
  F s, l2;
  F rho[P];
  F ux, uy, ry;
  F rx[P];
  Acc<F, A::kCompensated> ph[P];
  __device__ __forceinline__ void start(F x0, F y0) {
    ux = x0; uy = y0; ry = s * y0;
#pragma unroll
    for (int p = 0; p < P; ++p) { rx[p] = fma(s, x0, rho[p]); ph[p].zero(); }
  }
  __device__ __forceinline__ void step(F x1, F y1) { step_<0>(x1, y1); }
  template <int FORM>
  __device__ __forceinline__ void step_(F x1, F y1) {
    const F dx = s * (x1 - ux), dy = s * (y1 - uy);
    const F rydx = ry * dx;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      ph[p].add(fma(rx[p], dy, -rydx));
      rx[p] = fma(s, x1, rho[p]);
    }
    ux = x1; uy = y1; ry = s * y1;
  }
  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int p = 0; p < P; ++p) ph[p].fold();
  }
  // The spin integral of a constant field is B T: a unit "sum" times B T.
  __device__ __forceinline__ void raw(int p, double& ps, double& pc, double& ss,
                                      double& sc) const {
    ps = ph[p].s; pc = ph[p].c; ss = 1.0; sc = 0.0;
  }
};

// Split of a double into two floats (hi + lo) for double-float products.
struct F2 {
  float hi, lo;
};
__device__ __forceinline__ F2 split(double x) {
  const float h = static_cast<float>(x);
  return F2{h, static_cast<float>(x - static_cast<double>(h))};
}

// (s - c) * k for a compensated float sum (s, c) and k = k.hi + k.lo, as
// hi + lo with hi = fl(s k.hi) and lo the rounding error plus the small
// terms: accurate to a few units in the last place of the double result.
__device__ __forceinline__ F2 scaled(float s, float c, F2 k) {
  const float hi = s * k.hi;
  const float e = fmaf(s, k.hi, -hi);
  return F2{hi, e + fmaf(s, k.lo, -c * k.hi)};
}

// cosh(x) - 1 = 2 sinh^2(x/2): no cancellation at small x, +inf (not NaN)
// once cosh(x) leaves the double range.
__device__ __forceinline__ double cosh_m1_f64(double x) {
  const double h = sinh(0.5 * x);
  return 2.0 * h * h;
}

// The five per-loop terms (see WLN_C_*).
//  FP64: phase reduced in turns in double, everything in double.
//  FP32 compensated: phase and spin arrive as compensated sums times a
//   double scale, formed as double-float; the fractional turn is exact to
//   float rounding, so sin/cos are taken on |frac| <= 1/2 with sinpi/cospi.
//   cosh(spin) - 1 uses expm1f of |spin| (cosh is even) plus the
//   first-order term of the low part; spins above 80 (cosh beyond float
//   range) go through double.
//  FP32 naive: plain float phase in radians, cosf and coshf.
template <class A>
__device__ __forceinline__ void wilson_terms(double ph_s, double ph_c, double sp_s, double sp_c,
                                             F2 tp, F2 st, double tp_d, double st_d,
                                             double* w) {
  if constexpr (sizeof(typename A::F) == 8) {
    const double turns = ph_s * tp_d;
    const double fr = turns - rint(turns);
    const double h = sinpi(fr);
    const double scal_m1 = -2.0 * h * h;
    double sn, cs;
    sincospi(2.0 * fr, &sn, &cs);
    const double ferm_m1 = cs * cosh_m1_f64(sp_s * st_d) + scal_m1;
    w[0] = scal_m1; w[1] = ferm_m1; w[2] = sn;
    w[3] = scal_m1 * scal_m1; w[4] = ferm_m1 * ferm_m1;
  } else if constexpr (A::kCompensated) {
    const F2 t = scaled(static_cast<float>(ph_s), static_cast<float>(ph_c), tp);
    const float fr = (t.hi - rintf(t.hi)) + t.lo;
    const float h = sinpif(fr);
    const float scal_m1 = -2.0f * h * h;
    float sn, cs;
    sincospif(2.0f * fr, &sn, &cs);
    F2 sv = scaled(static_cast<float>(sp_s), static_cast<float>(sp_c), st);
    // cosh is even: evaluate at |spin| (a negative flux or field gives a
    // negative spin, and expm1 of a large negative argument reaches -1)
    // (a multiply by the sign, not a branch: the branch cost the pass 2%)
    const float sgn = copysignf(1.0f, sv.hi);
    sv.hi *= sgn;
    sv.lo *= sgn;
    double ferm_m1;
    if (sv.hi < 80.0f) {
      const float em1 = expm1f(sv.hi);
      const float inv = 1.0f / (em1 + 1.0f);
      const float sinh_v = 0.5f * (em1 + em1 * inv);
      const float cm1 = fmaf(sinh_v, sv.lo, 0.5f * em1 * (em1 * inv));
      ferm_m1 = static_cast<double>(fmaf(cs, cm1, scal_m1));
    } else {
      ferm_m1 = static_cast<double>(cs) *
                    cosh_m1_f64(static_cast<double>(sv.hi) + static_cast<double>(sv.lo)) +
                static_cast<double>(scal_m1);
    }
    const double sm = scal_m1;
    w[0] = sm; w[1] = ferm_m1; w[2] = sn;
    w[3] = sm * sm; w[4] = ferm_m1 * ferm_m1;
  } else {
    const float ph = static_cast<float>(ph_s) * static_cast<float>(6.283185307179586 * tp_d);
    float sn, cs;
    sincosf(ph, &sn, &cs);
    const float scal_m1 = cs - 1.0f;
    const float ferm_m1 = cs * coshf(static_cast<float>(sp_s) * static_cast<float>(st_d)) - 1.0f;
    w[0] = scal_m1; w[1] = ferm_m1; w[2] = sn;
    w[3] = static_cast<double>(scal_m1) * scal_m1;
    w[4] = static_cast<double>(ferm_m1) * ferm_m1;
  }
}

// Shared pipeline state of a CTA: a ring of staged chunks with full/empty
// mbarriers; thread 0 also refills it.
struct Pipe {
  float4* ring;
  uint64_t* full;
  uint64_t* empty;
  int stages, chunk_rows, chunks_per_block, rows_per_block;
  uint32_t chunk_bytes;
  int32_t kc = 0, issued = 0, total = 0;
  int32_t prod_item = 0;
  int prod_blk = 0, prod_chunk = 0;
};

__device__ __forceinline__ int blocks_in_item(const KParams& k, int64_t item) {
  const int c = static_cast<int>(item / k.n_tile_groups);
  const int b0 = c * k.chain;
  return min(b0 + k.chain, k.n_blocks) - b0;
}

__device__ __forceinline__ void issue_next(const KParams& k, Pipe& pp, int slot) {
  const int c = static_cast<int>(pp.prod_item / k.n_tile_groups);
  const int b = c * k.chain + pp.prod_blk;
  const float4* src = k.blocks + (static_cast<size_t>(b) * pp.rows_per_block +
                                  static_cast<size_t>(pp.prod_chunk) * pp.chunk_rows) * 32;
  mbar_arrive_expect_tx(&pp.full[slot], pp.chunk_bytes);
  bulk_load(pp.ring + static_cast<size_t>(slot) * pp.chunk_rows * 32, src, pp.chunk_bytes,
            &pp.full[slot]);
  ++pp.issued;
  if (++pp.prod_chunk == pp.chunks_per_block) {
    pp.prod_chunk = 0;
    if (++pp.prod_blk == blocks_in_item(k, pp.prod_item)) {
      pp.prod_blk = 0;
      pp.prod_item += gridDim.x;
    }
  }
}

// Phase and spin sums of one walk at radius p, as true sums (s - c) in
// double; the spin scaled by m (the walk's N / N').
template <class WalkT>
__device__ __forceinline__ void walk_sums(const WalkT& w, int p, double m, double& ph,
                                          double& sp) {
  double ps, pc, ss, sc;
  w.raw(p, ps, pc, ss, sc);
  ph = ps - pc;
  sp = (ss - sc) * m;
}

// W - 1 (scalar, spinor) of one level from its phase and spin sums.  The
// float flavours take the sums as a float pair (hi - lo = the double sum).
template <class A>
__device__ __forceinline__ void level_terms(double ph, double sp, F2 tp, F2 st, double tp_d,
                                            double st_d, double* out) {
  double w[kComps];
  if constexpr (sizeof(typename A::F) == 8) {
    wilson_terms<A>(ph, 0.0, sp, 0.0, tp, st, tp_d, st_d, w);
  } else {
    const float ph_hi = static_cast<float>(ph), sp_hi = static_cast<float>(sp);
    wilson_terms<A>(ph_hi, static_cast<float>(static_cast<double>(ph_hi) - ph), sp_hi,
                    static_cast<float>(static_cast<double>(sp_hi) - sp), tp, st, tp_d, st_d, w);
  }
  out[0] = w[0];
  out[1] = w[1];
}

// One work item for one warp: its tile against every loop of the chain.
// The rows of one staged chunk from row r on, with theta in form FORM
// (0: general, 1: at most pi/4, 2: at most atan(0.05)).
// Whole loops: a row holds two consecutive points.
template <int FORM, class WalkT>
__device__ __forceinline__ void rows_plain(WalkT* w, const float4* rowp, int r, int n) {
  for (; r < n; ++r) {
    const float4 v = rowp[r * 32];
    w[0].template step_<FORM>(v.x, v.y);
    w[0].template step_<FORM>(v.z, v.w);
    if ((r & 3) == 3) w[0].fold();   // every 8 segments
  }
}

// Nested loops: rows in pairs hold points 4j .. 4j + 3; the full walk takes
// all four, the even walk 4j and 4j + 2, the quarter walk 4j.
template <int FORM, class WalkT>
__device__ __forceinline__ void rows_nested(WalkT* w, const float4* rowp, int r, int n) {
  for (; r < n; r += 2) {
    const float4 a = rowp[r * 32], v = rowp[(r + 1) * 32];
    w[0].template step_<FORM>(a.x, a.y);
    w[0].template step_<FORM>(a.z, a.w);
    w[0].template step_<FORM>(v.x, v.y);
    w[0].template step_<FORM>(v.z, v.w);
    w[1].template step_<FORM>(a.x, a.y);
    w[1].template step_<FORM>(v.x, v.y);
    w[2].template step_<FORM>(a.x, a.y);
    if ((r & 3) == 2) {   // every 8 segments of the full walk
      w[0].fold(); w[1].fold(); w[2].fold();
    }
  }
}

// The paper's sub-loops: row r even holds points 2r (circle) and 2r + 1 =
// 1 mod 4 (square), row r + 1 holds 2r + 2 (circle) and 2r + 3 = 3 mod 4
// (triangle).
template <int FORM, class WalkT>
__device__ __forceinline__ void rows_levels(WalkT* w, const float4* rowp, int r, int n) {
  for (; r < n; r += 2) {
    const float4 a = rowp[r * 32], v = rowp[(r + 1) * 32];
    w[0].template step_<FORM>(a.x, a.y);
    w[1].template step_<FORM>(a.z, a.w);
    w[0].template step_<FORM>(v.x, v.y);
    w[2].template step_<FORM>(v.z, v.w);
    if ((r & 7) == 6) {   // every 8 circle segments
      w[0].fold(); w[1].fold(); w[2].fold();
    }
  }
}

// Per-lane W terms are added into the warp's shared-memory accumulators
// acc[j][lane] (j = radius * K + component, rows padded to 33 doubles); a
// flush sums each row over the lanes in lane order and writes the partial
// of (chain, group).  MODE kModeLevels walks the circle, square and triangle
// sub-loops (w[0..2], K = WLN_KL); kModeNested the loop through all points,
// the even points and the points 0 mod 4; kModeLoops writes every loop's
// W - 1 to global memory instead of accumulating (lanes store 32
// consecutive loops).
template <class A, int P, class WalkT, int MODE>
__device__ bool run_item(const KParams& k, Pipe& pp, double* acc, int c, const Tile& tile,
                         const ProfileDev& prof, bool active, volatile int* abort_flag,
                         int lane) {
  using F = typename A::F;
  constexpr bool LV = level_mode(MODE);
  constexpr bool NEST = MODE == kModeNested;
  constexpr bool PL = MODE == kModeLoops;
  constexpr int K = LV ? kLevelComps : kComps;
  constexpr int NW = LV ? 3 : 1;
  constexpr int V = P * K;
  WalkT w[NW];
#pragma unroll
  for (int q = 0; q < NW; ++q) {
    w[q].s = static_cast<F>(sqrt(tile.T));
    w[q].l2 = static_cast<F>(prof.l2);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const int i = p < tile.n_valid ? p : (tile.n_valid > 0 ? tile.n_valid - 1 : 0);
      w[q].rho[p] = static_cast<F>(k.rho[tile.rho0 + i]);
    }
  }
  const double st_d = prof.spin_per * tile.T;
  const F2 tp = split(prof.turns_per), st = split(st_d);
  // sub-loop segments join points up to 4 apart
  double rho_min = k.rho[tile.rho0];
  for (int p = 1; p < tile.n_valid; ++p) rho_min = fmin(rho_min, k.rho[tile.rho0 + p]);
  const LowAngle la{static_cast<float>(2.0 * (LV ? 4.0 : 1.0) * sqrt(tile.T)),
                    static_cast<float>(sqrt(tile.T)), static_cast<float>(rho_min),
                    static_cast<float>(prof.l2)};
  const bool la_ok =
      A::kLowAngle && k.low_angle && prof.kind == WLN_PROFILE_FLUX_TUBE && tile.n_valid > 0;
  const int b0 = c * k.chain;
  const int b1 = min(b0 + k.chain, k.n_blocks);
  int g_cur = (b0 * 32) / k.lpg;

  auto flush = [&](int g) {
    if (PL) return;
    __syncwarp();
    if (active) {
      double* dst = k.partial + tile.part_base +
                    (static_cast<size_t>(c + g) * tile.part_stride + tile.p0) * K;
      for (int j = lane; j < V; j += 32) {
        double sum = 0.0;
        const double* row = acc + j * 33;
#pragma unroll 8
        for (int l = 0; l < 32; ++l) sum += row[l];
        if (j / K < tile.n_valid) dst[j] = sum;
      }
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < V; ++j) acc[j * 33 + lane] = 0.0;
    __syncwarp();
  };

  for (int b = b0; b < b1; ++b) {
    const int loop = b * 32 + lane;
    const bool valid = loop < k.n_loops;
    const int form = la_ok ? min(la.block(k, b), k.low_angle) : 0;   // the same on every lane
    // first point of each walk, for the closing segments
    float fx[NW], fy[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q) { fx[q] = 0.f; fy[q] = 0.f; }
    for (int ch = 0; ch < pp.chunks_per_block; ++ch) {
      const int slot = static_cast<int>(pp.kc % pp.stages);
      const uint32_t parity = static_cast<uint32_t>((pp.kc / pp.stages) & 1);
      // every lane of the warp takes the same decision (the warp's
      // shuffles and syncs need all 32 lanes)
      if (!__all_sync(0xffffffffu, mbar_wait(&pp.full[slot], parity))) {
        if (lane == 0) atomicExch(k.flag, kErrTimeoutFull);
        *abort_flag = 1;
        return false;
      }
      const float4* rowp = pp.ring + static_cast<size_t>(slot) * pp.chunk_rows * 32 + lane;
      if (active) {
        if constexpr (!LV) {
          int r = 0;
          if (ch == 0) {
            const float4 v = rowp[0];
            fx[0] = v.x; fy[0] = v.y;
            w[0].start(v.x, v.y);
            w[0].step(v.z, v.w);
            r = 1;
          }
          // the form of theta for this block is the same on every lane
          if (form == 2) rows_plain<2>(w, rowp, r, pp.chunk_rows);
          else if (form == 1) rows_plain<1>(w, rowp, r, pp.chunk_rows);
          else rows_plain<0>(w, rowp, r, pp.chunk_rows);
        } else if constexpr (NEST) {
          // Rows in pairs hold points 4j .. 4j + 3: the full walk takes all
          // four, the even walk 4j and 4j + 2, the quarter walk 4j.  All three
          // start at point 0 and close back to it.
          int r = 0;
          if (ch == 0) {
            const float4 a = rowp[0], v = rowp[32];
#pragma unroll
            for (int q = 0; q < NW; ++q) { fx[q] = a.x; fy[q] = a.y; }
            w[0].start(a.x, a.y);
            w[0].step(a.z, a.w);
            w[0].step(v.x, v.y);
            w[0].step(v.z, v.w);
            w[1].start(a.x, a.y);
            w[1].step(v.x, v.y);
            w[2].start(a.x, a.y);
            r = 2;
          }
          // two copies only: a third of this long loop costs more in
          // instruction fetch than the short series saves
          if (form >= 1) rows_nested<1>(w, rowp, r, pp.chunk_rows);
          else rows_nested<0>(w, rowp, r, pp.chunk_rows);
        } else {
          // Rows come in pairs (chunk_rows is even): row r even holds points
          // 2r (circle) and 2r + 1 = 1 mod 4 (square), row r + 1 holds
          // 2r + 2 (circle) and 2r + 3 = 3 mod 4 (triangle).
          int r = 0;
          if (ch == 0) {
            const float4 a = rowp[0], v = rowp[32];
            fx[0] = a.x; fy[0] = a.y; fx[1] = a.z; fy[1] = a.w; fx[2] = v.z; fy[2] = v.w;
            w[0].start(a.x, a.y);
            w[1].start(a.z, a.w);
            w[0].step(v.x, v.y);
            w[2].start(v.z, v.w);
            r = 2;
          }
          if (form == 2) rows_levels<2>(w, rowp, r, pp.chunk_rows);
          else if (form == 1) rows_levels<1>(w, rowp, r, pp.chunk_rows);
          else rows_levels<0>(w, rowp, r, pp.chunk_rows);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&pp.empty[slot]);
      if (threadIdx.x == 0 && pp.issued < pp.total) {
        // The slot just released is the next one to refill.
        if (!mbar_wait(&pp.empty[slot], parity)) {
          atomicExch(k.flag, kErrTimeoutEmpty);
          *abort_flag = 1;
        } else {
          issue_next(k, pp, slot);
        }
      }
      ++pp.kc;
      if (__any_sync(0xffffffffu, *abort_flag != 0)) return false;
    }
    if (!active) continue;
#pragma unroll
    for (int q = 0; q < NW; ++q) {
      w[q].step(fx[q], fy[q]);  // closing segment back to the walk's first point
      w[q].fold();
    }
    if constexpr (PL) {
      if (valid) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          if (p < tile.n_valid) {
            double ps, pc, ss, sc, t[kComps];
            w[0].raw(p, ps, pc, ss, sc);
            wilson_terms<A>(ps, pc, ss, sc, tp, st, prof.turns_per, st_d, t);
            // evict-first store: the results stream past L2 without pushing
            // out the loop chain the CTAs are sweeping
            __stcs(reinterpret_cast<double2*>(k.loops_out) +
                       static_cast<int64_t>(tile.p0 + p) * k.n_loops + loop,
                   make_double2(t[0], t[1]));
          }
        }
      }
      continue;
    }
    const int g_lane = valid ? loop / k.lpg : -1;
    const int g_lo = (b * 32) / k.lpg;
    const int g_hi = min(b * 32 + 31, k.n_loops - 1) / k.lpg;
    for (int g = g_lo; g <= g_hi; ++g) {
      if (g != g_cur) { flush(g_cur); g_cur = g; }
      const bool mine = g_lane == g;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        if constexpr (!LV) {
          double ps, pc, ss, sc, t[K];
          w[0].raw(p, ps, pc, ss, sc);
          wilson_terms<A>(ps, pc, ss, sc, tp, st, prof.turns_per, st_d, t);
#pragma unroll
          for (int q = 0; q < K; ++q)
            if (mine) acc[(p * K + q) * 33 + lane] += t[q];
        } else {
          // Spin per segment is T/N' on a sub-loop of N' points: the circle's
          // sums count twice, the square's and triangle's four times, of the
          // full loop's T/N (a constant field's spin is B T on every loop);
          // the nested walks of N, N/2 and N/4 points count 1, 2 and 4 times.
          const bool tube = prof.kind != WLN_PROFILE_CONST_B;
          double po, so, pq, sq, pt, stt;
          walk_sums(w[0], p, tube ? (NEST ? 1.0 : 2.0) : 1.0, po, so);
          walk_sums(w[1], p, tube ? (NEST ? 2.0 : 4.0) : 1.0, pq, sq);
          walk_sums(w[2], p, tube ? 4.0 : 1.0, pt, stt);
          // Paper's levels: W_N = e^{i (circ/2 + sq/4 + tri/4)}, W_N/2 = e^{i circ},
          // W_N/4 = e^{i (sq + tri)/2}, the spins combined the same way.  Nested
          // levels: each walk is its own level.  One copy of the W arithmetic
          // serves the three levels (registers).
#pragma unroll 1
          for (int L = 0; L < 3; ++L) {
            double ph, sp;
            if (NEST) {
              ph = L == 0 ? po : (L == 1 ? pq : pt);
              sp = L == 0 ? so : (L == 1 ? sq : stt);
            } else {
              ph = L == 0 ? 0.5 * po + 0.25 * (pq + pt) : (L == 1 ? po : 0.5 * (pq + pt));
              sp = L == 0 ? 0.5 * so + 0.25 * (sq + stt) : (L == 1 ? so : 0.5 * (sq + stt));
            }
            double t[2];
            level_terms<A>(ph, sp, tp, st, prof.turns_per, st_d, t);
            if (mine) {
              acc[(p * K + 2 * L) * 33 + lane] += t[0];
              acc[(p * K + 2 * L + 1) * 33 + lane] += t[1];
            }
          }
        }
      }
    }
  }
  flush(g_cur);
  return true;
}

// Resident CTAs per SM the register budget is sized for (65536 registers a
// SM): the level pass (three walks per radius) and 8 radii per lane run 8
// warps per SM with up to 255 registers; 4 radii in CTAs of 4 warps run 12
// warps with up to 168; the other shapes 16 warps with up to 128.  Measured
// on the paper workload: 4 radii x 4 warps x 3 CTAs 664 ms, 8 radii x 8 warps
// x 1 CTA 659 ms, 4 radii x 8 warps x 2 CTAs 682 ms (spilling); the level
// pass 3 radii x 4 warps x 2 CTAs 757 ms, 4 x 8 x 1 774 ms.
constexpr int min_ctas(int P, int warps, int mode) {
  return (level_mode(mode) || P >= 8) ? 256 / (warps * 32)
                                         : (P == 4 && warps == 4) ? 3 : 512 / (warps * 32);
}

template <class A, int P, int WARPS, int MODE>
__global__ void __launch_bounds__(WARPS * 32, min_ctas(P, WARPS, MODE)) wilson_kernel(const KParams k) {
  constexpr int K = level_mode(MODE) ? kLevelComps : kComps;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int abort_flag;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Pipe pp;
  pp.rows_per_block = k.ppl / 2;
  pp.chunk_rows = k.rows < pp.rows_per_block ? k.rows : pp.rows_per_block;
  pp.chunks_per_block = pp.rows_per_block / pp.chunk_rows;
  pp.chunk_bytes = static_cast<uint32_t>(pp.chunk_rows) * 512u;
  pp.stages = k.stages;
  pp.ring = reinterpret_cast<float4*>(smem);
  const size_t ring_bytes = static_cast<size_t>(k.stages) * pp.chunk_rows * 512;
  double* acc = reinterpret_cast<double*>(smem + ring_bytes) + warp * (P * K * 33);
  pp.full = reinterpret_cast<uint64_t*>(smem + ring_bytes + WARPS * P * K * 33 * sizeof(double));
  pp.empty = pp.full + k.stages;
  for (int j = 0; j < P * K; ++j) acc[j * 33 + lane] = 0.0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < k.stages; ++s) {
      mbar_init(&pp.full[s], 1);
      mbar_init(&pp.empty[s], WARPS);
    }
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  for (int64_t it = blockIdx.x; it < k.n_items; it += gridDim.x)
    pp.total += blocks_in_item(k, it) * pp.chunks_per_block;
  pp.prod_item = blockIdx.x;
  if (threadIdx.x == 0) {
    for (int s = 0; s < k.stages && pp.issued < pp.total; ++s) issue_next(k, pp, s);
  }

  bool ok = true;
  for (int64_t item = blockIdx.x; item < k.n_items && ok; item += gridDim.x) {
    const int c = static_cast<int>(item / k.n_tile_groups);
    const int tg = static_cast<int>(item % k.n_tile_groups);
    const int t = tg * WARPS + warp;
    const Tile tile = k.tiles[t < k.n_tiles ? t : 0];
    const bool active = t < k.n_tiles && tile.n_valid > 0;   // n_valid 0: padding
    const ProfileDev prof = k.profs[tile.profile];
    // three walks per radius: Q fits in registers for up to 3 radii per lane
    constexpr bool CQ = !level_mode(MODE) || P <= 3;
    if (prof.kind == WLN_PROFILE_CONST_B)
      ok = run_item<A, P, WalkB<A, P>, MODE>(k, pp, acc, c, tile, prof, active, &abort_flag, lane);
    else
      ok = run_item<A, P, Walk<A, P, CQ>, MODE>(k, pp, acc, c, tile, prof, active, &abort_flag,
                                                lane);
  }

  if (!ok && threadIdx.x == 0) {
    // Let copies already in flight land before the CTA's shared memory goes away.
    for (int32_t q = pp.kc; q < pp.issued; ++q)
      (void)mbar_wait(&pp.full[q % pp.stages], static_cast<uint32_t>((q / pp.stages) & 1));
  }
}

// Failure-detection self-test: wait on an mbarrier phase that nothing will
// complete, with the same bounded wait the Wilson kernel uses; when the wait
// runs out the kernel records it in the device error flag and returns.
__global__ void selftest_wait_kernel(int* flag, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0, limit_ns)) atomicExch(flag, kErrTimeoutSelfTest);
}

// Sum the partials of each group over its chains, in chain order.
__global__ void reduce_partials_kernel(const double* partial, int64_t n_points, int32_t G,
                                       int32_t lpg, int32_t chain_loops, int32_t K,
                                       double* out) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n_points * G * K) return;
  const int q = static_cast<int>(i % K);
  const int g = static_cast<int>((i / K) % G);
  const int64_t p = i / (static_cast<int64_t>(K) * G);
  const int c_lo = static_cast<int>((static_cast<int64_t>(g) * lpg) / chain_loops);
  const int c_hi = static_cast<int>((static_cast<int64_t>(g + 1) * lpg - 1) / chain_loops);
  double s = 0.0;
  for (int c = c_lo; c <= c_hi; ++c)
    s += partial[(static_cast<size_t>(c + g) * n_points + p) * K + q];
  out[i] = s;
}

template <class A, int P, int WARPS, int MODE>
cudaError_t launch_t(cudaStream_t s, const KParams& kp, int grid, size_t smem) {
  auto kern = wilson_kernel<A, P, WARPS, MODE>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
  if (err != cudaSuccess) return err;
  kern<<<grid, WARPS * 32, smem, s>>>(kp);
  return cudaGetLastError();
}

template <class A, int P, int WARPS, int MODE>
int occupancy(size_t smem) {
  int n = 0;
  auto kern = wilson_kernel<A, P, WARPS, MODE>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess)
    return 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, WARPS * 32, smem) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

size_t smem_bytes(const WilsonPlan& p, int ppl) {
  const int chunk_rows = p.rows < ppl / 2 ? p.rows : ppl / 2;
  const int K = level_mode(p.mode) ? kLevelComps : kComps;
  return static_cast<size_t>(p.stages) * chunk_rows * 512 +
         static_cast<size_t>(p.warps) * p.P * K * 33 * sizeof(double) +
         2 * p.stages * sizeof(uint64_t);
}

}  // namespace

// Tuning applies to the float flavours; the FP64 comparison path keeps its
// own shape (2 radii per lane, 4 warps).  The discretisation levels run three
// walks per radius (4 radii per lane, FP64 1) and ignore the tuning of the
// plain pass.
int plan_points_per_lane(const wln_ctx* ctx, wln_prec prec, int mode) {
  if (level_mode(mode)) return prec == WLN_PREC_FP64 ? 1 : 3;
  if (mode == kModeLoops) return prec == WLN_PREC_FP64 ? 2 : 4;
  if (prec == WLN_PREC_FP64) return 2;
  return ctx->tune_P ? ctx->tune_P : 4;
}

WilsonPlan make_plan(const wln_ctx* ctx, const Ensemble& e, int n_tiles, wln_prec prec,
                     int mode) {
  WilsonPlan p{};
  p.P = plan_points_per_lane(ctx, prec, mode);
  p.mode = mode;
  p.low_angle = ctx->low_angle;
  const bool f64 = prec == WLN_PREC_FP64;
  const bool fixed = f64 || mode != kModeSums;   // shapes that ignore the tuning
  // Group sums: 4 radii x 8 warps, 2 CTAs per SM, 64-row chunks, 2 stages
  // (537 ms on the paper workload against 560 ms for 4 x 4 warps, 3 CTAs per
  // SM, 32 rows, 3 stages, once the low-angle forms made the walk lighter).
  // Per-loop values keep (4, 4); the levels (3, 4), 2 CTAs per SM.
  const bool wide = !fixed && p.P == 4;
  const int def_warps = (level_mode(mode) || (p.P == 4 && !wide)) ? 4 : 8;
  p.warps = f64 ? 4 : ((!fixed && ctx->tune_warps) ? ctx->tune_warps : def_warps);
  p.rows = (!fixed && ctx->tune_rows) ? ctx->tune_rows : (wide ? 64 : 32);
  p.stages = (!fixed && ctx->tune_stages) ? ctx->tune_stages : (wide ? 2 : 3);
  p.n_tiles = n_tiles;
  p.n_tile_groups = (n_tiles + p.warps - 1) / p.warps;
  if (ctx->tune_chain && !fixed) {
    p.chain = ctx->tune_chain;
  } else {
    // Enough items to keep every SM busy with a small tail, few partials;
    // then short enough chains that the one every CTA is sweeping stays in L2
    // (all CTAs work on the same chain at a time): measured on the paper
    // workload, 42 MB chains read the ensemble 2.9x from DRAM, 10 MB chains
    // 1.2x, in the same time.
    const int64_t target = static_cast<int64_t>(ctx->num_sms) * 32;
    const int64_t block_bytes = static_cast<int64_t>(e.ppl) * 16 * kLanes / 2;
    int chain = e.n_blocks;
    while (chain > 1 && static_cast<int64_t>((e.n_blocks + chain - 1) / chain) * p.n_tile_groups < target)
      chain = (chain + 1) / 2;
    while (chain > 1 && chain * block_bytes > (int64_t(16) << 20)) chain = (chain + 1) / 2;
    p.chain = chain;
  }
  p.n_chains = (e.n_blocks + p.chain - 1) / p.chain;
  p.n_items = static_cast<int64_t>(p.n_chains) * p.n_tile_groups;
  return p;
}

namespace {

cudaError_t launch_any(cudaStream_t s, const WilsonPlan& plan_in, const Ensemble& e,
                       const Tile* tiles, const ProfileDev* profs, const double* rho,
                       int32_t n_groups, int32_t loops_per_group, wln_prec prec,
                       double* partial, int64_t n_points, int* d_flag, int64_t* launches,
                       double* loops_out) {
  WilsonPlan plan = plan_in;
  KParams kp{};
  kp.loops_out = loops_out;
  kp.blocks = e.blocks; kp.n_blocks = e.n_blocks; kp.ppl = e.ppl; kp.n_loops = e.n_loops;
  kp.tiles = tiles; kp.n_tiles = plan.n_tiles; kp.profs = profs; kp.rho = rho;
  kp.lpg = loops_per_group; kp.G = n_groups; kp.partial = partial; kp.n_points = n_points;
  kp.rows = plan.rows; kp.stages = plan.stages; kp.chain = plan.chain;
  kp.n_tile_groups = plan.n_tile_groups; kp.n_chains = plan.n_chains; kp.n_items = plan.n_items;
  kp.flag = d_flag;
  kp.stats = e.stats;
  kp.low_angle = plan.low_angle;
  const size_t smem = smem_bytes(plan, e.ppl);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
#define WLN_CASE_L(A, P_, W_, M_)                                                    \
  if (plan.P == P_ && plan.warps == W_ && plan.mode == M_) {                         \
    const int occ = occupancy<A, P_, W_, M_>(smem);                                  \
    const int64_t g = static_cast<int64_t>(sms) * occ;                               \
    const int grid = static_cast<int>(g < plan.n_items ? g : plan.n_items);          \
    ++*launches;                                                                     \
    return launch_t<A, P_, W_, M_>(s, kp, grid, smem);                               \
  }
#define WLN_CASE(A, P_, W_) WLN_CASE_L(A, P_, W_, kModeSums)
  if (plan.mode == kModeLevels) {
    switch (prec) {
      case WLN_PREC_FP32_COMP: WLN_CASE_L(F32Comp, 3, 4, kModeLevels) break;
      case WLN_PREC_FP32_NAIVE: WLN_CASE_L(F32Naive, 3, 4, kModeLevels) break;
      case WLN_PREC_FP64: WLN_CASE_L(F64, 1, 4, kModeLevels) break;
    }
    return cudaErrorInvalidConfiguration;
  }
  if (plan.mode == kModeNested) {
    switch (prec) {
      case WLN_PREC_FP32_COMP: WLN_CASE_L(F32Comp, 3, 4, kModeNested) break;
      case WLN_PREC_FP32_NAIVE: WLN_CASE_L(F32Naive, 3, 4, kModeNested) break;
      case WLN_PREC_FP64: WLN_CASE_L(F64, 1, 4, kModeNested) break;
    }
    return cudaErrorInvalidConfiguration;
  }
  if (plan.mode == kModeLoops) {
    switch (prec) {
      case WLN_PREC_FP32_COMP: WLN_CASE_L(F32Comp, 4, 4, kModeLoops) break;
      case WLN_PREC_FP32_NAIVE: WLN_CASE_L(F32Naive, 4, 4, kModeLoops) break;
      case WLN_PREC_FP64: WLN_CASE_L(F64, 2, 4, kModeLoops) break;
    }
    return cudaErrorInvalidConfiguration;
  }
  switch (prec) {
    case WLN_PREC_FP32_COMP:
      WLN_CASE(F32Comp, 4, 4)
      WLN_CASE(F32Comp, 4, 8)
      WLN_CASE(F32Comp, 8, 8)
      WLN_CASE(F32Comp, 2, 8)
      break;
    case WLN_PREC_FP32_NAIVE:
      WLN_CASE(F32Naive, 4, 4)
      WLN_CASE(F32Naive, 4, 8)
      WLN_CASE(F32Naive, 8, 8)
      WLN_CASE(F32Naive, 2, 8)
      break;
    case WLN_PREC_FP64:
      WLN_CASE(F64, 2, 4)
      WLN_CASE(F64, 1, 4)
      break;
  }
#undef WLN_CASE
#undef WLN_CASE_L
  return cudaErrorInvalidConfiguration;
}

}  // namespace

cudaError_t launch_wilson(cudaStream_t s, const WilsonPlan& plan, const Ensemble& e,
                          const Tile* tiles, const ProfileDev* profs, const double* rho,
                          int32_t n_groups, int32_t loops_per_group, wln_prec prec,
                          double* partial, int64_t n_points, int* d_flag, int64_t* launches) {
  return launch_any(s, plan, e, tiles, profs, rho, n_groups, loops_per_group, prec, partial,
                    n_points, d_flag, launches, nullptr);
}

cudaError_t launch_wilson_loops(cudaStream_t s, const WilsonPlan& plan, const Ensemble& e,
                                const Tile* tiles, const ProfileDev* profs, const double* rho,
                                wln_prec prec, double* out, int* d_flag, int64_t* launches) {
  // groups play no part; lpg = n_loops keeps the group arithmetic in range
  return launch_any(s, plan, e, tiles, profs, rho, 1, e.n_loops, prec, nullptr, 0, d_flag,
                    launches, out);
}

cudaError_t launch_selftest_wait(cudaStream_t s, int* d_flag, uint64_t limit_ns) {
  selftest_wait_kernel<<<1, 32, 0, s>>>(d_flag, limit_ns);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials(cudaStream_t s, const WilsonPlan& plan, const Ensemble& e,
                                   const double* partial, int64_t n_points, int32_t n_groups,
                                   int32_t loops_per_group, double* group_sums) {
  (void)e;
  const int K = level_mode(plan.mode) ? kLevelComps : kComps;
  const int64_t n = n_points * n_groups * K;
  if (n == 0) return cudaSuccess;
  reduce_partials_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(
      partial, n_points, n_groups, loops_per_group, plan.chain * 32, K, group_sums);
  return cudaGetLastError();
}

}  // namespace wln
