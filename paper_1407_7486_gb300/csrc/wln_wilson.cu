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
// theta; the same bits); for u <= 0.15 (tan(theta) < 0.18) it takes
// int dt/Q = theta / sqrt(D) from five terms of the series of atan(t)/t,
// and for u <= 0.045 (tan(theta) < 0.05) from three, without 1/sqrt(D) (the
// spin then takes 1/D; the result moves by rounding only).  The choice is
// per block and the same on every lane, so the walk has no branch per
// segment: the row loop exists once per form, in every mode.
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
#include <type_traits>

#include "wln_internal.cuh"

namespace wln {
namespace {

constexpr int kComps = WLN_K;
constexpr int kLevelComps = WLN_KL;

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// mbarrier helpers take the barrier's shared-memory address.
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
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
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
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
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(bar)
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
// (The walk's short-series forms use the same series for theta / sqrt(D)
// directly; these serve walks that do not carry Q.)
__device__ __forceinline__ float atan2_tiny(float y, float x) {
  const float t = y * rcp_approx(x);
  const float s = t * t;
  return fmaf(t * s, fmaf(s, 0.2f, -0.333333343f), t);
}

// The angle when 0 < y <= 0.18 x: t (1 - t^2/3 + t^4/5 - t^6/7 + t^8/9),
// remainder below t^11/11, under 3.3e-9 of atan t there.
__device__ __forceinline__ float atan2_mid(float y, float x) {
  const float t = y * rcp_approx(x);
  const float s = t * t;
  float q = fmaf(s, 0.111111112f, -0.142857149f);
  q = fmaf(s, q, 0.2f);
  q = fmaf(s, q, -0.333333343f);
  return fmaf(t * s, q, t);
}

// Forms of the angle, by the largest angle a block's segments may subtend at
// the field axis: at2_form<0> the general angle, <1> at most pi/4, <2>
// tan(theta) < 0.18, <3> tan(theta) < 0.05 (kLowAngle: the flavour has the
// cheaper forms).
struct F32Comp {
  using F = float;
  static constexpr bool kCompensated = true;
  static constexpr bool kLowAngle = true;
  static constexpr bool kFiveTerm = true;   // the tan(theta) < 0.18 series form
  __device__ static float rcp(float x) { return rcp_approx(x); }
  __device__ static float rsq(float x) { return rsqrt_approx(x); }
  template <int FORM>
  __device__ static float at2_form(float y, float x) {
    return FORM == 3   ? atan2_tiny(y, x)
           : FORM == 2 ? atan2_mid(y, x)
           : FORM == 1 ? atan2_low(y, x)
                       : atan2_pos(y, x);
  }
};
struct F32Naive {
  using F = float;
  static constexpr bool kCompensated = false;
  static constexpr bool kLowAngle = true;
  static constexpr bool kFiveTerm = true;
  __device__ static float rcp(float x) { return rcp_approx(x); }
  __device__ static float rsq(float x) { return rsqrt_approx(x); }
  template <int FORM>
  __device__ static float at2_form(float y, float x) {
    return FORM == 3   ? atan2_tiny(y, x)
           : FORM == 2 ? atan2_mid(y, x)
           : FORM == 1 ? atan2_low(y, x)
                       : atan2_pos(y, x);
  }
};
// The FP64 flavour takes the three-term form's place with series long enough
// for double precision (below): on blocks with tan(theta) < 0.05 it needs
// neither the arctangent nor 1/sqrt(D); elsewhere the library's atan2 (its
// pi/4 form is the general one).
struct F64 {
  using F = double;
  static constexpr bool kCompensated = false;
  static constexpr bool kLowAngle = true;
  static constexpr bool kFiveTerm = false;
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
  __device__ __forceinline__ void add(F a, F b) { part = fma(a, b, part); }
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
  const float2* sub_stats;  // the same per (block, kSubRows rows)
  int32_t n_sub;         // sub-blocks per block
  const float* maxlen;   // per block: longest loop
  int* item_counter;     // items claimed beyond the first wave (zeroed before the launch);
                         // nullptr: the static round-robin schedule
  int32_t low_angle;     // highest form of theta a block may take (0: general everywhere)
  GuardBufs guard;       // precision guard (FP32 compensated group sums)
};

// Whether every segment of block b subtends at most pi/4 at the field axis
// for the warp's tile, i.e. theta <= pi/4, i.e. sqrt(D) <= Q0 + B.  With |d|
// the segment, D <= Q0 C = Q0 |d|^2 (Lagrange) and B >= -|r| |d| >= -sqrt(Q0)
// |d|, so 2 |d| <= sqrt(Q0) is enough, and Q0 >= lambda^2 + (rho -
// sqrt(T) |y|_max)^2 for rho > sqrt(T) |y|_max.  The segments are sqrt(T)
// times the unit loop's (up to span of them for a sub-loop), and a margin of
// 0.9 keeps the float comparison of the two sides on the same side.  Every
// lane computes the same answer from the same block statistics.
// The same bound gives t = tan(theta) <= u / (1 - u), u = |d| / sqrt(Q0):
// for u <= 0.15, t < 0.18 and five terms of the series of atan t suffice;
// for u <= 0.045, t < 0.05 and three.  Returns the form of theta for the
// block: 3 (t < 0.05), 2 (t < 0.18), 1 (theta <= pi/4) or 0 (general).  (In
// float: the margins are far above its rounding.)
struct LowAngle {
  float two_span_sT, sT, rho_min, l2;
  __device__ __forceinline__ int block(const KParams& k, int b) const { return of(k.stats[b]); }
  // the form the statistics st (longest segment, largest |y|) allow
  __device__ __forceinline__ int of(const float2 st) const {
    const float gap = fmaxf(0.0f, rho_min - sT * st.y);
    const float lhs = two_span_sT * st.x, rhs = sqrtf(l2 + gap * gap);
    return lhs <= 0.09f * rhs ? 3 : (lhs <= 0.3f * rhs ? 2 : (lhs <= 0.9f * rhs ? 1 : 0));
  }
};

// Per-lane walk of one loop for the P radii of a tile (flux tube).  CQ
// carries Q at the current point so that theta = atan2(sqrt(D), Q0 + B)
// (one multiply fewer per segment and radius, one register more per radius);
// without it theta = atan2(C sqrt(D), D + B (B + C)).  step_<1> may be used
// when every segment subtends at most pi/4 at the axis, step_<2> when
// tan(theta) < 0.18 and step_<3> when tan(theta) < 0.05 (the caller has
// checked): theta then needs no octant unfolding, and in the last two cases
// only five or three terms of its series.
//
// Spin unit: the spin sums hold 2 int dt/Q^2 per segment, except on blocks
// walked with step_<3> when kSeriesSpin: there they hold int dt/Q^2 itself,
// and the caller doubles the block's spin scale (exact in double).  On those
// segments, with r = 1/(Q0 + B) and t^2 = D r^2 (t = tan(theta)):
//   int dt/Q   = r f(t^2),                f(u) = atan(sqrt u)/sqrt u
//                                               = sum_k (-u)^k / (2k + 1),
//   int dt/Q^2 = -d/d(lambda^2) int dt/Q  (lambda^2 moves Q0 + B by 1 and D
//              by C)  = r^2 [f - (C r - 2 t^2) f'] = 1/(Q0 Q1) + C r^3 h(t^2),
//   h(u) = -f'(u) = 1/3 - 2u/5 + 3u^2/7 - ...,  using r^2/(1 + t^2) =
//   1/(Q0 Q1) (Q0 Q1 = (Q0 + B)^2 + D).  Two terms of h leave a remainder
//   under 3.6e-9 of int dt/Q^2 for t < 0.05 (C r < 0.0022 there); the spin
//   then needs neither 1/D nor a difference of nearly equal quotients.
template <class A, int P, bool CQ = true>
struct Walk {
  static constexpr bool kSeriesSpin = CQ;
  using F = typename A::F;
  F s, l2;           // sqrt(T), lambda^2
  F rho[P];
  // state at the current point
  F ux, uy;          // unit-loop point
  F ry;              // scaled y (shared by the radii)
  F rx[P];           // shifted, scaled x
  F q[P], rq[P];     // Q and 1/Q at the current point
  Acc<F, A::kCompensated> ph[P], sp[P];

  __device__ __forceinline__ void set_rho(int p, F v) { rho[p] = v; }

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
    // C h(t^2) = C/3 - (2C/5) t^2 on the three-term form (values the radii share)
    F c3 = F(0), cn25 = F(0);
    if constexpr (FORM == 3 && CQ && sizeof(F) == 4) {
      c3 = C * F(0.333333343);
      cn25 = C * F(-0.4);
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const F rx1 = fma(s, x1, rho[p]);
      const F q1 = fma(rx1, rx1, e1);
      const F rq1 = A::rcp(q1);
      const F B = fma(rx[p], dx, rydy);
      const F X = fma(rx[p], dy, -rydx);
      const F D = fma(X, X, l2C);
      const F BC = B + C;
      if constexpr (FORM >= 2 && CQ) {
        // tan(theta) = t with t^2 = D r^2, r = 1/(Q0 + B): int dt/Q =
        // theta / sqrt(D) = r atan(t) / t, without 1/sqrt(D); the spin takes
        // 1/D instead.  t < 0.05: r (1 - t^2/3 + t^4/5); t < 0.18: r (1 -
        // t^2/3 + t^4/5 - t^6/7 + t^8/9) (remainders under 3.3e-9).
        const F r = A::rcp(q[p] + B);
        const F r2 = r * r;
        const F t2 = D * r2;
        F poly;
        if constexpr (FORM == 3 && sizeof(F) == 8) {
          // double: six terms, remainder below t^12/13 < 2e-17
          poly = fma(t2, -1.0 / 11.0, 1.0 / 9.0);
          poly = fma(t2, poly, -1.0 / 7.0);
          poly = fma(t2, poly, 0.2);
          poly = fma(t2, poly, -1.0 / 3.0);
          poly = fma(t2, poly, 1.0);
        } else if constexpr (FORM == 3) {
          poly = fma(t2, fma(t2, F(0.2), F(-0.333333343)), F(1));
        } else {
          poly = fma(t2, F(0.111111112), F(-0.142857149));
          poly = fma(t2, poly, F(0.2));
          poly = fma(t2, poly, F(-0.333333343));
          poly = fma(t2, poly, F(1));
        }
        const F J1 = r * poly;
        ph[p].add(X, J1);
        if constexpr (FORM == 3 && sizeof(F) == 8) {
          // double: h to five terms (remainder below C r (6/13) t^10, 1e-16)
          F h = fma(t2, 5.0 / 11.0, -4.0 / 9.0);
          h = fma(t2, h, 3.0 / 7.0);
          h = fma(t2, h, -0.4);
          h = fma(t2, h, 1.0 / 3.0);
          sp[p].add(C * (r2 * r), h);
          sp[p].add(rq[p], rq1);
        } else if constexpr (FORM == 3) {
          // int dt/Q^2 = C r^3 (1/3 - 2 t^2/5) + 1/(Q0 Q1)  (unit: see above)
          sp[p].add(r2 * r, fma(t2, cn25, c3));
          sp[p].add(rq[p], rq1);
        } else {
          const F br = fma(fma(-B, BC, D) * rq[p], rq1, C * J1);
          sp[p].add(br * A::rcp(D));
        }
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
  static constexpr bool kSeriesSpin = false;
  using F = typename A::F;
  F s, l2;
  F rho[P];
  F ux, uy, ry;
  F rx[P];
  Acc<F, A::kCompensated> ph[P];
  __device__ __forceinline__ void set_rho(int p, F v) { rho[p] = v; }
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

// ------------------------------------------------- paired FP32 arithmetic
// The sm_100 family issues two FP32 operations of a float2 in one instruction
// (fma, add, mul), each lane rounded exactly as the scalar _rn operation.
// Neither subtraction nor negation exists in paired form; both are written
// exactly: fma(a, -1, b) rounds as b - a, and negating one factor of a
// product (or every input of an fma) negates the rounded result.
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  return __ffma2_rn(a, b, c);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
template <class A>
__device__ __forceinline__ float2 rcp2(float2 x) {
  return make_float2(A::rcp(x.x), A::rcp(x.y));
}
template <class A>
__device__ __forceinline__ float2 rsq2(float2 x) {
  return make_float2(A::rsq(x.x), A::rsq(x.y));
}

// atan_unit, atan2_low and atan2_pos on a pair, bitwise equal per lane.
__device__ __forceinline__ float2 atan_unit2(float2 t) {
  const float2 s = mul2(t, t);
  float2 q = fma2(bc2(0.002920693f), s, bc2(-0.01636793f));
  q = fma2(q, s, bc2(0.043211866f));
  q = fma2(q, s, bc2(-0.07552215f));
  q = fma2(q, s, bc2(0.106660046f));
  q = fma2(q, s, bc2(-0.14211056f));
  q = fma2(q, s, bc2(0.19993773f));
  q = fma2(q, s, bc2(-0.33333153f));
  return fma2(mul2(t, s), q, t);
}

__device__ __forceinline__ float2 atan2_low2(float2 y, float2 x) {
  return atan_unit2(mul2(y, make_float2(rcp_approx(x.x), rcp_approx(x.y))));
}

__device__ __forceinline__ float2 atan2_pos2(float2 y, float2 x) {
  const float2 ax = make_float2(fabsf(x.x), fabsf(x.y));
  const float2 mn = make_float2(fminf(y.x, ax.x), fminf(y.y, ax.y));
  const float2 mx = make_float2(fmaxf(y.x, ax.x), fmaxf(y.y, ax.y));
  float2 r = atan_unit2(mul2(mn, make_float2(rcp_approx(mx.x), rcp_approx(mx.y))));
  const float2 up = fma2(r, bc2(-1.0f), bc2(1.5707963267948966f));   // pi/2 - r
  r = make_float2(y.x > ax.x ? up.x : r.x, y.y > ax.y ? up.y : r.y);
  const float2 left = fma2(r, bc2(-1.0f), bc2(3.14159265358979323846f));   // pi - r
  return make_float2(x.x < 0.0f ? left.x : r.x, x.y < 0.0f ? left.y : r.y);
}

// Acc on a pair; nc holds the compensation negated (so that every step is a
// paired add or fma).
template <bool kComp>
struct Acc2 {
  float2 s, nc, part;
  __device__ __forceinline__ void zero() {
    s = bc2(0.0f); nc = bc2(0.0f); part = bc2(0.0f);
  }
  __device__ __forceinline__ void add(float2 a, float2 b) { part = fma2(a, b, part); }
  __device__ __forceinline__ void fold() {
    if (kComp) {
      const float2 y = add2(part, nc);                 // part - c
      const float2 t = add2(s, y);
      const float2 u = fma2(s, bc2(-1.0f), t);         // t - s
      nc = fma2(u, bc2(-1.0f), y);                     // -((t - s) - y)
      s = t;
    } else {
      s = add2(s, part);
    }
    part = bc2(0.0f);
  }
  __device__ __forceinline__ void lane(int i, double& sum, double& comp) const {
    sum = i ? s.y : s.x;
    comp = -(i ? nc.y : nc.x);
  }
};

// The flux-tube walk of Walk<A, P, true> for the float flavours with the
// radii of a lane in pairs: the same operations in the same order, bitwise
// equal per radius, two radii per instruction.  The values every radius
// shares (the segment, the scaled y) are formed once in scalar arithmetic and
// broadcast to both lanes of a pair: a paired instruction takes two cycles of
// the FMA pipe, which bounds this walk, so work the radii share stays scalar.
template <class A, int P>
struct Walk2 {
  static constexpr bool kSeriesSpin = true;   // as Walk<A, P, true>
  static_assert(P % 2 == 0, "radii in pairs");
  static constexpr int H = P / 2;
  using F = float;
  F s, l2;
  float2 rho[H];
  F ux, uy, ry;               // the current point; ry = s y
  float2 rx[H], q[H], rq[H];
  Acc2<A::kCompensated> ph[H], sp[H];

  __device__ __forceinline__ void set_rho(int p, F v) {
    if (p & 1) rho[p >> 1].y = v;
    else rho[p >> 1].x = v;
  }

  __device__ __forceinline__ void start(F x0, F y0) {
    ux = x0; uy = y0;
    ry = s * y0;
    const float2 e0 = bc2(fmaf(ry, ry, l2));
#pragma unroll
    for (int j = 0; j < H; ++j) {
      rx[j] = fma2(bc2(s), bc2(x0), rho[j]);
      q[j] = fma2(rx[j], rx[j], e0);
      rq[j] = rcp2<A>(q[j]);
      ph[j].zero();
      sp[j].zero();
    }
  }

  __device__ __forceinline__ void step(F x1, F y1) { step_<0>(x1, y1); }

  template <int FORM>
  __device__ __forceinline__ void step_(F x1, F y1) {
    const F dxs = s * (x1 - ux), dys = s * (y1 - uy);
    const F Cs = fmaf(dxs, dxs, dys * dys);
    const F ry1 = s * y1;
    const float2 M1 = bc2(-1.0f), S = bc2(s), X1 = bc2(x1);
    const float2 dx = bc2(dxs), dy = bc2(dys), C = bc2(Cs), nC = bc2(-Cs);
    const float2 l2C = bc2(l2 * Cs);
    const float2 e1 = bc2(fmaf(ry1, ry1, l2));
    const float2 rydy = bc2(ry * dys);
    const float2 nrydx = bc2(-(ry * dxs));
    float2 c3 = bc2(0.0f), cn25 = bc2(0.0f);
    if constexpr (FORM == 3) { c3 = bc2(Cs * 0.333333343f); cn25 = bc2(Cs * -0.4f); }
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const float2 rx1 = fma2(S, X1, rho[j]);
      const float2 q1 = fma2(rx1, rx1, e1);
      const float2 rq1 = rcp2<A>(q1);
      const float2 B = fma2(rx[j], dx, rydy);
      const float2 X = fma2(rx[j], dy, nrydx);
      const float2 D = fma2(X, X, l2C);
      const float2 xa = add2(q[j], B);                // Q0 + B
      if constexpr (FORM == 3) {
        // theta / sqrt(D) = r atan(t) / t and int dt/Q^2 = C r^3 (1/3 -
        // 2 t^2/5) + 1/(Q0 Q1), t^2 = D r^2, r = 1/(Q0 + B) (as in Walk)
        const float2 r = rcp2<A>(xa);
        const float2 r2 = mul2(r, r);
        const float2 t2 = mul2(D, r2);
        const float2 poly = fma2(t2, fma2(t2, bc2(0.2f), bc2(-0.333333343f)), bc2(1.0f));
        ph[j].add(X, mul2(r, poly));
        sp[j].add(mul2(r2, r), fma2(t2, cn25, c3));
        sp[j].add(rq[j], rq1);
      } else {
        float2 J1, w;
        if constexpr (FORM == 2) {
          // theta / sqrt(D) = r atan(t) / t, t^2 = D r^2, r = 1/(Q0 + B)
          const float2 r = rcp2<A>(xa);
          const float2 t2 = mul2(D, mul2(r, r));
          float2 poly = fma2(t2, bc2(0.111111112f), bc2(-0.142857149f));
          poly = fma2(t2, poly, bc2(0.2f));
          poly = fma2(t2, poly, bc2(-0.333333343f));
          poly = fma2(t2, poly, bc2(1.0f));
          J1 = mul2(r, poly);
          w = rcp2<A>(D);
        } else {
          const float2 rsD = rsq2<A>(D);
          const float2 ya = mul2(D, rsD);
          const float2 theta = FORM == 1 ? atan2_low2(ya, xa) : atan2_pos2(ya, xa);
          J1 = mul2(theta, rsD);
          w = mul2(rsD, rsD);
        }
        ph[j].add(X, J1);
        // ((C + B)/Q1 - B/Q0 + C J1) / D with the quotients' difference as
        // (D - B (B + C)) / (Q0 Q1)
        const float2 nBC = fma2(B, M1, nC);             // -(B + C)
        const float2 br = fma2(mul2(fma2(B, nBC, D), rq[j]), rq1, mul2(C, J1));
        sp[j].add(br, w);
      }
      rx[j] = rx1;
      q[j] = q1;
      rq[j] = rq1;
    }
    ux = x1; uy = y1; ry = ry1;
  }

  __device__ __forceinline__ void fold() {
#pragma unroll
    for (int j = 0; j < H; ++j) { ph[j].fold(); sp[j].fold(); }
  }

  __device__ __forceinline__ void raw(int p, double& ps, double& pc, double& ss,
                                      double& sc) const {
    ph[p >> 1].lane(p & 1, ps, pc);
    sp[p >> 1].lane(p & 1, ss, sc);
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
                                             double* w, float* spin_abs = nullptr) {
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
    if (spin_abs) *spin_abs = sv.hi;
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
// mbarriers (kept as 32-bit shared-memory addresses); thread 0 also refills
// it, with its bookkeeping in shared memory (no other thread needs it, so it
// takes no registers in the walking threads).
struct Pipe {
  float4* ring;
  uint32_t full, empty;   // shared addresses of the mbarrier arrays
  int stages, chunk_rows, chunks_per_block;
  int32_t kc = 0;
};

struct ProdState {
  int32_t issued;     // chunks issued
  int32_t blk, chunk; // position within the current item
  int64_t item;       // the item being issued
  int32_t started, done;
};
__shared__ ProdState s_prod;
// The item of each staged chunk, or -1 once the items are exhausted (written
// by thread 0 before the chunk's barrier completes, read by the warps after).
constexpr int kMaxStages = 8;
__shared__ int32_t s_chunk_item[kMaxStages];

__device__ __forceinline__ int blocks_in_item(const KParams& k, int64_t item) {
  const int c = static_cast<int>(item / k.n_tile_groups);
  const int b0 = c * k.chain;
  return min(b0 + k.chain, k.n_blocks) - b0;
}

// Thread 0: the next chunk of the CTA's items into ring slot `slot`.  The
// first item of a CTA is its block index; later items are claimed one at a
// time from the launch's counter when their first chunk is issued (dynamic
// schedule: CTAs that finish early take more), or taken round-robin without
// a counter.  Past the last item the slot gets the sentinel -1 and its full
// barrier completes without a copy, so every warp's wait ends.
__device__ __forceinline__ void issue_next(const KParams& k, const Pipe& pp, int slot) {
  ProdState& ps = s_prod;
  if (ps.blk == 0 && ps.chunk == 0) {
    int64_t item;
    if (!ps.started) {
      item = blockIdx.x;
      ps.started = 1;
    } else if (k.item_counter) {
      item = static_cast<int64_t>(gridDim.x) + atomicAdd(k.item_counter, 1);
    } else {
      item = ps.item + gridDim.x;
    }
    ps.item = item;
    if (item >= k.n_items) {
      s_chunk_item[slot] = -1;
      ps.done = 1;
      mbar_arrive(pp.full + 8u * slot);
      return;
    }
  }
  s_chunk_item[slot] = static_cast<int32_t>(ps.item);
  const int c = static_cast<int>(ps.item / k.n_tile_groups);
  const int b = c * k.chain + ps.blk;
  const uint32_t bytes = static_cast<uint32_t>(pp.chunk_rows) * 512u;
  const float4* src = k.blocks + (static_cast<size_t>(b) * (k.ppl / 2) +
                                  static_cast<size_t>(ps.chunk) * pp.chunk_rows) * 32;
  mbar_arrive_expect_tx(pp.full + 8u * slot, bytes);
  bulk_load(pp.ring + static_cast<size_t>(slot) * pp.chunk_rows * 32, src, bytes,
            pp.full + 8u * slot);
  ++ps.issued;
  if (++ps.chunk == pp.chunks_per_block) {
    ps.chunk = 0;
    if (++ps.blk == blocks_in_item(k, ps.item)) ps.blk = 0;
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

// ------------------------------------------------------- precision guard
// A model of the float walk's rounding (measured against the oracle on
// GB300, 640 loops of 2048 points, flux tubes F = 10..100, lambda = 0.1..1,
// T up to 20): a loop's phase is off by a random amount of rms
// c_ph * (sum of |segment phases|) / sqrt(N), c_ph <= 1.9e-7, and its spin by
// a relative 3.6e-8 at most (systematic: the float scale sqrt(T) and the
// approximate reciprocals) plus a random part that averages over the loops.
// The model takes c_ph = 2e-7 and a spin error beta |spin|, beta = 5e-8,
// counted as systematic.  The sum of
// |segment phases| of a loop in block b at radius rho is at most
// calF sqrt(T) L_b h, L_b the block's longest unit loop and h the largest
// rho/(lambda^2 + rho^2) over the block's reach, 1/(2 lambda) if the block
// comes within lambda of the axis.  Loops below kGuardFloor have cosh(spin)
// < 3.77 and are not recorded; the model counts them in bulk.
constexpr float kCoshFloor = 3.76219569f;   // cosh(2)
constexpr float kGuardBeta = 5e-8f;
constexpr float kGuardCph = 2e-7f;
constexpr float kGuardBudget = 0.5e-6f;     // half of the 1e-6 bar
constexpr float kGuardSigmas = 2.0f;        // random part counted at 2 sigma

struct GuardScratch {
  float* bmax;   // [bpg][P]: the block's largest |spin|, -1 below the floor
  float* s;      // [bpg][P][32]: |spin|, then the loop's systematic error share
  float* sn;     // [bpg][P][32]: sin(phase), then the loop's random error share
  double* f1;    // [bpg][P][32]: the float W_ferm - 1
  int* sel;      // [kGuardSel]: selected (block << 5 | lane)
  __device__ GuardScratch(char* base, int bpg, int P) {
    const int recs = bpg * P;
    bmax = reinterpret_cast<float*>(base);
    s = reinterpret_cast<float*>(base + (recs * 4 + 15) / 16 * 16);
    sn = s + recs * 32;
    f1 = reinterpret_cast<double*>(sn + recs * 32);
    sel = reinterpret_cast<int*>(f1 + recs * 32);
  }
};

__device__ __forceinline__ float warp_sum_f(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Bound on a loop's random phase error (rms) in block b at radius rho.
__device__ __forceinline__ float guard_sigma(const KParams& k, int b, float sT, float rho,
                                             float calF, float l2, float lam, float inv_sqrtN) {
  const float gap = fmaxf(0.0f, rho - sT * k.stats[b].y);
  const float h = gap >= lam ? gap / (l2 + gap * gap) : 0.5f / lam;
  return kGuardCph * calF * sT * k.maxlen[b] * h * inv_sqrtN;
}

// End of a group for the warp's tile: per radius, the error estimate of the
// group's spinor sum against the budget 0.5e-6 max(lpg, sum of cosh(spin)),
// all quantities relative to cosh of the group's largest spin; while it is
// over, select the recorded loop with the largest share (ties: lowest block,
// then lane).  If kGuardSel loops bring it under the budget they are queued;
// if not (the error is spread over many loops of similar spin, as in fields
// nearly constant across the loops) nothing is, and the group is counted as
// saturated.  Every lane takes part; the order is fixed.
template <int P>
__device__ __forceinline__ void guard_select(const KParams& k, char* scr, const Tile& tile,
                                             const ProfileDev& prof, int t_index, int c, int g,
                                             int lane) {
  const GuardBufs& G = k.guard;
  const int bpg = G.bpg;
  GuardScratch R(scr, bpg, P);
  __syncwarp();
  const float sT = sqrtf(static_cast<float>(tile.T));
  const float calF = static_cast<float>(6.283185307179586 * prof.turns_per);
  const float l2 = static_cast<float>(prof.l2), lam = sqrtf(l2);
  const float inv_sqrtN = rsqrtf(static_cast<float>(k.ppl));
  for (int p = 0; p < tile.n_valid; ++p) {
    float smax = -1.0f;
    for (int bi = 0; bi < bpg; ++bi) smax = fmaxf(smax, R.bmax[bi * P + p]);
    if (smax < kGuardFloor) continue;
    const float rho = static_cast<float>(k.rho[tile.rho0 + p]);
    const float e2m = __expf(-2.0f * smax);
    const float inv = 2.0f * __expf(-smax) / (1.0f + e2m);   // 1 / cosh(smax)
    float csum = 0.0f, sys = 0.0f, rnd2 = 0.0f, sig_nc = 0.0f;
    int n_nc = 0;
    for (int bi = 0; bi < bpg; ++bi) {
      const float sig = guard_sigma(k, g * bpg + bi, sT, rho, calF, l2, lam, inv_sqrtN);
      if (R.bmax[bi * P + p] < kGuardFloor) {
        n_nc += 32;
        sig_nc = fmaxf(sig_nc, sig);
        continue;
      }
      const int r = (bi * P + p) * 32 + lane;
      const float sp = R.s[r], sn = R.sn[r];
      // cosh(sp) / cosh(smax), sp <= smax
      const float w = __expf(sp - smax) * (1.0f + __expf(-2.0f * sp)) / (1.0f + e2m);
      const float es = w * kGuardBeta * sp, er = w * fabsf(sn) * sig;
      csum += w;
      sys += es;
      rnd2 += er * er;
      R.s[r] = es;    // the shares replace the inputs
      R.sn[r] = er;
    }
    csum = warp_sum_f(csum);
    sys = warp_sum_f(sys);
    rnd2 = warp_sum_f(rnd2);
    const float nc = static_cast<float>(n_nc);
    csum += nc * inv;
    sys += nc * kCoshFloor * inv * kGuardBeta * kGuardFloor;
    rnd2 += nc * (kCoshFloor * inv * sig_nc) * (kCoshFloor * inv * sig_nc);
    const float budget = kGuardBudget * fmaxf(static_cast<float>(k.lpg) * inv, csum);
    int n = 0;
    uint64_t taken = 0;   // this lane's loop, blocks already selected
    while ((G.all || sys + kGuardSigmas * sqrtf(fmaxf(rnd2, 0.0f)) > budget) && n < kGuardSel) {
      float best = -1.0f;
      int bbi = 0;
      for (int bi = 0; bi < bpg; ++bi) {
        if (R.bmax[bi * P + p] < kGuardFloor || ((taken >> bi) & 1)) continue;
        const int r = (bi * P + p) * 32 + lane;
        const float key = R.s[r] + kGuardSigmas * R.sn[r];
        if (key > best) { best = key; bbi = bi; }
      }
      // warp argmax of (key, -(block, lane)): keys are >= 0 or -1 (none)
      uint64_t v = best < 0.0f ? 0ull
                               : (static_cast<uint64_t>(__float_as_uint(best) + 1u) << 32) |
                                     (0xFFFFFFFFu - static_cast<uint32_t>(bbi * 32 + lane));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const uint64_t u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
      }
      if ((v >> 32) == 0ull || (!G.all && (v >> 32) == 1ull)) break;   // none left / zero shares
      const int idx = static_cast<int>(0xFFFFFFFFu - static_cast<uint32_t>(v & 0xFFFFFFFFull));
      const int wbi = idx >> 5, wl = idx & 31;
      if (lane == wl) taken |= 1ull << wbi;
      const int r = (wbi * P + p) * 32 + wl;
      sys -= R.s[r];
      rnd2 -= R.sn[r] * R.sn[r];
      if (lane == 0) R.sel[n] = idx;
      ++n;
    }
    if (!G.all && sys + kGuardSigmas * sqrtf(fmaxf(rnd2, 0.0f)) > budget) {
      if (lane == 0) atomicAdd(&G.counters[3], 1);
      n = 0;
    }
    if (n == 0) continue;
    __syncwarp();
    int base = 0;
    if (lane == 0) base = atomicAdd(&G.counters[0], n);
    base = __shfl_sync(0xffffffffu, base, 0);
    const bool fits = static_cast<int64_t>(base) + n <= G.cap;
    for (int j = lane; j < n; j += 32) {
      if (static_cast<int64_t>(base) + j >= G.cap) continue;
      const int idx = R.sel[j], bi = idx >> 5, ln = idx & 31;
      GuardItem it;
      it.tile = fits ? t_index : -1;
      it.p_loop = (p << 24) | ((g * bpg + bi) * 32 + ln);
      it.f1 = R.f1[(bi * P + p) * 32 + ln];
      G.items[base + j] = it;
    }
    if (lane == 0) {
      if (fits) {
        const int si = atomicAdd(&G.counters[1], 1);
        GuardSlot sl;
        sl.dst = tile.part_base +
                 (static_cast<int64_t>(c + g) * tile.part_stride + tile.p0 + p) * kComps;
        sl.item0 = base;
        sl.n = n;
        G.slots[si] = sl;
      } else {
        atomicAdd(&G.counters[2], 1);   // counted; these loops keep float precision
      }
    }
    __syncwarp();
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
// The tile and profile are read where they are needed rather than held in
// registers across the walk (the row loop is register-bound).
template <class A, int P, class WalkT, int MODE>
__device__ bool run_item(const KParams& k, Pipe& pp, double* acc, int c, const Tile& tile,
                         const ProfileDev& prof, bool active, volatile int* abort_flag,
                         int lane, int t_index) {
  using F = typename A::F;
  // precision guard: FP32-compensated group sums of flux tubes
  constexpr bool GUARD = std::is_same<A, F32Comp>::value && MODE == kModeSums;
  const bool guard_tile = GUARD && k.guard.on && active && prof.kind == WLN_PROFILE_FLUX_TUBE;
  // this warp's guard records (derived when used: no register across the walk)
  auto gscr = [&]() {
    return k.guard.scratch +
           (static_cast<size_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5)) *
               k.guard.warp_bytes;
  };
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
      w[q].set_rho(p, static_cast<F>(k.rho[tile.rho0 + i]));
    }
  }
  // the spin's scale T spin_per and the phase's turns per unit sum, as
  // double and double-float, formed where W is formed
  auto st_d = [&]() { return prof.spin_per * tile.T; };
  // the form of theta for block b (the same on every lane), from the block's
  // statistics (sub == -1) or those of its sub-block sub; sub-loop segments
  // join points up to 4 apart
  auto block_form = [&](int b, int sub) {
    if (!(A::kLowAngle && k.low_angle && prof.kind == WLN_PROFILE_FLUX_TUBE && tile.n_valid > 0))
      return 0;
    double rho_min = k.rho[tile.rho0];
    for (int p = 1; p < tile.n_valid; ++p) rho_min = fmin(rho_min, k.rho[tile.rho0 + p]);
    const LowAngle la{static_cast<float>(2.0 * (LV ? 4.0 : 1.0) * sqrt(tile.T)),
                      static_cast<float>(sqrt(tile.T)), static_cast<float>(rho_min),
                      static_cast<float>(prof.l2)};
    int f = sub < 0 ? la.block(k, b)
                    : la.of(k.sub_stats[static_cast<size_t>(b) * k.n_sub + sub]);
    if (!A::kFiveTerm && f == 2) f = 1;
    return k.low_angle >= 2 ? f : min(f, k.low_angle);   // level 2: the series forms too
  };
  // Whole loops, a chunk of rows [r0, r0 + n): the block's form, or where
  // the block does not take the three-term series (whose spin unit holds
  // for the whole block), the best of the block's and the chunk's sub-blocks'
  // forms up to the five-term series.
  auto chunk_form = [&](int b, int bform, int r0, int n) {
    if (bform == 3) return 3;
    int f = A::kFiveTerm ? 2 : 1;
    for (int sb = r0 / kSubRows; sb <= (r0 + n - 1) / kSubRows && f > bform; ++sb)
      f = min(f, block_form(b, sb));
    return max(f, bform);
  };
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
    const int form = block_form(b, -1);
    // the block's spin sums hold int dt/Q^2 itself, not twice it, where its
    // segments take the three-term series
    const bool half_spin = WalkT::kSeriesSpin && form == 3;
    // first point of each walk, for the closing segments
    float fx[NW], fy[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q) { fx[q] = 0.f; fy[q] = 0.f; }
    for (int ch = 0; ch < pp.chunks_per_block; ++ch) {
      const int slot = static_cast<int>(pp.kc % pp.stages);
      const uint32_t parity = static_cast<uint32_t>((pp.kc / pp.stages) & 1);
      // every lane of the warp takes the same decision (the warp's
      // shuffles and syncs need all 32 lanes)
      if (!__all_sync(0xffffffffu, mbar_wait(pp.full + 8u * slot, parity))) {
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
            if (half_spin) w[0].template step_<3>(v.z, v.w);
            else w[0].step(v.z, v.w);
            r = 1;
          }
          // the form of theta for this chunk is the same on every lane
          const int cf = chunk_form(b, form, ch * pp.chunk_rows, pp.chunk_rows);
          if (cf == 3) rows_plain<3>(w, rowp, r, pp.chunk_rows);
          else if (cf == 2) rows_plain<2>(w, rowp, r, pp.chunk_rows);
          else if (cf == 1) rows_plain<1>(w, rowp, r, pp.chunk_rows);
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
            w[1].start(a.x, a.y);
            w[2].start(a.x, a.y);
            if (half_spin) {
              w[0].template step_<3>(a.z, a.w);
              w[0].template step_<3>(v.x, v.y);
              w[0].template step_<3>(v.z, v.w);
              w[1].template step_<3>(v.x, v.y);
            } else {
              w[0].step(a.z, a.w);
              w[0].step(v.x, v.y);
              w[0].step(v.z, v.w);
              w[1].step(v.x, v.y);
            }
            r = 2;
          }
          if (form == 3) rows_nested<3>(w, rowp, r, pp.chunk_rows);
          else if (form == 2) rows_nested<2>(w, rowp, r, pp.chunk_rows);
          else if (form == 1) rows_nested<1>(w, rowp, r, pp.chunk_rows);
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
            if (half_spin) w[0].template step_<3>(v.x, v.y);
            else w[0].step(v.x, v.y);
            w[2].start(v.z, v.w);
            r = 2;
          }
          if (form == 3) rows_levels<3>(w, rowp, r, pp.chunk_rows);
          else if (form == 2) rows_levels<2>(w, rowp, r, pp.chunk_rows);
          else if (form == 1) rows_levels<1>(w, rowp, r, pp.chunk_rows);
          else rows_levels<0>(w, rowp, r, pp.chunk_rows);
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(pp.empty + 8u * slot);
      if (threadIdx.x == 0 && !s_prod.done) {
        // The slot just released is the next one to refill.
        if (!mbar_wait(pp.empty + 8u * slot, parity)) {
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
      // closing segment back to the walk's first point
      if (half_spin) w[q].template step_<3>(fx[q], fy[q]);
      else w[q].step(fx[q], fy[q]);
      w[q].fold();
    }
    // the spin's scale for this block's sums (doubling is exact)
    auto st_b = [&]() { return half_spin ? 2.0 * st_d() : st_d(); };
    if constexpr (PL) {
      if (valid) {
#pragma unroll
        for (int p = 0; p < P; ++p) {
          if (p < tile.n_valid) {
            double ps, pc, ss, sc, t[kComps];
            w[0].raw(p, ps, pc, ss, sc);
            wilson_terms<A>(ps, pc, ss, sc, split(prof.turns_per), split(st_b()), prof.turns_per,
                            st_b(), t);
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
      if (g != g_cur) {
        if constexpr (GUARD) {
          if (guard_tile) guard_select<P>(k, gscr(), tile, prof, t_index, c, g_cur, lane);
        }
        flush(g_cur);
        g_cur = g;
      }
      const bool mine = g_lane == g;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        if constexpr (!LV) {
          double ps, pc, ss, sc, t[K];
          float sabs = 0.0f;
          w[0].raw(p, ps, pc, ss, sc);
          wilson_terms<A>(ps, pc, ss, sc, split(prof.turns_per), split(st_b()), prof.turns_per,
                          st_b(), t, &sabs);
#pragma unroll
          for (int q = 0; q < K; ++q)
            if (mine) acc[(p * K + q) * 33 + lane] += t[q];
          if constexpr (GUARD) {
            // the block's largest spin; above the floor, every loop's spin,
            // sin(phase) and float W_ferm - 1 for the group-end selection
            if (guard_tile && p < tile.n_valid) {
              const float sv = valid ? sabs : 0.0f;
              const float bm = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(sv)));
              GuardScratch R(gscr(), k.guard.bpg, P);
              const int idx = (b - g * k.guard.bpg) * P + p;
              if (bm >= kGuardFloor) {
                R.s[idx * 32 + lane] = sv;
                R.sn[idx * 32 + lane] = static_cast<float>(t[2]);
                R.f1[idx * 32 + lane] = t[1];
              }
              if (lane == 0) R.bmax[idx] = bm >= kGuardFloor ? bm : -1.0f;
            }
          }
        } else {
          // Spin per segment is T/N' on a sub-loop of N' points: the circle's
          // sums count twice, the square's and triangle's four times, of the
          // full loop's T/N (a constant field's spin is B T on every loop);
          // the nested walks of N, N/2 and N/4 points count 1, 2 and 4 times.
          const bool tube = prof.kind != WLN_PROFILE_CONST_B;
          const double hs = half_spin ? 2.0 : 1.0;
          double po, so, pq, sq, pt, stt;
          walk_sums(w[0], p, tube ? (NEST ? 1.0 : 2.0) * hs : 1.0, po, so);
          walk_sums(w[1], p, tube ? (NEST ? 2.0 : 4.0) * hs : 1.0, pq, sq);
          walk_sums(w[2], p, tube ? 4.0 * hs : 1.0, pt, stt);
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
            level_terms<A>(ph, sp, split(prof.turns_per), split(st_d()), prof.turns_per, st_d(),
                           t);
            if (mine) {
              acc[(p * K + 2 * L) * 33 + lane] += t[0];
              acc[(p * K + 2 * L + 1) * 33 + lane] += t[1];
            }
          }
        }
      }
    }
  }
  if constexpr (GUARD) {
    if (guard_tile) guard_select<P>(k, gscr(), tile, prof, t_index, c, g_cur, lane);
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
// pass with the scalar walk 3 radii x 4 warps x 2 CTAs 757 ms, 4 x 8 x 1
// 774 ms, with the radii in pairs 4 x 4 x 2 541 ms.
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
  const int rows_per_block = k.ppl / 2;
  pp.chunk_rows = k.rows < rows_per_block ? k.rows : rows_per_block;
  pp.chunks_per_block = rows_per_block / pp.chunk_rows;
  pp.stages = k.stages;
  pp.ring = reinterpret_cast<float4*>(smem);
  const size_t ring_bytes = static_cast<size_t>(k.stages) * pp.chunk_rows * 512;
  double* acc = reinterpret_cast<double*>(smem + ring_bytes) + warp * (P * K * 33);
  pp.full = smem_u32(smem + ring_bytes + WARPS * P * K * 33 * sizeof(double));
  pp.empty = pp.full + 8u * k.stages;
  for (int j = 0; j < P * K; ++j) acc[j * 33 + lane] = 0.0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < k.stages; ++s) {
      mbar_init(pp.full + 8u * s, 1);
      mbar_init(pp.empty + 8u * s, WARPS);
    }
    abort_flag = 0;
    s_prod.issued = 0;
    s_prod.blk = 0;
    s_prod.chunk = 0;
    s_prod.item = 0;
    s_prod.started = 0;
    s_prod.done = 0;
    fence_mbar_init();
    for (int s = 0; s < k.stages && !s_prod.done; ++s) issue_next(k, pp, s);
  }
  __syncthreads();

  bool ok = true;
  while (ok) {
    // the next item: the index thread 0 wrote with the chunk it staged first
    {
      const int slot = static_cast<int>(pp.kc % pp.stages);
      const uint32_t parity = static_cast<uint32_t>((pp.kc / pp.stages) & 1);
      if (!__all_sync(0xffffffffu, mbar_wait(pp.full + 8u * slot, parity))) {
        if (lane == 0) atomicExch(k.flag, kErrTimeoutFull);
        abort_flag = 1;
        ok = false;
        break;
      }
    }
    const int64_t item = s_chunk_item[pp.kc % pp.stages];
    if (item < 0) break;
    const int c = static_cast<int>(item / k.n_tile_groups);
    const int tg = static_cast<int>(item % k.n_tile_groups);
    const int t = tg * WARPS + warp;
    const Tile& tile = k.tiles[t < k.n_tiles ? t : 0];
    const bool active = t < k.n_tiles && tile.n_valid > 0;   // n_valid 0: padding
    const ProfileDev& prof = k.profs[tile.profile];
    // three walks per radius: the scalar walk carries Q for up to 3 radii
    constexpr bool CQ = !level_mode(MODE) || P <= 3;
    // the float flavours walk the radii in pairs, in every mode
    constexpr bool PAIRED = sizeof(typename A::F) == 4 && P % 2 == 0;
    using TubeWalk = std::conditional_t<PAIRED, Walk2<A, (PAIRED ? P : 2)>, Walk<A, P, CQ>>;
    if (prof.kind == WLN_PROFILE_CONST_B)
      ok = run_item<A, P, WalkB<A, P>, MODE>(k, pp, acc, c, tile, prof, active, &abort_flag, lane,
                                             t);
    else
      ok = run_item<A, P, TubeWalk, MODE>(k, pp, acc, c, tile, prof, active, &abort_flag, lane,
                                          t);
  }

  if (!ok && threadIdx.x == 0) {
    // Let copies already in flight land before the CTA's shared memory goes away.
    for (int32_t q = pp.kc; q < s_prod.issued; ++q)
      (void)mbar_wait(pp.full + 8u * (q % pp.stages), static_cast<uint32_t>((q / pp.stages) & 1));
  }
}

// Failure-detection self-test: wait on an mbarrier phase that nothing will
// complete, with the same bounded wait the Wilson kernel uses; when the wait
// runs out the kernel records it in the device error flag and returns.
__global__ void selftest_wait_kernel(int* flag, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(smem_u32(&bar), 0, limit_ns))
    atomicExch(flag, kErrTimeoutSelfTest);
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
  if (level_mode(mode)) return prec == WLN_PREC_FP64 ? 1 : 4;
  if (mode == kModeLoops) return prec == WLN_PREC_FP64 ? 2 : 4;
  if (prec == WLN_PREC_FP64) return 2;
  return ctx->tune_P ? ctx->tune_P : 4;
}

WilsonPlan make_plan(const wln_ctx* ctx, const Ensemble& e, int n_tiles, wln_prec prec,
                     int mode, int guard_bpg) {
  WilsonPlan p{};
  p.P = plan_points_per_lane(ctx, prec, mode);
  p.mode = mode;
  p.low_angle = ctx->low_angle;
  const bool f64 = prec == WLN_PREC_FP64;
  const bool fixed = f64 || mode != kModeSums;   // shapes that ignore the tuning
  // Group sums: 4 radii x 8 warps, 2 CTAs per SM, 64-row chunks, 2 stages
  // (537 ms on the paper workload against 560 ms for 4 x 4 warps, 3 CTAs per
  // SM, 32 rows, 3 stages, once the low-angle forms made the walk lighter).
  // Per-loop values keep (4, 4); the levels (4, 4), 2 CTAs per SM.
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
  // the precision guard sees whole groups in one item
  if (guard_bpg > 0) p.chain = p.chain < guard_bpg ? guard_bpg : p.chain / guard_bpg * guard_bpg;
  p.n_chains = (e.n_blocks + p.chain - 1) / p.chain;
  p.n_items = static_cast<int64_t>(p.n_chains) * p.n_tile_groups;
  return p;
}

namespace {

cudaError_t launch_any(cudaStream_t s, const WilsonPlan& plan_in, const Ensemble& e,
                       const Tile* tiles, const ProfileDev* profs, const double* rho,
                       int32_t n_groups, int32_t loops_per_group, wln_prec prec,
                       double* partial, int64_t n_points, int* d_flag, int64_t* launches,
                       double* loops_out, const GuardBufs* guard, int* grid_out = nullptr,
                       int* item_counter = nullptr) {
  WilsonPlan plan = plan_in;
  if (plan.stages > kMaxStages) return cudaErrorInvalidConfiguration;
  KParams kp{};
  kp.item_counter = item_counter;
  kp.loops_out = loops_out;
  kp.blocks = e.blocks; kp.n_blocks = e.n_blocks; kp.ppl = e.ppl; kp.n_loops = e.n_loops;
  kp.tiles = tiles; kp.n_tiles = plan.n_tiles; kp.profs = profs; kp.rho = rho;
  kp.lpg = loops_per_group; kp.G = n_groups; kp.partial = partial; kp.n_points = n_points;
  kp.rows = plan.rows; kp.stages = plan.stages; kp.chain = plan.chain;
  kp.n_tile_groups = plan.n_tile_groups; kp.n_chains = plan.n_chains; kp.n_items = plan.n_items;
  kp.flag = d_flag;
  kp.stats = e.stats;
  kp.sub_stats = e.sub_stats;
  kp.n_sub = e.n_sub;
  kp.maxlen = e.maxlen;
  kp.low_angle = plan.low_angle;
  if (guard) kp.guard = *guard;
  const size_t smem = smem_bytes(plan, e.ppl);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
#define WLN_CASE_L(A, P_, W_, M_)                                                    \
  if (plan.P == P_ && plan.warps == W_ && plan.mode == M_) {                         \
    const int occ = occupancy<A, P_, W_, M_>(smem);                                  \
    const int64_t g = static_cast<int64_t>(sms) * occ;                               \
    const int grid = static_cast<int>(g < plan.n_items ? g : plan.n_items);          \
    if (grid_out) { *grid_out = grid; return cudaSuccess; }                          \
    if (item_counter) {                                                              \
      const cudaError_t e = cudaMemsetAsync(item_counter, 0, sizeof(int), s);         \
      if (e != cudaSuccess) return e;                                                \
    }                                                                                \
    ++*launches;                                                                     \
    return launch_t<A, P_, W_, M_>(s, kp, grid, smem);                               \
  }
#define WLN_CASE(A, P_, W_) WLN_CASE_L(A, P_, W_, kModeSums)
  if (plan.mode == kModeLevels) {
    switch (prec) {
      case WLN_PREC_FP32_COMP: WLN_CASE_L(F32Comp, 4, 4, kModeLevels) break;
      case WLN_PREC_FP32_NAIVE: WLN_CASE_L(F32Naive, 4, 4, kModeLevels) break;
      case WLN_PREC_FP64: WLN_CASE_L(F64, 1, 4, kModeLevels) break;
    }
    return cudaErrorInvalidConfiguration;
  }
  if (plan.mode == kModeNested) {
    switch (prec) {
      case WLN_PREC_FP32_COMP: WLN_CASE_L(F32Comp, 4, 4, kModeNested) break;
      case WLN_PREC_FP32_NAIVE: WLN_CASE_L(F32Naive, 4, 4, kModeNested) break;
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
                          double* partial, int64_t n_points, int* d_flag, int64_t* launches,
                          const GuardBufs* guard, int* item_counter) {
  return launch_any(s, plan, e, tiles, profs, rho, n_groups, loops_per_group, prec, partial,
                    n_points, d_flag, launches, nullptr, guard, nullptr, item_counter);
}

int wilson_grid(const WilsonPlan& plan, const Ensemble& e, wln_prec prec) {
  int grid = 0;
  int64_t none = 0;
  if (launch_any(nullptr, plan, e, nullptr, nullptr, nullptr, 1, e.n_loops, prec, nullptr, 0,
                 nullptr, &none, nullptr, nullptr, &grid) != cudaSuccess)
    return 0;
  return grid;
}

cudaError_t launch_wilson_loops(cudaStream_t s, const WilsonPlan& plan, const Ensemble& e,
                                const Tile* tiles, const ProfileDev* profs, const double* rho,
                                wln_prec prec, double* out, int* d_flag, int64_t* launches,
                                int* item_counter) {
  // groups play no part; lpg = n_loops keeps the group arithmetic in range
  return launch_any(s, plan, e, tiles, profs, rho, 1, e.n_loops, prec, nullptr, 0, d_flag,
                    launches, out, nullptr, nullptr, item_counter);
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
