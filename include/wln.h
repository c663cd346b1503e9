/*
 * wln.h — C ABI of the GB300 worldline Wilson-loop library (libwln.so).
 *
 * The library computes ensemble averages of Wilson loops in cylindrically
 * symmetric magnetic fields by worldline numerics, following D. Mazur and
 * J. S. Heyl, "Parallel Worldline Numerics: Implementation and Error
 * Analysis" (arXiv:1407.7486):
 *   - unit loops of N points drawn on the device (Sec. "Loop Generation");
 *   - per loop and per point (rho_cm, T): the loop scaled by sqrt(T), shifted
 *     to x_cm = (rho_cm, 0), the phase e * closed line integral of A along
 *     straight segments (Sec. "Wilson Loop", Eqs. rhoi-Ci) and the spin factor
 *     cosh(e int B dtau) (Sec. "Fermion Part", Eq. Wfermfpl);
 *   - sums of W over contiguous groups of loops, and the group statistics
 *     (Sec. "Grouping Worldlines");
 *   - the effective-action density by quadrature over rho_cm and T, done for
 *     every group separately (Eq. cylEA; Sec. "Computing an Effective Action").
 *
 * Units: e = m = 1.  A flux-tube profile has raw flux F and radius lambda:
 *   A_phi(rho) = F rho / (2 pi (lambda^2 + rho^2)),
 *   e B(rho)   = (F / (pi lambda^2)) (1 + rho^2/lambda^2)^-2,
 * i.e. f(rho^2) = rho^2/(lambda^2 + rho^2) and calF = F / (2 pi).
 *
 * Conventions for every call:
 *   - Every call returns a wln_status.  On failure the context keeps a
 *     message (wln_last_error).  The library never aborts the process.
 *   - Device work is ordered on the context's stream.  Unless stated
 *     otherwise, output arrays may be host or device memory; the library
 *     inspects each pointer.  A call with any host output synchronises the
 *     stream before it returns.  A call whose outputs are all device
 *     pointers returns as soon as the work is queued.
 *   - Arrays described as "host" must be host memory.  The caller owns
 *     every array it passes.  The library owns contexts and ensembles.
 *   - Errors detected on the device (a bounded wait that ran out) are
 *     reported as WLN_ETIMEOUT by the next call that synchronises, or by
 *     wln_synchronize.
 */
#ifndef WLN_H_
#define WLN_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wln_ctx wln_ctx;            /* opaque; one device, one stream */
typedef struct wln_ensemble wln_ensemble;  /* opaque; device-resident loops */

typedef enum {
  WLN_OK = 0,
  WLN_EINVAL = 1,    /* an argument breaks a documented rule */
  WLN_ENOMEM = 2,    /* device or pinned host allocation failed */
  WLN_ECUDA = 3,     /* a CUDA runtime call failed (message holds its text) */
  WLN_ETIMEOUT = 4,  /* a bounded device-side wait ran out */
  WLN_EBUSY = 5      /* resource in use (server full, request pending) */
} wln_status;

typedef enum {
  WLN_PREC_FP64 = 0,        /* segment sums and transcendentals in double */
  WLN_PREC_FP32_COMP = 1,   /* FP32 segments, compensated (Kahan) sums, phase
                               range-reduced in turns, W and its sums in FP64 */
  WLN_PREC_FP32_NAIVE = 2   /* FP32 segments and plain FP32 sums */
} wln_prec;

enum {
  WLN_PROFILE_FLUX_TUBE = 0,  /* uses F and lambda (lambda > 0) */
  WLN_PROFILE_CONST_B = 1     /* uses B: phase = B * area, spin = B T */
};

typedef struct {
  int32_t kind;       /* WLN_PROFILE_* */
  int32_t reserved;   /* set to 0 */
  double F;           /* flux-tube raw flux */
  double lambda;      /* flux-tube radius */
  double B;           /* constant field strength */
} wln_profile;

/* Components of a group sum, in this order (WLN_K per point and group). */
#define WLN_K 5
enum {
  WLN_C_SCAL = 0,     /* sum over the group of (W_scal - 1), W_scal = cos(phase) */
  WLN_C_FERM = 1,     /* sum of (W_ferm - 1), W_ferm = cos(phase) cosh(spin) */
  WLN_C_SIN = 2,      /* sum of sin(phase) (imaginary part, zero on average) */
  WLN_C_SCAL_SQ = 3,  /* sum of (W_scal - 1)^2 */
  WLN_C_FERM_SQ = 4   /* sum of (W_ferm - 1)^2 */
};

/* Components of a discretisation-level group sum (WLN_KL per point and
 * group; see wln_wilson_levels): W - 1 at N, N/2 and N/4 points per loop. */
#define WLN_KL 6
enum {
  WLN_L_SCAL_N = 0,   /* sum of (W_scal - 1) at level N */
  WLN_L_FERM_N = 1,   /* sum of (W_ferm - 1) at level N */
  WLN_L_SCAL_N2 = 2,  /* level N/2 */
  WLN_L_FERM_N2 = 3,
  WLN_L_SCAL_N4 = 4,  /* level N/4 */
  WLN_L_FERM_N4 = 5
};

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  `cuda_stream` is a
 * cudaStream_t (NULL: the legacy default stream).  The caller keeps
 * ownership of the stream. */
wln_status wln_create(wln_ctx** out, int device, void* cuda_stream);
wln_status wln_destroy(wln_ctx* ctx);
/* Replace the stream used by later calls. */
wln_status wln_set_stream(wln_ctx* ctx, void* cuda_stream);
/* Wait for all queued work; report device-side errors. */
wln_status wln_synchronize(wln_ctx* ctx);
/* Message of the last failure on this context ("" if none).  The string is
 * owned by the context and valid until its next call. */
const char* wln_last_error(const wln_ctx* ctx);
/* Number of kernel launches this context has issued since creation. */
int64_t wln_launch_count(const wln_ctx* ctx);

/*
 * Failure-detection self-test (no counterpart in the paper): one kernel waits
 * on a device barrier that nothing completes, using the bounded wait of the
 * Wilson kernel with a limit of timeout_ms (1..2000).  The wait runs out, the
 * kernel records it and returns, and this call reports WLN_ETIMEOUT; the
 * context stays usable.  Anything else means the timeout path is broken.
 */
wln_status wln_selftest_wait(wln_ctx* ctx, int32_t timeout_ms);

/* --------------------------------------------------------------- ensembles */

/*
 * Draw n_loops closed unit loops of ppl points (Sec. "Loop Generation"):
 * loops loop0 .. loop0 + n_loops - 1 of the ensemble defined by seed, so
 * ranks can hold disjoint slices of one ensemble (loop0 + n_loops < 2^32).
 * Loop l uses Philox-4x32-10 (Salmon et al., SC'11) with counter (j, l, 0, 0),
 * j = 0 .. ppl/2 - 1, and key (seed & 0xffffffff, seed >> 32).  The four
 * words u0..u3 of call j map to u = (k + 1/2) 2^-32, and Box-Muller gives
 *   (u0, u1) -> (xi_x[2j], xi_y[2j]),  (u2, u3) -> (xi_x[2j+1], xi_y[2j+1]),
 *   z = sqrt(-2 ln u_a) (cos 2 pi u_b, sin 2 pi u_b),  xi = z sqrt(2/ppl),
 * the discretised free action's increment law (variance 2/ppl per component).
 * Then, in double precision: xi <- xi - mean(xi) (closure), y_k = sum_{j<k}
 * xi_j, y <- y - mean(y) (common centre of mass, d-loop step 5).  The points
 * are stored as float on the device.  keep_fp64 != 0 also keeps a double copy.
 * The raw increments are held in the context's scratch between drawing and
 * closing: 16 bytes per point plus chunk sums (a sixteenth of that from
 * ppl = 256 on), in slices of blocks of at most 1 GiB; WLN_ENOMEM if it
 * cannot grow.
 * Rules: ppl a power of two, 4 <= ppl <= 16384; 1 <= n_loops <= 2^24.
 * The call synchronises.  It returns WLN_EINVAL if two consecutive stored
 * points coincide (a zero-length segment), which has negligible probability.
 */
wln_status wln_gen_loops(wln_ctx* ctx, uint64_t seed, int64_t loop0, int32_t n_loops,
                         int32_t ppl, int32_t keep_fp64, wln_ensemble** out);

/*
 * The paper's own generator, d-loops (Sec. "Loop Generation", Eqs. yn2 and
 * ynk): from the point y_N = y_0, level k (N_k = 2^k points) adds the points
 * q N/N_k (q odd), each Gaussian about the mean of its two level-(k-1)
 * neighbours with variance 1/N_k per component; at N_k = ppl the common
 * centre of mass is removed (step 5).  Same joint law as wln_gen_loops,
 * different draws: Gaussian number m in creation order (level 1 first, then
 * q increasing within a level) uses Philox call m/2 with counter
 * (m/2, loop, 1, 0), (u0,u1) for even m and (u2,u3) for odd m, through the
 * same Box-Muller.  Arguments, rules and result as wln_gen_loops; the call
 * needs 16 * 32 * ceil(n_loops/32) * ppl bytes of scratch.
 */
wln_status wln_gen_dloops(wln_ctx* ctx, uint64_t seed, int64_t loop0, int32_t n_loops,
                          int32_t ppl, int32_t keep_fp64, wln_ensemble** out);

/*
 * Make an ensemble from given loops, e.g. a saved one.  xy is
 * float[n_loops][2][ppl] (x block, then y block of each loop).  It may be host
 * or device memory.  Same rules as wln_gen_loops, and no two consecutive points
 * of a loop (cyclically) may coincide.  The library copies the data.  The call
 * synchronises.
 */
wln_status wln_ensemble_from_host(wln_ctx* ctx, const float* xy, int32_t n_loops,
                                  int32_t ppl, wln_ensemble** out);
/*
 * Free an ensemble.  With a context (on the ensemble's device) the call waits
 * for the context's stream, and the context keeps the device memory of up to
 * two freed ensembles for the next ensemble of the same shape it makes (no
 * cudaMalloc / cudaFree, which wait for the whole device, in a loop that
 * draws and frees an ensemble every step); wln_destroy releases it.  Work on
 * the ensemble queued on other streams must be complete before the call.
 * With ctx NULL the memory is released at once.
 */
wln_status wln_free_ensemble(wln_ctx* ctx, wln_ensemble* ens);
/* Sizes of an ensemble; any output may be NULL. */
wln_status wln_ensemble_info(const wln_ensemble* ens, int32_t* n_loops, int32_t* ppl,
                             int32_t* has_fp64);
/*
 * Copy the loops out as float[n_loops][2][ppl] and/or double[n_loops][2][ppl]
 * (host or device).  Either pointer may be NULL.  The double copy needs
 * keep_fp64.
 */
wln_status wln_loops_copy(wln_ctx* ctx, const wln_ensemble* ens, float* xy_f32,
                          double* xy_f64);
/*
 * The raw Philox words used for loops loop0 .. loop0 + n_loops - 1 (the
 * first step of wln_gen_loops).  out is uint32[n_loops][n_calls][4], host or
 * device.
 */
wln_status wln_philox_stream(wln_ctx* ctx, uint64_t seed, int64_t loop0, int32_t n_loops,
                             int32_t n_calls, uint32_t* out);

/* ------------------------------------------------------------ Wilson loops */

/*
 * Group sums of Wilson loops for a batch of profiles, each with its own grid.
 *
 * Points: profile q has radii rho_cm[rho_off[q] .. rho_off[q+1]) and proper
 * times T[T_off[q] .. T_off[q+1]).  Its points are all (rho, T) pairs.
 * Point index: p = base_q + iT * n_rho_q + i_rho, where base_q counts the
 * points of profiles 0..q-1.  For each point and each loop the loop is
 * r_k = (rho_cm, 0) + sqrt(T) y_k, k = 0..N-1, closed by straight segments
 * r_k -> r_{k+1 mod N}:
 *   phase = e * closed int A.dr along the segments, exactly (Eqs. rhoi-Ci);
 *   spin  = e int_0^T B dtau, each segment taking proper time T/N, exactly.
 * W_scal = cos(phase), W_ferm = cos(phase) cosh(spin) (Eq. wilsonloop, its
 * real part).
 * Group g holds loops g n/G .. (g+1) n/G - 1 (Sec. "Grouping Worldlines").
 *
 * group_sums: double[n_points][n_groups][WLN_K], host or device (see
 * WLN_C_*).  Every point's sums are accumulated in one fixed order, whatever
 * else is in the batch, so a point's result does not depend on the batch.
 * profiles, rho_cm, rho_off, T, T_off: host arrays.
 * Rules: n_groups >= 2 divides n_loops; T > 0; rho_cm >= 0; lambda > 0 for
 * flux tubes; every profile has at least one rho and one T.
 *
 * Precision guard (WLN_PREC_FP32_COMP, flux tubes, groups of a whole number
 * of 32-loop blocks, at most 64 of them; see wln_set_precision_guard): the
 * spinor sums (WLN_C_FERM, WLN_C_FERM_SQ) of a group are dominated by its
 * loops of largest spin, whose float rounding cosh(spin) magnifies (Sec.
 * "Uncertainties and the Fermion Problem").  The float pass estimates each
 * group's spinor error from a rounding model of the float walk; where it
 * exceeds half of 1e-6 max(1, <cosh spin>) it recomputes the loops carrying
 * most of it in double-float (~2^-44) and corrects the sums.  The other
 * components stay float.  A group with more than 64 such loops per radius
 * keeps the rest in float (counted in wln_precision_guard_stats).  The
 * corrections are applied in a fixed order, so results stay independent of
 * the batch and of scheduling.  The queue of loops to recompute holds 64
 * entries per (point, group) whose spin can reach 2 at all (T eB at the
 * closest approach to the axis that the ensemble's loops allow), everything
 * a pass can select, when that is at most 2^22 entries.  Beyond that it
 * starts with 8 per such (point, group); the call then waits for the float
 * pass to read how many loops it selected, and if they exceed the queue it
 * runs the pass again with the queue sized to that number (the selection is
 * deterministic).  A queue that still overflows leaves those loops in float
 * and makes the call (for a device output, the next synchronising call)
 * return WLN_ENOMEM.
 */
wln_status wln_wilson_avg(wln_ctx* ctx, const wln_ensemble* ens,
                          const wln_profile* profiles, int32_t n_profiles,
                          const double* rho_cm, const int32_t* rho_off,
                          const double* T, const int32_t* T_off,
                          int32_t n_groups, wln_prec prec, double* group_sums);

/*
 * The precision guard of the FP32-compensated group sums (wln_wilson_avg,
 * wln_wilson_avg_noalloc, batches created afterwards, servers created
 * afterwards): enabled = 1 (the default) or 0.  enabled = 2 recomputes every
 * loop of the blocks it records (those reaching spin 2), up to 64 per group
 * and radius, whatever the error estimate: a check of the double-float walk
 * against the oracle, not for production.  No paper counterpart: the paper
 * runs FP32 throughout.
 */
wln_status wln_set_precision_guard(wln_ctx* ctx, int32_t enabled);

/*
 * Running totals of the precision guard over the guarded launches on this
 * context (and on batches and servers created from it): loops recomputed in
 * double-float, launches, (group, radius) selections dropped because the
 * queue was full, and (group, radius) selections left in float because 64
 * loops would not bring the estimate under the budget.  Waits for the context's
 * stream; reset = 1 zeroes the totals.  Any pointer may be NULL.
 */
wln_status wln_precision_guard_stats(wln_ctx* ctx, int64_t* escalated_loops, int64_t* launches,
                                     int64_t* overflows, int64_t* saturated, int32_t reset);

/*
 * wln_wilson_avg without any allocation: the same group sums, with the same
 * arguments and results, but the call allocates no device or pinned host
 * memory.  The paper has no counterpart; this entry point exists for callers
 * that cannot allocate device memory themselves or through the library: a
 * host framework whose own caching allocator owns the device memory and
 * forbids direct cudaMalloc, a latency-bound loop that must not take the
 * implicit device synchronisation of cudaMalloc/cudaFree, or a service that
 * reserved the device memory up front.
 *
 * Working memory (inputs copied from the host, the work list, the partial
 * sums, and the group sums when group_sums is host memory) comes from one
 * 64 MiB array compiled into the library.  Every GPU on which the library is
 * used holds that array until the process exits.  A problem that needs more
 * than 64 MiB returns WLN_EINVAL with the size it needed: the partial sums take
 * (chains + n_groups) * n_points * WLN_K * 8 bytes.
 * The first call on a device looks up the array's device address (and may load
 * the library's device code).  The call must not be made inside a CUDA stream
 * capture: it copies its inputs from host memory and, for a host output,
 * synchronises the stream.  All calls share the array and it keeps the last
 * call's contents: every word a call reads is written by that call first, so
 * nothing needs clearing, but calls whose GPU work overlaps in time (other
 * streams, other threads) race on it and must be serialised by the caller.
 *
 * Inputs (profiles, grids, offsets) may be reused as soon as the call returns:
 * pageable host inputs are staged by the copy itself, and when any input is
 * page-locked the call waits until the stream has read it.  Errors of a
 * bounded device wait: with a host output the call waits for the stream and
 * returns WLN_ETIMEOUT (and clears the device flag, so later calls start
 * clean); with a device output the flag is read by the next synchronising
 * call, as for wln_wilson_avg.  The precision guard's queue lives in the same
 * array, sized as wln_wilson_avg first sizes it; it cannot grow, so a pass
 * that selects more loops than it holds returns WLN_ENOMEM the same way.
 */
wln_status wln_wilson_avg_noalloc(wln_ctx* ctx, const wln_ensemble* ens,
                                  const wln_profile* profiles, int32_t n_profiles,
                                  const double* rho_cm, const int32_t* rho_off,
                                  const double* T, const int32_t* T_off,
                                  int32_t n_groups, wln_prec prec, double* group_sums);

/*
 * Discretisation levels (Sec. "Estimating the Discretization Uncertainties"):
 * every loop of N points is split into three interleaved closed sub-loops,
 *   circle:   points 0, 2, 4, ...          (N/2 points)
 *   square:   points 1, 5, 9, ... (1 mod 4) (N/4 points)
 *   triangle: points 3, 7, 11, ... (3 mod 4) (N/4 points)
 * each walked like a loop in wln_wilson_avg (straight segments, exact
 * integrals, proper time T/N' per segment for N' points; the same centre of
 * mass, no re-centring).  With o, s, t the phases of the three sub-loops,
 *   W_N/4 = e^{i (t + s)/2},  W_N/2 = e^{i o},  W_N = e^{i o/2} e^{i s/4} e^{i t/4},
 * and the spin integrals combine with the same weights (W_ferm = cos(phase)
 * cosh(spin) at each level).  group_sums: double[n_points][n_groups][WLN_KL]
 * (see WLN_L_*), host or device.  Arguments and rules as wln_wilson_avg, and
 * the ensemble's ppl must be a multiple of 4 and at least 8.  The pass costs
 * about what wln_wilson_avg does (N segments per loop and point).
 */
wln_status wln_wilson_levels(wln_ctx* ctx, const wln_ensemble* ens,
                             const wln_profile* profiles, int32_t n_profiles,
                             const double* rho_cm, const int32_t* rho_off,
                             const double* T, const int32_t* T_off,
                             int32_t n_groups, wln_prec prec, double* group_sums);

/*
 * Every loop's W - 1 at every point: the per-worldline values behind the
 * correlation coefficients of Eq. corrcoef (Sec. "Correlations between
 * Wilson Loops") and behind any regrouping (wln_group_sums_loops).
 * Arguments and rules as wln_wilson_avg, without groups.
 * loop_values: double[n_points][n_loops][2] = (W_scal - 1, W_ferm - 1),
 * host or device (16 bytes per loop and point).
 */
wln_status wln_wilson_loops(wln_ctx* ctx, const wln_ensemble* ens,
                            const wln_profile* profiles, int32_t n_profiles,
                            const double* rho_cm, const int32_t* rho_off,
                            const double* T, const int32_t* T_off, wln_prec prec,
                            double* loop_values);

/* -------------------------------------------------------------- statistics */

/*
 * Group statistics of component `comp` of group sums (layout as
 * wln_wilson_avg), Sec. "Grouping Worldlines":
 *   m_g(p) = S_g(p) / loops_per_group       (the group means)
 *   mean(p) = (1/G) sum_g m_g(p)             (= the mean over all loops)
 *   sem(p) = sqrt(sum_g (m_g - mean)^2 / (G (G - 1)))
 *   jk_var(p) = (G-1)/G sum_g (m_(-g) - mean)^2, m_(-g) = (G mean - m_g)/(G-1)
 *   cov(p, q) = sum_g (m_g(p) - mean(p)) (m_g(q) - mean(q)) / (G (G - 1))
 * For comp = WLN_C_SCAL or WLN_C_FERM the mean is <W> - 1.
 * Arrays: group_sums double[n_points][n_groups][WLN_K]; mean, sem, jk_var
 * double[n_points]; cov double[n_points][n_points].  jk_var and cov may be
 * NULL.  All arrays are host or device.
 */
wln_status wln_jackknife(wln_ctx* ctx, const double* group_sums, int32_t n_points,
                         int32_t n_groups, int32_t loops_per_group, int32_t comp,
                         double* mean, double* sem, double* jk_var, double* cov);
/*
 * As wln_jackknife, with the covariance (symmetric) as its upper triangle,
 * row by row: cov_packed double[n_points (n_points + 1) / 2], cov(p, q) for
 * q >= p at p n_points - p (p - 1) / 2 + (q - p).  The same values as the
 * full matrix's, bit for bit, in half the bytes (host or device).
 */
wln_status wln_jackknife_packed(wln_ctx* ctx, const double* group_sums, int32_t n_points,
                                int32_t n_groups, int32_t loops_per_group, int32_t comp,
                                double* mean, double* sem, double* jk_var, double* cov_packed);

/*
 * Group sums from per-loop values (wln_wilson_loops), with the paper's
 * randomised grouping as an option (Sec. "Grouping Worldlines": assign the
 * worldlines to groups at random, anew for every evaluation of the
 * integrand, so that the group means of different evaluations decorrelate).
 *   shuffle == 0: group g holds loops g n/G .. (g+1) n/G - 1 (the grouping
 *                 of wln_wilson_avg);
 *   shuffle != 0: the loops of point p are put in the order a[0..n-1] of a
 *                 Fisher-Yates shuffle: a = identity; for t = 0 .. n-2,
 *                 i = n-1-t, j = (u (i+1)) >> 32, swap a[i], a[j], where u is
 *                 word t mod 4 of Philox-4x32-10 at counter (t/4, p, 2, 0) with
 *                 key (seed & 0xffffffff, seed >> 32); group g holds loops
 *                 a[g n/G .. (g+1) n/G - 1].
 * Each group is summed in that order.  group_sums: double[n_points][n_groups]
 * [WLN_K]; WLN_C_SIN is NaN (the imaginary part is not in the per-loop
 * values); the squares are sums of squared per-loop values.  perm:
 * int32[n_points][n_loops], the order used (only with shuffle), or NULL.
 * loop_values, group_sums and perm are host or device.  Rules: n_groups >= 2
 * divides n_loops; n_points <= 2^32.
 */
wln_status wln_group_sums_loops(wln_ctx* ctx, const double* loop_values, int64_t n_points,
                                int32_t n_loops, int32_t n_groups, int32_t shuffle,
                                uint64_t seed, double* group_sums, int32_t* perm);

/*
 * Correlation coefficients of Eq. corrcoef between the evaluation in row ref
 * and every row of x, over the row's samples:
 *   r = sum (x - <x>)(y - <y>) / sqrt(sum (x - <x>)^2 sum (y - <y>)^2),
 * element n of row r at x[(r n_samples + n) stride + comp]: per-loop values
 * (n_samples = n_loops, stride 2, comp 0 scalar / 1 spinor) or group sums
 * (n_samples = n_groups, stride WLN_K, comp WLN_C_*), giving the three
 * curves of the paper's Fig. corr (loops, groups, shuffled groups).
 * out: double[n_rows]; NaN for a row without spread.  Host or device.
 */
wln_status wln_corrcoef(wln_ctx* ctx, const double* x, int32_t n_rows, int32_t n_samples,
                        int32_t stride, int32_t comp, int32_t ref, double* out);

/*
 * Standard error in the mean over individual loops (Sec. "The Worldline
 * Ensemble Distribution is not Normal"), from the sums of W - 1 (comp_sum) and
 * (W - 1)^2 (comp_sq):
 *   sqrt((sum w^2 - (sum w)^2 / n_loops) / (n_loops (n_loops - 1))).
 * out: double[n_points], host or device.
 */
wln_status wln_loop_sem(wln_ctx* ctx, const double* group_sums, int32_t n_points,
                        int32_t n_groups, int32_t n_loops, int32_t comp_sum,
                        int32_t comp_sq, double* out);

/*
 * Discretisation levels from nested loops: W - 1 of every loop through all
 * N points, through the even points (N/2) and through the points 0 mod 4
 * (N/4), each walked like a loop in wln_wilson_avg (proper time T/N' per
 * segment; the same centre of mass).  Same layout, arguments and rules as
 * wln_wilson_levels.  Read as printed, the paper's level N of
 * wln_wilson_levels is a point-weighted mean of interleaved sub-loop phases
 * rather than the N-point loop, so it is not a discretisation hierarchy;
 * these nested levels are, and wln_extrapolate's parabola in 1/N applies to
 * them.  The pass walks 1.75 N segments per loop and point.
 */
wln_status wln_wilson_levels_nested(wln_ctx* ctx, const wln_ensemble* ens,
                                    const wln_profile* profiles, int32_t n_profiles,
                                    const double* rho_cm, const int32_t* rho_off,
                                    const double* T, const int32_t* T_off,
                                    int32_t n_groups, wln_prec prec, double* group_sums);

/*
 * Extrapolation to infinitely many points per loop and the discretisation
 * uncertainty (Sec. "Estimating the Discretization Uncertainties"), from the
 * level sums of wln_wilson_levels or wln_wilson_levels_nested (the parabola
 * presumes genuine levels of one loop, which the nested ones are).  For x in
 * (scalar, spinor) and each point:
 *   m_L = mean over all loops of W - 1 at level L in (N, N/2, N/4);
 *   W_inf - 1 = 8/3 m_N - 2 m_N/2 + 1/3 m_N/4 (the parabola in 1/N through
 *   the three levels, taken at 1/N = 0);
 *   sem_inf = the group standard error of that combination (it is linear, so
 *   each group's extrapolation is the combination of its means);
 *   delta = |m_N - (W_inf - 1)|, the paper's discretisation uncertainty.
 * out: double[n_points][2][6] = (m_N, m_N/2, m_N/4, W_inf - 1, sem_inf,
 * delta) for the scalar, then the spinor loop.  level_sums and out host or
 * device.
 */
wln_status wln_extrapolate(wln_ctx* ctx, const double* level_sums, int32_t n_points,
                           int32_t n_groups, int32_t loops_per_group, double* out);

/*
 * Effective-action density per group and its group mean and standard error
 * (Eq. cylEA; Sec. "Grouping Worldlines": integrate each group separately):
 *   Gamma_g = (1/4 pi) int rho drho int dT e^{-T}/T^3 {<W>_g - 1 - c (eB T)^2}
 * with c = 1/3 for the spinor loop (spinor != 0, component WLN_C_FERM) and
 * c = -1/6 for the scalar loop (component WLN_C_SCAL, counterterm of Eq.
 * scalI).  eB is the profile's field at rho_cm.  Quadrature: Simpson in rho
 * on evenly spaced radii, and Simpson in u = ln T on geometrically spaced
 * proper times (dT = T du).  An even point count ends with a 3/8 panel; two
 * points use the trapezoid; one point gives zero.
 * Profiles and grids as in wln_wilson_avg (host arrays); each profile's rho
 * must be evenly spaced and its T geometric (relative tolerance 1e-9), else
 * WLN_EINVAL.  group_sums as written by wln_wilson_avg for the same batch.
 * gamma_groups: double[n_profiles][n_groups] or NULL; gamma_mean_sem:
 * double[n_profiles][2] (mean, standard error).  Host or device.
 */
wln_status wln_effective_action(wln_ctx* ctx, const wln_profile* profiles,
                                int32_t n_profiles, const double* rho_cm,
                                const int32_t* rho_off, const double* T,
                                const int32_t* T_off, const double* group_sums,
                                int32_t n_groups, int32_t loops_per_group, int32_t spinor,
                                double* gamma_groups, double* gamma_mean_sem);

/*
 * Quadrature grids of the full effective action.  Sec. "Computing an
 * Effective Action" maps integrals over [0, inf) to a finite interval with
 * x = 1/(1 + v/scale) and applies Simpson's rule in x.  Per profile:
 *   rho_kind  WLN_GRID_LINEAR: evenly spaced radii, Simpson over [rho_0, rho_last];
 *             WLN_GRID_MAPPED: radii from wln_mapped_grid(n_rho, rho_scale, rho_0),
 *             integral over [rho_0, inf).
 *   T_kind    WLN_GRID_LOG: geometric times, Simpson in u = ln T over [T_0, T_last];
 *             WLN_GRID_MAPPED: times from wln_mapped_grid(n_T, T_scale, T_0),
 *             integral over [T_0, inf).
 *   small_T   != 0: add the exact integral over [0, T_0] of the small-T
 *             expansion of the integrand (Eq. fermI, or Eq. scalI for the
 *             scalar loop; m = 1, eB at rho), the split of Sec. "Renormalization"
 *             with a = T_0.
 * A mapped axis of n nodes v_i = scale (1/x_i - 1), x_i = x0 (n - i)/n,
 * x0 = 1/(1 + v_0/scale), takes Simpson weights over the n + 1 points
 * x_0 = 0 .. x_n = x0 (the integrand is 0 at x = 0, v = inf) times
 * dv/dx = scale/x^2.  An even point count ends with a 3/8 panel.
 */
enum { WLN_GRID_LINEAR = 0, WLN_GRID_LOG = 1, WLN_GRID_MAPPED = 2 };
typedef struct {
  int32_t rho_kind;   /* WLN_GRID_LINEAR or WLN_GRID_MAPPED */
  int32_t T_kind;     /* WLN_GRID_LOG or WLN_GRID_MAPPED */
  double rho_scale;   /* mapped radii: scale (> 0) */
  double T_scale;     /* mapped times: T_max (> 0) */
  int32_t small_T;    /* add the small-T part over [0, T_0] */
  int32_t reserved;   /* set to 0 */
} wln_quad;

/*
 * Nodes of a mapped grid, ascending: out[i] = scale (1/x_i - 1) with
 * x_i = x0 (n - i)/n, x0 = 1/(1 + start/scale), i = 0 .. n-1 (out[0] = start).
 * Host only; no context.  Rules: n >= 1, scale > 0, start >= 0, out host.
 */
wln_status wln_mapped_grid(int32_t n, double scale, double start, double* out);

/*
 * The full effective action with error bars and the LCF comparison
 * (Eq. cylEA; Sec. "Renormalization"; Sec. "Computing an Effective Action";
 * Eq. LCFferm and Sec. "Verification and Validation").  For profile q with
 * radii rho_i and times T_j (the grids its group sums were computed on) and
 * quadrature weights w_j (T axis) and w_i (rho axis) from quad[q]:
 *   I_g(rho_i, T_j) = e^{-T}/T^3 (m_g - c (eB T)^2),  m_g = group mean of W - 1,
 *   D_g(rho_i) = [int_0^{T_0} of the small-T expansion] + sum_j w_j I_g(rho_i, T_j),
 *   Gamma_g = (1/4 pi) sum_i w_i rho_i D_g(rho_i),
 * c = 1/3 for the spinor loop (spinor != 0, WLN_C_FERM), -1/6 for the scalar
 * loop (WLN_C_SCAL); eB = eB(rho_i) of the profile.  The LCF approximation
 * replaces m_g - c (eB T)^2 by the constant-field bracket x coth x - 1 - x^2/3
 * (scalar: x / sinh x - 1 + x^2/6), x = eB(rho_i) T_j, with the same
 * quadrature and small-T part.
 * Outputs (host or device; any of gamma_groups, density, integrand may be NULL):
 *   gamma_groups double[n_profiles][n_groups]  Gamma_g
 *   gamma        double[n_profiles][3]          mean over groups, its standard error, LCF
 *   density      double[n_rho_total][3]         D(rho): mean, standard error, LCF
 *                                               (indexed like rho_cm)
 *   integrand    double[n_points][3]            I(rho, T): mean, standard error, LCF
 *                                               (points ordered as in wln_wilson_avg)
 * quad: host array of n_profiles (NULL: every profile LINEAR radii, LOG times,
 * no small-T part, as wln_effective_action).  Grids must match their kind
 * (relative tolerance 1e-9), else WLN_EINVAL.
 */
wln_status wln_effective_action_full(wln_ctx* ctx, const wln_profile* profiles,
                                     int32_t n_profiles, const double* rho_cm,
                                     const int32_t* rho_off, const double* T,
                                     const int32_t* T_off, const wln_quad* quad,
                                     const double* group_sums, int32_t n_groups,
                                     int32_t loops_per_group, int32_t spinor,
                                     double* gamma_groups, double* gamma, double* density,
                                     double* integrand);

/* ------------------------------------------------------- runtime: tuning */

/*
 * Work decomposition of later Wilson launches on this context (0 = automatic):
 * points_per_lane (radii held by one lane) and warps per CTA, one of the
 * shapes (2, 8), (4, 4), (4, 8), (8, 8) (automatic: (4, 8), two CTAs per
 * SM, with 64 rows and 2 stages), rows (float4 rows of loop data per staged
 * chunk, a power of two), stages (chunks in flight, 2..8) and chain_blocks
 * (consecutive 32-loop blocks per work item).  The paper has no counterpart
 * (its kernel used one
 * thread per loop and one launch per point); the autotuner sets these.  The
 * FP64 path, the discretisation levels and the per-loop values keep their
 * own shapes.
 */
wln_status wln_set_tuning(wln_ctx* ctx, int32_t points_per_lane, int32_t warps, int32_t rows,
                          int32_t stages, int32_t chain_blocks);

/*
 * The float walks evaluate theta = atan2(sqrt(D), Q0 + B) (the angle a
 * segment subtends at the field axis, Sec. "Wilson Loop", Eqs. rhoi-Ci) in
 * cheaper forms where every segment of a 32-loop block is known to subtend a
 * small angle.  With u = |d| / sqrt(lambda^2 + (rho_cm - sqrt(T) |y|max)_+^2),
 * |d| the block's longest scaled segment (times 4 for the sub-loops of the
 * discretisation levels), theta <= atan(u / (1 - u)):
 *   level 1: blocks with u <= 0.45 (theta <= pi/4) skip the arctangent's
 *            range fold and octant unfolding -- the same angle bit for bit;
 *   level 2: blocks with u <= 0.15 (tan theta < 0.18) take int dt/Q =
 *            theta / sqrt(D) from five terms of the series of atan(t)/t,
 *            and blocks with u <= 0.045 (tan theta < 0.05) from three
 *            (relative remainders below 3.3e-9, so results move by float
 *            rounding only; the level passes keep the three-term form).
 * Later launches on this context use forms up to `level`: 0 = the general
 * form everywhere, 1, or 2 (the default).  Any other value: WLN_EINVAL.
 */
wln_status wln_set_low_angle(wln_ctx* ctx, int32_t level);

/* -------------------------------------------------------- runtime: batches */

/*
 * A batch fixes a set of profiles and grids against one ensemble (arguments
 * as wln_wilson_avg) and keeps its work list, quadrature tables and results
 * in device memory it owns.  The paper has no counterpart: its host loop
 * launched one kernel per (rho_cm, T) point.
 * wln_batch_run enqueues one pass: the Wilson group sums, the mean and group
 * SEM of W_scal - 1 and W_ferm - 1 per point, and (when every profile's radii
 * are evenly spaced and its times geometric) the per-group effective action
 * of the spinor and the scalar loop.  use_graph != 0 records the pass into a
 * CUDA graph on the first call and replays the graph afterwards (the context
 * stream must not be the legacy default stream).  With the precision guard,
 * the batch's first run is a direct one that waits for its float pass and, if
 * the guard selected more loops than its queue holds, regrows the queue and
 * runs the float pass again (as wln_wilson_avg does); the graph is recorded
 * by the next use_graph call.  The ensemble must outlive the batch.
 * wln_batch_results copies the results out (each pointer may be NULL; host or
 * device): group_sums double[n_points][G][WLN_K]; stats double[4][n_points]
 * = mean and SEM of W_scal - 1, mean and SEM of W_ferm - 1; gamma
 * double[2][n_profiles][2] = (mean, SEM) of the spinor, then of the scalar
 * effective action (WLN_EINVAL if the grids do not allow it).
 */
typedef struct wln_batch wln_batch;
wln_status wln_batch_create(wln_ctx* ctx, const wln_ensemble* ens, const wln_profile* profiles,
                            int32_t n_profiles, const double* rho_cm, const int32_t* rho_off,
                            const double* T, const int32_t* T_off, int32_t n_groups,
                            wln_prec prec, wln_batch** out);
wln_status wln_batch_run(wln_ctx* ctx, wln_batch* batch, int32_t use_graph);
wln_status wln_batch_results(wln_ctx* ctx, const wln_batch* batch, double* group_sums,
                             double* stats, double* gamma);
/* Sizes and decomposition of a batch; any output may be NULL. */
wln_status wln_batch_info(const wln_batch* batch, int64_t* n_points, int32_t* n_tiles,
                          int32_t* points_per_lane, int32_t* chain_blocks,
                          int64_t* kernels_per_run);
wln_status wln_batch_free(wln_ctx* ctx, wln_batch* batch);

/* --------------------------------------------------------- runtime: server */

/*
 * Continuous-batching request server over one device-resident ensemble.  The
 * paper has no counterpart.  A request is one profile with its own radii and
 * proper times.  Its working memory (partial sums, results) comes from a
 * device arena of arena_bytes owned by the server; requests are admitted in
 * arrival order as arena space frees up.  Each wln_server_step launches one
 * Wilson kernel over up to tile_groups_per_step tile groups (one tile per
 * warp of a CTA: by default 8 tiles of 4 radii each), taken from the oldest
 * admitted requests first, so work of
 * several requests shares a launch; at most two steps are in flight.  When
 * all of a request's tile groups are done, its group sums, statistics and
 * effective action are computed on a second stream and copied to pinned host
 * memory.  A request's sums are accumulated in the same order whatever it
 * shares its steps with, so its results do not depend on the mix.
 * wln_server_submit fails with WLN_EINVAL if the request could never fit the
 * arena.  wln_server_poll sets *state (0 queued, 1 running, 2 finishing,
 * 3 done, 4 cancelled) and, when done, copies the results (layouts as
 * wln_batch_results, n_profiles = 1; any pointer may be NULL; host memory).
 * wln_server_release drops a done or cancelled request's host results.
 * wln_server_step waits only when two steps are already in flight.  Before a
 * step is launched, its precision-guard queue is sized for every loop its
 * points could select (64 per (point, group) whose spin can reach 2), grown
 * when a step needs more than its slot holds.  The server is not thread-safe:
 * drive it from one thread.
 */
typedef struct wln_server wln_server;
wln_status wln_server_create(wln_ctx* ctx, const wln_ensemble* ens, int32_t n_groups,
                             wln_prec prec, int64_t arena_bytes, int32_t tile_groups_per_step,
                             wln_server** out);
wln_status wln_server_submit(wln_server* server, const wln_profile* profile, const double* rho_cm,
                             int32_t n_rho, const double* T, int32_t n_T, int64_t* request_id);
wln_status wln_server_step(wln_server* server, int32_t* n_active, int32_t* n_queued);
wln_status wln_server_poll(wln_server* server, int64_t request_id, int32_t* state,
                           double* group_sums, double* stats, double* gamma);
wln_status wln_server_cancel(wln_server* server, int64_t request_id);
wln_status wln_server_release(wln_server* server, int64_t request_id);
wln_status wln_server_info(const wln_server* server, int64_t* steps, int64_t* arena_free_bytes,
                           int32_t* n_active, int32_t* n_queued);
wln_status wln_server_free(wln_server* server);

#ifdef __cplusplus
}
#endif

#endif /* WLN_H_ */
