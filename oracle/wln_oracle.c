/*
 * Plain FP64 CPU oracle for the worldline Wilson-loop path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or constant with the CUDA path; the two meet only in the
 * seeded workload descriptions (seeds, grids, field parameters).
 *
 * Everything is written for clarity, in double precision, one loop at a time,
 * in the order the paper states the steps.  OpenMP only splits independent
 * (point, loop) work between threads; each reported sum is accumulated in a
 * fixed sequential order.
 *
 * Paper: D. Mazur and J. S. Heyl, "Parallel Worldline Numerics:
 * Implementation and Error Analysis" (arXiv:1407.7486).
 *
 * Units: e = m = 1.  Profile kind 0 is the flux tube of the Sec.
 * "Verification and Validation", f(rho^2) = rho^2/(lambda^2 + rho^2), with raw
 * flux F and dimensionless flux calF = F/(2 pi) (Sec. "Cylindrical Magnetic
 * Fields").  Profile kind 1 is a constant field B (Sec. "Renormalization").
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Philox-4xW-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  One round: two widening products of the even  */
/* counter words with the round multipliers, the high halves xored with the  */
/* odd words and the key, words permuted; the key is bumped by the Weyl      */
/* constants between rounds.  The body is written once for both widths so   */
/* that checking the 64-bit instance checks the round structure of the      */
/* 32-bit one.                                                              */
/* ------------------------------------------------------------------------ */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

#define DEFINE_PHILOX4(W, UINT, MUL0, MUL1, WEYL0, WEYL1)                      \
  void wln_oracle_philox4x##W(const UINT* ctr, const UINT* key, int rounds,    \
                              UINT* out) {                                     \
    UINT c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];                    \
    UINT k0 = key[0], k1 = key[1];                                             \
    for (int r = 0; r < rounds; ++r) {                                         \
      if (r > 0) {                                                             \
        k0 += (UINT)(WEYL0);                                                   \
        k1 += (UINT)(WEYL1);                                                   \
      }                                                                        \
      UINT hi0, lo0, hi1, lo1;                                                 \
      mulhilo##W((UINT)(MUL0), c0, &hi0, &lo0);                                \
      mulhilo##W((UINT)(MUL1), c2, &hi1, &lo1);                                \
      UINT n0 = hi1 ^ c1 ^ k0;                                                 \
      UINT n1 = lo1;                                                           \
      UINT n2 = hi0 ^ c3 ^ k1;                                                 \
      UINT n3 = lo0;                                                           \
      c0 = n0; c1 = n1; c2 = n2; c3 = n3;                                      \
    }                                                                          \
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;                         \
  }

DEFINE_PHILOX4(32, uint32_t, 0xD2511F53u, 0xCD9E8D57u, 0x9E3779B9u, 0xBB67AE85u)
DEFINE_PHILOX4(64, uint64_t, 0xD2E7470EE14C6C93ull, 0xCA5A826395121157ull,
               0x9E3779B97F4A7C15ull, 0xBB67AE8584CAA73Bull)

/* The stream used for loop generation: call j of loop l uses counter
 * (j, l, 0, 0) and key (seed_lo, seed_hi).  out[l][j][0..3]. */
void wln_oracle_philox_stream(uint64_t seed, int64_t loop0, int64_t n_loops,
                              int32_t n_calls, uint32_t* out) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int64_t l = 0; l < n_loops; ++l)
    for (int32_t j = 0; j < n_calls; ++j) {
      uint32_t ctr[4] = {(uint32_t)j, (uint32_t)(loop0 + l), 0u, 0u};
      wln_oracle_philox4x32(ctr, key, 10, out + ((size_t)l * n_calls + j) * 4);
    }
}

/* ------------------------------------------------------------------------ */
/* Unit loops (Sec. "Loop Generation").  The discretised free action        */
/* (N/4) sum_k (y_{k+1}-y_k)^2 makes each increment component Gaussian with */
/* variance 2/N; closing the loop conditions the increments on summing to   */
/* zero, which for i.i.d. Gaussians is subtracting their mean; the points   */
/* are the partial sums, and the common centre of mass is then removed      */
/* (d-loop step 5).                                                         */
/* ------------------------------------------------------------------------ */

/* u in (0,1): the midpoint of the k-th of 2^32 equal cells. */
static double uniform_open(uint32_t k) { return ((double)k + 0.5) * 0x1p-32; }

/* Box-Muller: two independent N(0,1) from two uniforms. */
static void box_muller(double ua, double ub, double* z0, double* z1) {
  double radius = sqrt(-2.0 * log(ua));
  double angle = 2.0 * M_PI * ub;
  *z0 = radius * cos(angle);
  *z1 = radius * sin(angle);
}

/* Increments before closure: xi[c][k], c = 0 (x), 1 (y).  Philox call j
 * gives (u0,u1) -> (xi_x[2j], xi_y[2j]) and (u2,u3) -> (xi_x[2j+1],
 * xi_y[2j+1]). */
void wln_oracle_raw_increments(uint64_t seed, int64_t loop, int32_t N, double* xi) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  double scale = sqrt(2.0 / (double)N);
  for (int32_t j = 0; j < N / 2; ++j) {
    uint32_t ctr[4] = {(uint32_t)j, (uint32_t)loop, 0u, 0u}, u[4];
    wln_oracle_philox4x32(ctr, key, 10, u);
    double z0, z1, z2, z3;
    box_muller(uniform_open(u[0]), uniform_open(u[1]), &z0, &z1);
    box_muller(uniform_open(u[2]), uniform_open(u[3]), &z2, &z3);
    xi[0 * N + 2 * j] = scale * z0;
    xi[1 * N + 2 * j] = scale * z1;
    xi[0 * N + 2 * j + 1] = scale * z2;
    xi[1 * N + 2 * j + 1] = scale * z3;
  }
}

/* One CM-centred unit loop: y[c][k], k = 0..N-1. */
void wln_oracle_unit_loop(uint64_t seed, int64_t loop, int32_t N, double* y) {
  double* xi = (double*)malloc(sizeof(double) * 2 * (size_t)N);
  wln_oracle_raw_increments(seed, loop, N, xi);
  for (int c = 0; c < 2; ++c) {
    double* e = xi + (size_t)c * N;
    double* p = y + (size_t)c * N;
    double mean_e = 0.0;
    for (int32_t k = 0; k < N; ++k) mean_e += e[k];
    mean_e /= (double)N;
    for (int32_t k = 0; k < N; ++k) e[k] -= mean_e;      /* closure */
    p[0] = 0.0;
    for (int32_t k = 1; k < N; ++k) p[k] = p[k - 1] + e[k - 1];  /* positions */
    double cm = 0.0;
    for (int32_t k = 0; k < N; ++k) cm += p[k];
    cm /= (double)N;
    for (int32_t k = 0; k < N; ++k) p[k] -= cm;           /* centre of mass */
  }
  free(xi);
}

/* Loops loop0 .. loop0+n_loops-1 into y[l][c][k]. */
void wln_oracle_gen_loops(uint64_t seed, int64_t loop0, int64_t n_loops, int32_t N,
                          double* y, int32_t threads) {
#pragma omp parallel for schedule(static) num_threads(threads > 0 ? threads : 1)
  for (int64_t l = 0; l < n_loops; ++l)
    wln_oracle_unit_loop(seed, loop0 + l, N, y + (size_t)l * 2 * N);
}

/* ------------------------------------------------------------------------ */
/* d-loops (Sec. "Loop Generation", Eqs. yn2 and ynk).  Start from one point  */
/* y_N (taken as the origin; index N is index 0 of the closed loop).  Level 1 */
/* adds y_{N/2}, Gaussian about y_N with variance 1/N_1 = 1/2 per component.  */
/* Level k (N_k = 2^k) adds the points q N/N_k, q = 1, 3, ..., N_k - 1, each  */
/* Gaussian about the mean of its two neighbours of the previous level with   */
/* variance 1/N_k.  The last level has N_k = N; then the centre of mass is    */
/* removed (step 5).                                                           */
/* Gaussian number m (m = 0 for level 1; level k uses m = 2^(k-1) - 1 +       */
/* (q-1)/2) comes from Philox call j = m/2 with counter (j, loop, 1, 0):      */
/* (u0,u1) give the x and y of even m, (u2,u3) those of odd m (Box-Muller).   */
/* ------------------------------------------------------------------------ */
static void dloop_gaussian(uint64_t seed, int64_t loop, int32_t m, double* gx, double* gy) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {(uint32_t)(m / 2), (uint32_t)loop, 1u, 0u}, u[4];
  wln_oracle_philox4x32(ctr, key, 10, u);
  if (m % 2 == 0) box_muller(uniform_open(u[0]), uniform_open(u[1]), gx, gy);
  else box_muller(uniform_open(u[2]), uniform_open(u[3]), gx, gy);
}

void wln_oracle_dloop(uint64_t seed, int64_t loop, int32_t N, double* y) {
  double* yx = y;
  double* yy = y + N;
  yx[0] = 0.0;
  yy[0] = 0.0;
  int32_t m = 0;
  for (int32_t Nk = 2; Nk <= N; Nk *= 2) {
    const int32_t stride = N / Nk;          /* index distance between neighbours at this level */
    const double sigma = sqrt(1.0 / (double)Nk);
    for (int32_t q = 1; q < Nk; q += 2) {
      const int32_t i = q * stride;
      const int32_t left = (q - 1) * stride, right = ((q + 1) * stride) % N;
      double gx, gy;
      dloop_gaussian(seed, loop, m++, &gx, &gy);
      yx[i] = 0.5 * (yx[left] + yx[right]) + sigma * gx;
      yy[i] = 0.5 * (yy[left] + yy[right]) + sigma * gy;
    }
  }
  for (int c = 0; c < 2; ++c) {
    double* p = y + (size_t)c * N;
    double cm = 0.0;
    for (int32_t k = 0; k < N; ++k) cm += p[k];
    cm /= (double)N;
    for (int32_t k = 0; k < N; ++k) p[k] -= cm;
  }
}

void wln_oracle_gen_dloops(uint64_t seed, int64_t loop0, int64_t n_loops, int32_t N,
                           double* y, int32_t threads) {
#pragma omp parallel for schedule(static) num_threads(threads > 0 ? threads : 1)
  for (int64_t l = 0; l < n_loops; ++l)
    wln_oracle_dloop(seed, loop0 + l, N, y + (size_t)l * 2 * N);
}

/* ------------------------------------------------------------------------ */
/* Wilson loop of one discretised loop at one (rho_cm, T).                  */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t kind;      /* 0 flux tube, 1 constant field */
  int32_t reserved;
  double F;          /* raw flux of the tube */
  double lambda;     /* tube radius */
  double B;          /* constant field strength */
} oracle_profile;

/*
 * Phase e * (closed line integral of A) and spin integral e * int_0^T B dtau
 * along the polygon r_k = x_cm + sqrt(T) y_k, k = 0..N-1, joined by straight
 * segments r_k -> r_{k+1 mod N}, each traversed in proper time T/N.
 *
 * Flux tube (Sec. "Wilson Loop", Eqs. rhoi-Ci; Sec. "Fermion Part", Eq.
 * Wfermfpl with the loop-sum form that follows it): on segment k,
 *   rho^2(t) = A + 2 B t + C t^2,
 *   e int A.dr = calF (x^k y^{k+1} - y^k x^{k+1}) int_0^1 dt f/rho^2,
 *   with f/rho^2 = 1/(lambda^2 + rho^2) for this profile, and
 *   e B(rho^2) = 2 calF f'(rho^2) = 2 calF lambda^2/(lambda^2 + rho^2)^2,
 *   so e int B dtau over the segment is (T/N) 2 calF lambda^2 int_0^1 dt/Q^2,
 *   Q(t) = lambda^2 + rho^2(t).  Both integrals are done in closed form, which
 * keeps gauge invariance exact (the paper's remark after Eq. Ci).
 *
 * Constant field: A = (B/2)(-y, x), whose line integral over straight
 * segments is B times the shoelace area; e int B dtau = B T.
 */
void wln_oracle_loop_phase_spin(const double* y, int32_t N, const oracle_profile* prof,
                                double rho_cm, double T, double* phase, double* spin) {
  const double* yx = y;
  const double* yy = y + N;
  const double sqT = sqrt(T);
  if (prof->kind == 1) {
    double twice_area = 0.0;
    for (int32_t k = 0; k < N; ++k) {
      int32_t k1 = (k + 1) % N;
      double x0 = rho_cm + sqT * yx[k], y0 = sqT * yy[k];
      double x1 = rho_cm + sqT * yx[k1], y1 = sqT * yy[k1];
      twice_area += x0 * y1 - y0 * x1;
    }
    *phase = prof->B * 0.5 * twice_area;
    *spin = prof->B * T;
    return;
  }
  const double calF = prof->F / (2.0 * M_PI);
  const double l2 = prof->lambda * prof->lambda;
  double ph = 0.0, sp = 0.0;
  for (int32_t k = 0; k < N; ++k) {
    int32_t k1 = (k + 1) % N;
    double x0 = rho_cm + sqT * yx[k], y0 = sqT * yy[k];
    double x1 = rho_cm + sqT * yx[k1], y1 = sqT * yy[k1];
    double dx = x1 - x0, dy = y1 - y0;
    double A = x0 * x0 + y0 * y0;
    double B = x0 * dx + y0 * dy;
    double C = dx * dx + dy * dy;
    double X = x0 * y1 - y0 * x1;
    if (C == 0.0) {
      /* A stationary step adds no phase, but the particle still spends proper
       * time T/N at that point, so the spin integral gains e B(rho^2) T/N. */
      double Q0s = l2 + A;
      sp += (T / (double)N) * 2.0 * calF * l2 / (Q0s * Q0s);
      continue;
    }
    /* Q(t) = C t^2 + 2 B t + (lambda^2 + A); its discriminant
     * C (lambda^2 + A) - B^2 equals lambda^2 C + X^2 (Lagrange identity
     * A C - B^2 = X^2), which is > 0 for lambda > 0. */
    double D = l2 * C + X * X;
    double sD = sqrt(D);
    /* int_0^1 dt/Q = [atan((C t + B)/sqrt D)]_0^1 / sqrt D; the difference
     * of the two arctangents is taken as one atan2, in (0, pi). */
    double theta = atan2(C * sD, D + B * (B + C));
    double J1 = theta / sD;
    /* int_0^1 dt/Q^2 = [ (C t + B)/Q ]_0^1 / (2D) + C J1 / (2D). */
    double Q0 = l2 + A;
    double Q1 = l2 + x1 * x1 + y1 * y1;
    double J2 = ((C + B) / Q1 - B / Q0 + C * J1) / (2.0 * D);
    ph += calF * X * J1;
    sp += (T / (double)N) * 2.0 * calF * l2 * J2;
  }
  *phase = ph;
  *spin = sp;
}

/* Sum over segments of |phase of the segment|: the condition number of the
 * phase sum (how much rounding in the terms can move the total).  Same
 * closed forms as wln_oracle_loop_phase_spin; flux tube only (the constant
 * field returns |B| times the sum of |shoelace terms| / 2). */
double wln_oracle_loop_phase_abs(const double* y, int32_t N, const oracle_profile* prof,
                                 double rho_cm, double T) {
  const double* yx = y;
  const double* yy = y + N;
  const double sqT = sqrt(T);
  const double calF = prof->F / (2.0 * M_PI);
  const double l2 = prof->lambda * prof->lambda;
  double acc = 0.0;
  for (int32_t k = 0; k < N; ++k) {
    int32_t k1 = (k + 1) % N;
    double x0 = rho_cm + sqT * yx[k], y0 = sqT * yy[k];
    double x1 = rho_cm + sqT * yx[k1], y1 = sqT * yy[k1];
    double X = x0 * y1 - y0 * x1;
    if (prof->kind == 1) {
      acc += fabs(prof->B * 0.5 * X);
      continue;
    }
    double dx = x1 - x0, dy = y1 - y0;
    double B = x0 * dx + y0 * dy, C = dx * dx + dy * dy;
    if (C == 0.0) continue;
    double D = l2 * C + X * X, sD = sqrt(D);
    acc += fabs(calF * X * atan2(C * sD, D + B * (B + C)) / sD);
  }
  return acc;
}

void wln_oracle_phase_abs_many(const double* y, int64_t n_loops, int32_t N,
                               const oracle_profile* prof, double rho_cm, double T,
                               double* out, int32_t threads) {
#pragma omp parallel for schedule(static) num_threads(threads > 0 ? threads : 1)
  for (int64_t l = 0; l < n_loops; ++l)
    out[l] = wln_oracle_loop_phase_abs(y + (size_t)l * 2 * N, N, prof, rho_cm, T);
}

/* Per-loop phase and spin for loops y[l][2][N] at one point. */
void wln_oracle_phase_spin_many(const double* y, int64_t n_loops, int32_t N,
                                const oracle_profile* prof, double rho_cm, double T,
                                double* phase, double* spin, int32_t threads) {
#pragma omp parallel for schedule(static) num_threads(threads > 0 ? threads : 1)
  for (int64_t l = 0; l < n_loops; ++l)
    wln_oracle_loop_phase_spin(y + (size_t)l * 2 * N, N, prof, rho_cm, T, phase + l, spin + l);
}

/* ------------------------------------------------------------------------ */
/* Group sums (Sec. "Grouping Worldlines"): group g holds loops              */
/* g n/G .. (g+1) n/G - 1.  For each point and group five sums:             */
/*   0: sum (W_scal - 1),  W_scal = cos(phase)                              */
/*   1: sum (W_ferm - 1),  W_ferm = cos(phase) cosh(spin)                   */
/*   2: sum sin(phase)     (imaginary part; zero on average)                */
/*   3: sum (W_scal - 1)^2                                                  */
/*   4: sum (W_ferm - 1)^2                                                  */
/* W - 1 uses the half-angle forms cos p - 1 = -2 sin^2(p/2) and            */
/* cosh s - 1 = 2 sinh^2(s/2), which are exact identities.                  */
/* Point p = (profile q, T index b, rho index a) is stored at               */
/* out[((p_index) * G + g) * 5 + c] with p_index = b * n_rho + a.           */
/* ------------------------------------------------------------------------ */
void wln_oracle_wilson_terms(double phase, double spin, double* w) {
  double h = sin(0.5 * phase);
  double scal_m1 = -2.0 * h * h;
  double sh = sinh(0.5 * spin);
  double ferm_m1 = cos(phase) * 2.0 * sh * sh + scal_m1;
  w[0] = scal_m1;
  w[1] = ferm_m1;
  w[2] = sin(phase);
  w[3] = scal_m1 * scal_m1;
  w[4] = ferm_m1 * ferm_m1;
}

void wln_oracle_group_sums(const double* y, int64_t n_loops, int32_t N,
                           const oracle_profile* prof, const double* rho, int32_t n_rho,
                           const double* T, int32_t n_T, int32_t G, double* out,
                           int32_t threads) {
  const int64_t per_group = n_loops / G;
  const int64_t n_pts = (int64_t)n_rho * n_T;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : 1)
  for (int64_t pg = 0; pg < n_pts * G; ++pg) {
    int64_t p = pg / G, g = pg % G;
    double rho_cm = rho[p % n_rho], Tp = T[p / n_rho];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int64_t l = g * per_group; l < (g + 1) * per_group; ++l) {
      double ph, sp, w[5];
      wln_oracle_loop_phase_spin(y + (size_t)l * 2 * N, N, prof, rho_cm, Tp, &ph, &sp);
      wln_oracle_wilson_terms(ph, sp, w);
      for (int c = 0; c < 5; ++c) acc[c] += w[c];
    }
    for (int c = 0; c < 5; ++c) out[(size_t)pg * 5 + c] = acc[c];
  }
}

int32_t wln_oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Per-loop values and randomised groups (Sec. "Correlations between Wilson  */
/* Loops" and Sec. "Grouping Worldlines": assign the worldlines to groups    */
/* at random, anew for every evaluation of the integrand).                  */
/* ------------------------------------------------------------------------ */

/* W - 1 of every loop at every point: out[p][l][0] scalar, [1] spinor,
 * points p = iT * n_rho + i_rho. */
void wln_oracle_loop_values(const double* y, int64_t n_loops, int32_t N,
                            const oracle_profile* prof, const double* rho, int32_t n_rho,
                            const double* T, int32_t n_T, double* out, int32_t threads) {
  const int64_t n_pts = (int64_t)n_rho * n_T;
#pragma omp parallel for schedule(dynamic, 16) num_threads(threads > 0 ? threads : 1)
  for (int64_t pl = 0; pl < n_pts * n_loops; ++pl) {
    int64_t p = pl / n_loops, l = pl % n_loops;
    double ph, sp, w[5];
    wln_oracle_loop_phase_spin(y + (size_t)l * 2 * N, N, prof, rho[p % n_rho], T[p / n_rho],
                               &ph, &sp);
    wln_oracle_wilson_terms(ph, sp, w);
    out[(size_t)pl * 2] = w[0];
    out[(size_t)pl * 2 + 1] = w[1];
  }
}

/* The random grouping of evaluation `point`: a uniformly random permutation
 * a[0..n-1] of the loops by the Fisher-Yates shuffle (Durstenfeld's form):
 * for t = 0 .. n-2, i = n-1-t, draw j uniform in [0, i] and swap a[i], a[j].
 * Draw t takes 32-bit word t mod 4 of Philox-4x32-10 with counter
 * (t / 4, point, 2, 0) and key (seed_lo, seed_hi), and j = (u (i+1)) >> 32
 * (the multiply-shift map, bias below (i+1)/2^32).  Group g then holds
 * loops a[g n/G .. (g+1) n/G - 1]. */
void wln_oracle_shuffle(uint64_t seed, int64_t point, int32_t n, int32_t* a) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t u[4] = {0, 0, 0, 0};
  for (int32_t k = 0; k < n; ++k) a[k] = k;
  for (int32_t t = 0; t < n - 1; ++t) {
    if (t % 4 == 0) {
      uint32_t ctr[4] = {(uint32_t)(t / 4), (uint32_t)point, 2u, 0u};
      wln_oracle_philox4x32(ctr, key, 10, u);
    }
    int32_t i = n - 1 - t;
    int32_t j = (int32_t)(((uint64_t)u[t % 4] * (uint64_t)(i + 1)) >> 32);
    int32_t s = a[i];
    a[i] = a[j];
    a[j] = s;
  }
}
