// Group statistics and effective-action quadrature on the device, in double
// precision (paper Sec. "Grouping Worldlines"; Eq. cylEA; Sec. "Computing an
// Effective Action").  Every sum runs in a fixed order, so results do not
// depend on scheduling.
#include <math_constants.h>

#include "wln_internal.cuh"

namespace wln {
namespace {

constexpr int kComps = WLN_K;

// Group means m_g = S_g / loops_per_group, their mean, the group standard
// error and the delete-one-group jackknife variance; the deviations
// m_g - mean go to dev[g][p] for the covariance.
__global__ void jackknife_kernel(const double* S, int32_t n_points, int32_t G, int32_t lpg,
                                 int32_t comp, double* mean, double* sem, double* jk_var,
                                 double* dev) {
  const int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (p >= n_points) return;
  const double* s = S + p * G * kComps + comp;
  const double inv = 1.0 / lpg;
  double m = 0.0;
  for (int g = 0; g < G; ++g) m += s[g * kComps] * inv;
  m /= G;
  double ss = 0.0, jj = 0.0;
  for (int g = 0; g < G; ++g) {
    const double mg = s[g * kComps] * inv;
    const double d = mg - m;
    ss += d * d;
    const double loo = (G * m - mg) / (G - 1);
    jj += (loo - m) * (loo - m);
    if (dev) dev[static_cast<int64_t>(g) * n_points + p] = d;
  }
  mean[p] = m;
  sem[p] = sqrt(ss / (static_cast<double>(G) * (G - 1)));
  if (jk_var) jk_var[p] = (G - 1.0) / G * jj;
}

// Extrapolation to infinitely many points per loop (Sec. "Estimating the
// Discretization Uncertainties"): the parabola in 1/N through the level
// means at N, N/2, N/4, at 1/N = 0, weights 8/3, -2, 1/3.  One thread per
// (point, scalar|spinor); out[p][x][6] = (m_N, m_N/2, m_N/4, W_inf - 1,
// its group standard error, |m_N - (W_inf - 1)|).
__global__ void extrapolate_kernel(const double* S, int32_t n_points, int32_t G, int32_t lpg,
                                   double* out) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= 2 * static_cast<int64_t>(n_points)) return;
  const int64_t p = i >> 1;
  const int x = static_cast<int>(i & 1);
  const double* s = S + p * G * WLN_KL + x;
  const double inv = 1.0 / lpg;
  double m[3] = {0.0, 0.0, 0.0}, e = 0.0;
  for (int g = 0; g < G; ++g) {
    const double* sg = s + g * WLN_KL;
    const double a = sg[0] * inv, b = sg[2] * inv, c = sg[4] * inv;
    m[0] += a; m[1] += b; m[2] += c;
    e += (8.0 / 3.0) * a - 2.0 * b + (1.0 / 3.0) * c;
  }
  for (int j = 0; j < 3; ++j) m[j] /= G;
  e /= G;
  double ss = 0.0;
  for (int g = 0; g < G; ++g) {
    const double* sg = s + g * WLN_KL;
    const double eg = (8.0 / 3.0) * (sg[0] * inv) - 2.0 * (sg[2] * inv) + (1.0 / 3.0) * (sg[4] * inv);
    ss += (eg - e) * (eg - e);
  }
  double* o = out + i * 6;
  o[0] = m[0]; o[1] = m[1]; o[2] = m[2];
  o[3] = e;
  o[4] = sqrt(ss / (static_cast<double>(G) * (G - 1)));
  o[5] = fabs(m[0] - e);
}

// cov[p][q] = sum_g dev[g][p] dev[g][q] / (G (G - 1)).  64x64 tiles, only
// tiles on or above the diagonal are computed; the mirror image is written
// through a shared-memory transpose so both stores are coalesced.  Packed:
// only q >= p, row p at p n - p (p - 1) / 2 (the upper triangle row by row).
constexpr int kTile = 64, kKc = 16;
__device__ __forceinline__ int64_t packed_index(int64_t p, int64_t q, int64_t n) {
  return p * n - p * (p - 1) / 2 + (q - p);
}
__global__ void __launch_bounds__(256) covariance_kernel(const double* dev, int32_t n_points,
                                                         int32_t G, double* cov, int packed) {
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (ti > tj) return;
  __shared__ double a[kKc][kTile], b[kKc][kTile];
  __shared__ double tr[kTile][kTile + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int g0 = 0; g0 < G; g0 += kKc) {
    for (int i = threadIdx.x; i < kKc * kTile; i += 256) {
      const int gg = g0 + i / kTile, c = i % kTile;
      const int pa = ti * kTile + c, pb = tj * kTile + c;
      a[i / kTile][c] = (gg < G && pa < n_points) ? dev[static_cast<int64_t>(gg) * n_points + pa] : 0.0;
      b[i / kTile][c] = (gg < G && pb < n_points) ? dev[static_cast<int64_t>(gg) * n_points + pb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kKc; ++kk) {
      double ra[4], rb[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) ra[r] = a[kk][ty * 4 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) rb[c] = b[kk][tx * 4 + c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(ra[r], rb[c], acc[r][c]);
    }
    __syncthreads();
  }
  const double scale = 1.0 / (static_cast<double>(G) * (G - 1));
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int p = ti * kTile + ty * 4 + r;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int q = tj * kTile + tx * 4 + c;
      acc[r][c] *= scale;
      if (packed) {
        if (q >= p && q < n_points) cov[packed_index(p, q, n_points)] = acc[r][c];
      } else {
        if (p < n_points && q < n_points) cov[static_cast<int64_t>(p) * n_points + q] = acc[r][c];
        tr[ty * 4 + r][tx * 4 + c] = acc[r][c];
      }
    }
  }
  if (packed || ti == tj) return;
  __syncthreads();
  for (int i = threadIdx.x; i < kTile * kTile; i += 256) {
    const int row = i / kTile, col = i % kTile;  // output row in tile tj, column in tile ti
    const int p = tj * kTile + row, q = ti * kTile + col;
    if (p < n_points && q < n_points) cov[static_cast<int64_t>(p) * n_points + q] = tr[col][row];
  }
}

__global__ void loop_sem_kernel(const double* S, int32_t n_points, int32_t G, int32_t n_loops,
                                int32_t cs, int32_t cq, double* out) {
  const int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (p >= n_points) return;
  double s1 = 0.0, s2 = 0.0;
  for (int g = 0; g < G; ++g) {
    s1 += S[(p * G + g) * kComps + cs];
    s2 += S[(p * G + g) * kComps + cq];
  }
  const double ss = s2 - s1 * s1 / n_loops;
  out[p] = sqrt((ss > 0.0 ? ss : 0.0) / (static_cast<double>(n_loops) * (n_loops - 1)));
}

// Composite Simpson weight of point j of n evenly spaced points (spacing h);
// an even n ends with a 3/8 panel over the last three intervals.
__device__ double simpson_weight(int j, int n, double h) {
  if (n == 1) return 0.0;
  if (n == 2) return 0.5 * h;
  const int m = (n & 1) ? n : n - 3;
  double w = 0.0;
  if (m >= 3 && j < m) w += (j == 0 || j == m - 1) ? h / 3.0 : ((j & 1) ? 4.0 * h / 3.0 : 2.0 * h / 3.0);
  if (!(n & 1) && j >= n - 4) {
    const int t = j - (n - 4);
    w += 3.0 * h / 8.0 * ((t == 0 || t == 3) ? 1.0 : 3.0);
  }
  return w;
}

// One CTA per (profile, group): Gamma_g = (1/4 pi) sum_ab w_a rho_a w_b T_b
// e^{-T_b}/T_b^3 (m_g(a, b) - c (eB(rho_a) T_b)^2), m_g the group mean of W - 1.
__global__ void __launch_bounds__(256) effective_action_kernel(
    const QuadProfile* qp, const double* rho, const double* T, const double* S, int32_t G,
    int32_t lpg, int32_t spinor, double* gamma_groups) {
  const int q = blockIdx.y, g = blockIdx.x;
  const QuadProfile pr = qp[q];
  const int comp = spinor ? WLN_C_FERM : WLN_C_SCAL;
  const double c_ct = spinor ? 1.0 / 3.0 : -1.0 / 6.0;
  const int n = pr.n_rho * pr.n_T;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int it = i / pr.n_rho, ir = i % pr.n_rho;
    const double r = rho[pr.rho_base + ir], t = T[pr.T_base + it];
    const double wr = simpson_weight(ir, pr.n_rho, pr.h_rho) * r;
    const double wt = simpson_weight(it, pr.n_T, pr.h_u) * t;
    double eB;
    if (pr.kind == WLN_PROFILE_CONST_B) {
      eB = pr.eB_scale;
    } else {
      const double q2 = pr.l2 + r * r;
      eB = pr.eB_scale / (q2 * q2);
    }
    const double m = S[((pr.p0 + i) * G + g) * kComps + comp] / lpg;
    const double et = eB * t;
    acc += wr * wt * exp(-t) / (t * t * t) * (m - c_ct * et * et);
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) gamma_groups[q * G + g] = red[0] / (4.0 * 3.14159265358979323846);
}

// ------------------------------------------------ full effective action
// Small-argument series of the constant-field brackets (coefficients of
// x^4, x^6, ..., x^26; gen_lcf_series.py, exact Bernoulli numbers):
//   x coth x - 1 - x^2/3 (spinor),  x / sinh x - 1 + x^2/6 (scalar).
__constant__ double kLcfSpin[12] = {
    -0.022222222222222223, 0.0021164021164021165, -0.00021164021164021165,
    2.1377799155576935e-05, -2.1644042808063972e-06, 2.1925947851873778e-07,
    -2.2214608789979678e-08, 2.2507846516808994e-09, -2.2805151204592183e-10,
    2.3106432599002624e-11, -2.3411706819824882e-12, 2.3721017400233653e-13};
__constant__ double kLcfScal[12] = {
    0.019444444444444445, -0.00205026455026455, 0.0002099867724867725,
    -2.1336045641601196e-05, 2.1633474427786596e-06, -2.192327134456764e-07,
    2.2213930853920414e-08, -2.2507674795567867e-09, 2.280510770721821e-10,
    -2.3106421580996967e-11, 2.3411704028931947e-12, -2.3721016693292245e-13};

// The LCF bracket at x = eB T (Eq. LCFferm and its scalar counterpart): the
// series below |x| = 1/2, where the closed form cancels to ~x^4.
__device__ double lcf_bracket(double x, bool spinor) {
  x = fabs(x);
  if (x < 0.5) {
    const double* c = spinor ? kLcfSpin : kLcfScal;
    const double x2 = x * x;
    double p = c[11];
    for (int k = 10; k >= 0; --k) p = fma(p, x2, c[k]);
    return p * x2 * x2;
  }
  return spinor ? x / tanh(x) - 1.0 - x * x / 3.0 : x / sinh(x) - 1.0 + x * x / 6.0;
}

// int_0^a of the small-T expansion of the integrand, term by term (Eq. fermI
// for the spinor loop, Eq. scalI for the scalar loop, m = 1).
__device__ double small_T_part(double eB, double a, bool spinor) {
  const double b2 = eB * eB, b4 = b2 * b2, b6 = b4 * b2;
  double c0, c1, c2, c3;   // coefficients of T, T^2, T^3, T^4
  if (spinor) {
    c0 = -b4 / 45.0; c1 = b4 / 45.0; c2 = 2.0 * b6 / 945.0 - b4 / 90.0;
    c3 = (7.0 * b4 - 4.0 * b6) / 1890.0;
  } else {
    c0 = 7.0 * b4 / 360.0; c1 = -7.0 * b4 / 360.0; c2 = (147.0 * b4 - 31.0 * b6) / 15120.0;
    c3 = (31.0 * b6 - 49.0 * b4) / 15120.0;
  }
  const double a2 = a * a;
  return a2 * (c0 / 2.0 + a * (c1 / 3.0 + a * (c2 / 4.0 + a * (c3 / 5.0))));
}

__device__ double profile_eB(const QuadProfile& pr, double r) {
  if (pr.kind == WLN_PROFILE_CONST_B) return pr.eB_scale;
  const double q2 = pr.l2 + r * r;
  return pr.eB_scale / (q2 * q2);
}

// Weight of node i of a mapped axis of n nodes: Simpson in x over the n + 1
// points 0, x0/n, .., x0 (node i sits at x = x0 (n - i)/n), times scale/x^2.
__device__ double mapped_weight(int i, int n, double x0, double scale) {
  const int k = n - i;
  const double x = x0 * k / n;
  return simpson_weight(k, n + 1, x0 / n) * scale / (x * x);
}

__device__ double T_weight(const QuadProfile& pr, int j, double t) {
  return pr.T_kind == WLN_GRID_MAPPED ? mapped_weight(j, pr.n_T, pr.T_x0, pr.T_scale)
                                      : simpson_weight(j, pr.n_T, pr.h_u) * t;
}

__device__ double rho_weight(const QuadProfile& pr, int i) {
  return pr.rho_kind == WLN_GRID_MAPPED ? mapped_weight(i, pr.n_rho, pr.rho_x0, pr.rho_scale)
                                        : simpson_weight(i, pr.n_rho, pr.h_rho);
}

// One thread per (radius of profile q, group g) and one more "group" g = G
// for the LCF: D(rho_i) = small-T part + sum_j w_j I(rho_i, T_j), in T order.
__global__ void density_kernel(const QuadProfile* qp, const double* rho, const double* T,
                               const double* S, int32_t G, int32_t lpg, int32_t spinor,
                               double* d_groups, double* density) {
  const int q = blockIdx.y;
  const QuadProfile pr = qp[q];
  const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (idx >= static_cast<int64_t>(pr.n_rho) * (G + 1)) return;
  const int i = static_cast<int>(idx / (G + 1)), g = static_cast<int>(idx % (G + 1));
  const bool sp = spinor != 0;
  const int comp = sp ? WLN_C_FERM : WLN_C_SCAL;
  const double c_ct = sp ? 1.0 / 3.0 : -1.0 / 6.0;
  const double r = rho[pr.rho_base + i];
  const double eB = profile_eB(pr, r);
  double acc = pr.small_T ? small_T_part(eB, T[pr.T_base], sp) : 0.0;
  for (int j = 0; j < pr.n_T; ++j) {
    const double t = T[pr.T_base + j];
    const double et = eB * t;
    const double pref = exp(-t) / (t * t * t);
    double b;
    if (g < G) {
      const int64_t p = pr.p0 + static_cast<int64_t>(j) * pr.n_rho + i;
      b = S[(p * G + g) * kComps + comp] / lpg - c_ct * et * et;
    } else {
      b = lcf_bracket(et, sp);
    }
    acc += T_weight(pr, j, t) * pref * b;
  }
  const int64_t ri = pr.rho_base + i;
  if (g < G) d_groups[ri * G + g] = acc;
  else density[ri * 3 + 2] = acc;
}

// One CTA per (group, profile); group index G is the LCF.  Gamma = (1/4 pi)
// sum_i w_i rho_i D(rho_i), each thread over a fixed stride of radii, then a
// fixed tree.
__global__ void __launch_bounds__(256) action_kernel(const QuadProfile* qp, const double* rho,
                                                     int32_t G, const double* d_groups,
                                                     const double* density,
                                                     double* gamma_groups, double* gamma) {
  const int q = blockIdx.y, g = blockIdx.x;
  const QuadProfile pr = qp[q];
  double acc = 0.0;
  for (int i = threadIdx.x; i < pr.n_rho; i += blockDim.x) {
    const int64_t ri = pr.rho_base + i;
    const double D = g < G ? d_groups[ri * G + g] : density[ri * 3 + 2];
    acc += rho_weight(pr, i) * rho[ri] * D;
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double v = red[0] / (4.0 * 3.14159265358979323846);
    if (g < G) gamma_groups[q * G + g] = v;
    else gamma[q * 3 + 2] = v;
  }
}

// Mean over groups and its standard error of rows x[r][G], into out[r * stride + 0, 1].
__global__ void mean_sem_rows_kernel(const double* x, int32_t n_rows, int32_t G, double* out,
                                     int32_t stride) {
  const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (r >= n_rows) return;
  const double* v = x + r * G;
  double m = 0.0;
  for (int g = 0; g < G; ++g) m += v[g];
  m /= G;
  double ss = 0.0;
  for (int g = 0; g < G; ++g) ss += (v[g] - m) * (v[g] - m);
  out[r * stride] = m;
  out[r * stride + 1] = sqrt(ss / (static_cast<double>(G) * (G - 1)));
}

// The integrand at every point: mean and standard error over groups of
// I_g = e^{-T}/T^3 (m_g - c (eB T)^2), and the LCF integrand.
__global__ void integrand_kernel(const QuadProfile* qp, const int32_t* point_profile,
                                 const double* rho, const double* T, const double* S,
                                 int64_t n_points, int32_t G, int32_t lpg, int32_t spinor,
                                 double* out) {
  const int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (p >= n_points) return;
  const QuadProfile pr = qp[point_profile[p]];
  const int64_t local = p - pr.p0;
  const int j = static_cast<int>(local / pr.n_rho), i = static_cast<int>(local % pr.n_rho);
  const bool sp = spinor != 0;
  const int comp = sp ? WLN_C_FERM : WLN_C_SCAL;
  const double c_ct = sp ? 1.0 / 3.0 : -1.0 / 6.0;
  const double t = T[pr.T_base + j];
  const double et = profile_eB(pr, rho[pr.rho_base + i]) * t;
  const double pref = exp(-t) / (t * t * t);
  const double ct = c_ct * et * et;
  const double* s = S + p * G * kComps + comp;
  double m = 0.0;
  for (int g = 0; g < G; ++g) m += pref * (s[g * kComps] / lpg - ct);
  m /= G;
  double ss = 0.0;
  for (int g = 0; g < G; ++g) {
    const double d = pref * (s[g * kComps] / lpg - ct) - m;
    ss += d * d;
  }
  out[p * 3] = m;
  out[p * 3 + 1] = sqrt(ss / (static_cast<double>(G) * (G - 1)));
  out[p * 3 + 2] = pref * lcf_bracket(et, sp);
}

// ------------------------------------- randomised groups and correlations
// Fisher-Yates shuffle of the loops of every evaluation (one thread per
// point): for t = 0 .. n-2, i = n-1-t, j = (u (i + 1)) >> 32 with u word
// t mod 4 of Philox-4x32-10 at counter (t/4, point, 2, 0), swap a[i], a[j].
__global__ void shuffle_kernel(int64_t n_points, int32_t n, uint32_t k0, uint32_t k1,
                               int32_t* perm) {
  const int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (p >= n_points) return;
  int32_t* a = perm + p * n;
  for (int32_t k = 0; k < n; ++k) a[k] = k;
  uint4 u = make_uint4(0u, 0u, 0u, 0u);
  for (int32_t t = 0; t < n - 1; ++t) {
    if ((t & 3) == 0)
      u = philox4x32_10(make_uint4(static_cast<uint32_t>(t >> 2), static_cast<uint32_t>(p), 2u, 0u),
                        k0, k1);
    const uint32_t w = (t & 3) == 0 ? u.x : (t & 3) == 1 ? u.y : (t & 3) == 2 ? u.z : u.w;
    const int32_t i = n - 1 - t;
    const int32_t j = static_cast<int32_t>((static_cast<uint64_t>(w) * static_cast<uint64_t>(i + 1)) >> 32);
    const int32_t x = a[i];
    a[i] = a[j];
    a[j] = x;
  }
}

// Group sums of per-loop values W[p][l] = (W_scal - 1, W_ferm - 1): group g
// of point p holds the loops at positions g n/G .. (g+1) n/G - 1 of the
// point's order (perm, or the generation order), summed in that order.
// Layout [p][g][WLN_K]; the imaginary part is not kept per loop: NaN.
__global__ void group_sums_loops_kernel(const double2* W, int64_t n_points, int32_t n, int32_t G,
                                        const int32_t* perm, double* S) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n_points * G) return;
  const int64_t p = i / G;
  const int g = static_cast<int>(i % G);
  const int lpg = n / G;
  const double2* w = W + p * n;
  const int32_t* a = perm ? perm + p * n : nullptr;
  double s0 = 0.0, s1 = 0.0, q0 = 0.0, q1 = 0.0;
  for (int k = g * lpg; k < (g + 1) * lpg; ++k) {
    const double2 v = w[a ? a[k] : k];
    s0 += v.x; s1 += v.y;
    q0 += v.x * v.x; q1 += v.y * v.y;
  }
  double* o = S + i * kComps;
  o[WLN_C_SCAL] = s0; o[WLN_C_FERM] = s1; o[WLN_C_SIN] = CUDART_NAN;
  o[WLN_C_SCAL_SQ] = q0; o[WLN_C_FERM_SQ] = q1;
}

// Eq. corrcoef between row ref and every row of X over its samples, one warp
// per row: x(r, n) = X[(r n_samples + n) stride + comp].  Two passes (means,
// then centred sums) with lanes striding the samples and a fixed butterfly.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void corrcoef_kernel(const double* X, int32_t n_rows, int32_t n_samples,
                                int32_t stride, int32_t comp, int32_t ref, double* out) {
  const int64_t row = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n_rows) return;
  const double* x = X + row * static_cast<int64_t>(n_samples) * stride + comp;
  const double* y = X + static_cast<int64_t>(ref) * n_samples * stride + comp;
  double sx = 0.0, sy = 0.0;
  for (int n = lane; n < n_samples; n += 32) {
    sx += x[static_cast<int64_t>(n) * stride];
    sy += y[static_cast<int64_t>(n) * stride];
  }
  const double mx = warp_sum(sx) / n_samples, my = warp_sum(sy) / n_samples;
  double sxy = 0.0, sxx = 0.0, syy = 0.0;
  for (int n = lane; n < n_samples; n += 32) {
    const double dx = x[static_cast<int64_t>(n) * stride] - mx;
    const double dy = y[static_cast<int64_t>(n) * stride] - my;
    sxy += dx * dy; sxx += dx * dx; syy += dy * dy;
  }
  sxy = warp_sum(sxy); sxx = warp_sum(sxx); syy = warp_sum(syy);
  if (lane == 0) out[row] = sxy / sqrt(sxx * syy);
}

__global__ void group_mean_sem_kernel(const double* x, int32_t n_rows, int32_t G, double* out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_rows) return;
  double m = 0.0;
  for (int g = 0; g < G; ++g) m += x[q * G + g];
  m /= G;
  double ss = 0.0;
  for (int g = 0; g < G; ++g) ss += (x[q * G + g] - m) * (x[q * G + g] - m);
  out[2 * q] = m;
  out[2 * q + 1] = sqrt(ss / (static_cast<double>(G) * (G - 1)));
}

}  // namespace

cudaError_t launch_jackknife(cudaStream_t s, const double* S, int32_t n_points, int32_t G,
                             int32_t lpg, int32_t comp, double* mean, double* sem,
                             double* jk_var, double* dev_scratch, double* cov, int64_t* launches,
                             bool cov_packed) {
  const unsigned blocks = static_cast<unsigned>((n_points + 255) / 256);
  jackknife_kernel<<<blocks, 256, 0, s>>>(S, n_points, G, lpg, comp, mean, sem, jk_var,
                                          cov ? dev_scratch : nullptr);
  ++*launches;
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess || !cov) return err;
  const unsigned nt = static_cast<unsigned>((n_points + kTile - 1) / kTile);
  covariance_kernel<<<dim3(nt, nt), 256, 0, s>>>(dev_scratch, n_points, G, cov, cov_packed ? 1 : 0);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_extrapolate(cudaStream_t s, const double* level_sums, int32_t n_points,
                               int32_t G, int32_t lpg, double* out) {
  const int64_t n = 2 * static_cast<int64_t>(n_points);
  extrapolate_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(level_sums, n_points,
                                                                           G, lpg, out);
  return cudaGetLastError();
}

cudaError_t launch_group_sums_loops(cudaStream_t s, const double* W, int64_t n_points,
                                    int32_t n_loops, int32_t G, bool shuffle, uint64_t seed,
                                    int32_t* perm, double* S, int64_t* launches) {
  cudaError_t err = cudaSuccess;
  if (shuffle) {
    shuffle_kernel<<<static_cast<unsigned>((n_points + 127) / 128), 128, 0, s>>>(
        n_points, n_loops, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32), perm);
    ++*launches;
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  const int64_t n = n_points * G;
  group_sums_loops_kernel<<<static_cast<unsigned>((n + 127) / 128), 128, 0, s>>>(
      reinterpret_cast<const double2*>(W), n_points, n_loops, G, shuffle ? perm : nullptr, S);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_corrcoef(cudaStream_t s, const double* X, int32_t n_rows, int32_t n_samples,
                            int32_t stride, int32_t comp, int32_t ref, double* out) {
  const int64_t threads = static_cast<int64_t>(n_rows) * 32;
  corrcoef_kernel<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, s>>>(
      X, n_rows, n_samples, stride, comp, ref, out);
  return cudaGetLastError();
}

cudaError_t launch_loop_sem(cudaStream_t s, const double* S, int32_t n_points, int32_t G,
                            int32_t n_loops, int32_t comp_sum, int32_t comp_sq, double* out) {
  loop_sem_kernel<<<static_cast<unsigned>((n_points + 255) / 256), 256, 0, s>>>(
      S, n_points, G, n_loops, comp_sum, comp_sq, out);
  return cudaGetLastError();
}

cudaError_t launch_effective_action_full(cudaStream_t s, const QuadProfile* qp,
                                         int32_t n_profiles, int32_t max_rho,
                                         int32_t n_rho_total, int64_t n_points,
                                         const int32_t* point_profile, const double* rho,
                                         const double* T, const double* S, int32_t G,
                                         int32_t lpg, int32_t spinor, double* d_groups,
                                         double* gamma_groups, double* gamma, double* density,
                                         double* integrand, int64_t* launches) {
  // density (n_rho_total x 3, never null) carries the LCF T integral in column 2.
  const int64_t n_thr = static_cast<int64_t>(max_rho) * (G + 1);
  density_kernel<<<dim3(static_cast<unsigned>((n_thr + 127) / 128), n_profiles), 128, 0, s>>>(
      qp, rho, T, S, G, lpg, spinor, d_groups, density);
  ++*launches;
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  action_kernel<<<dim3(G + 1, n_profiles), 256, 0, s>>>(qp, rho, G, d_groups, density,
                                                        gamma_groups, gamma);
  ++*launches;
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  mean_sem_rows_kernel<<<static_cast<unsigned>((n_profiles + 127) / 128), 128, 0, s>>>(
      gamma_groups, n_profiles, G, gamma, 3);
  ++*launches;
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  mean_sem_rows_kernel<<<static_cast<unsigned>((n_rho_total + 127) / 128), 128, 0, s>>>(
      d_groups, n_rho_total, G, density, 3);
  ++*launches;
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (integrand) {
    integrand_kernel<<<static_cast<unsigned>((n_points + 127) / 128), 128, 0, s>>>(
        qp, point_profile, rho, T, S, n_points, G, lpg, spinor, integrand);
    ++*launches;
    err = cudaGetLastError();
  }
  return err;
}

cudaError_t launch_effective_action(cudaStream_t s, const QuadProfile* qp, int32_t n_profiles,
                                    const double* rho, const double* T, const double* S,
                                    int32_t G, int32_t lpg, int32_t spinor, double* gamma_groups,
                                    double* gamma_mean_sem, int64_t* launches) {
  effective_action_kernel<<<dim3(G, n_profiles), 256, 0, s>>>(qp, rho, T, S, G, lpg, spinor,
                                                              gamma_groups);
  ++*launches;
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  group_mean_sem_kernel<<<(n_profiles + 127) / 128, 128, 0, s>>>(gamma_groups, n_profiles, G,
                                                                 gamma_mean_sem);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace wln
