// Unit-loop generation on the device (paper Sec. "Loop Generation").
//
// Each loop is a closed, centre-of-mass-centred polygon of N points whose
// increments follow the discretised free action: Gaussian, variance 2/N per
// component, conditioned on closing.  The increments come from
// Philox-4x32-10 (Salmon et al., SC'11) through Box-Muller, with counter
// (j, loop, 0, 0) and key (seed_lo, seed_hi), so any loop can be regenerated
// on its own.  Arithmetic after the integer stream is in double precision;
// points are stored as float in the blocked layout described in
// wln_internal.cuh.
#include "wln_internal.cuh"

namespace wln {
namespace {

// u in (0, 1): centre of the k-th of 2^32 cells (exact in double).
__device__ __forceinline__ double uniform_open(uint32_t k) {
  return (static_cast<double>(k) + 0.5) * 0x1p-32;
}

// Four increments xi_x[2j], xi_y[2j], xi_x[2j+1], xi_y[2j+1] of one loop.
__device__ __forceinline__ void increments(uint64_t seed, uint32_t loop, uint32_t j,
                                           double scale, double& x0, double& y0, double& x1,
                                           double& y1) {
  const uint4 u = philox4x32_10(make_uint4(j, loop, 0u, 0u), static_cast<uint32_t>(seed),
                                static_cast<uint32_t>(seed >> 32));
  double s, c;
  const double ra = scale * sqrt(-2.0 * log(uniform_open(u.x)));
  sincospi(2.0 * uniform_open(u.y), &s, &c);
  x0 = ra * c;
  y0 = ra * s;
  const double rb = scale * sqrt(-2.0 * log(uniform_open(u.z)));
  sincospi(2.0 * uniform_open(u.w), &s, &c);
  x1 = rb * c;
  y1 = rb * s;
}

__global__ void philox_stream_kernel(uint64_t seed, int64_t loop0, int32_t n_loops,
                                     int32_t n_calls, uint4* out) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= static_cast<int64_t>(n_loops) * n_calls) return;
  const uint32_t loop = static_cast<uint32_t>(loop0 + i / n_calls);
  const uint32_t j = static_cast<uint32_t>(i % n_calls);
  out[i] = philox4x32_10(make_uint4(j, loop, 0u, 0u), static_cast<uint32_t>(seed),
                         static_cast<uint32_t>(seed >> 32));
}

// Loop generation in two kernels over a slice of blocks (32 loops each,
// lane = loop).  gen_increments_kernel: one warp per (block, chunk of M
// points) draws the chunk's raw increments xi_k once, keeps them in `xi`
// ([block][point][lane], double2) and writes the chunk's sums of xi_k and
// k xi_k to `part` ([block][chunk][4][lane]).  Its many short warps spread
// the double-precision Box-Muller work evenly over the SMs.
// gen_close_kernel: one CTA per block, warp w taking points
// [w N / WG, (w + 1) N / WG).  The warp adds up its chunks' sums, and a scan
// over the warps gives its starting partial sum S_{k0}.  With mu = mean(xi)
// the closed positions are p_k = S_k - k mu (S_k = sum_{j<k} xi_j), and their
// mean is (1/N) sum_j xi_j (N - 1 - j) - mu (N - 1)/2.  The warp writes
// y_k = p_k - mean(p) for its points from the stored increments.
__global__ void __launch_bounds__(32 * kGenWarps) gen_increments_kernel(
    uint64_t seed, int64_t loop0, int32_t ppl, int32_t b0, int32_t n_items, int32_t M,
    double2* xi, double* part) {
  const int lane = threadIdx.x & 31;
  const int item = static_cast<int>(blockIdx.x) * kGenWarps + static_cast<int>(threadIdx.x >> 5);
  if (item >= n_items) return;
  const int C = ppl / M;
  const int bl = item / C;
  const int k0 = (item - bl * C) * M;
  // Philox counter word 1: the loop's global index
  const uint32_t loop =
      static_cast<uint32_t>(loop0 + (static_cast<int64_t>(b0) + bl) * 32 + lane);
  const double scale = sqrt(2.0 / ppl);
  double sx = 0.0, sy = 0.0, wx = 0.0, wy = 0.0;
  double2* out = xi + (static_cast<size_t>(bl) * ppl + k0) * 32 + lane;
  for (int k = k0; k < k0 + M; k += 2) {
    double x0, y0, x1, y1;
    increments(seed, loop, k >> 1, scale, x0, y0, x1, y1);
    sx += x0; sy += y0;
    wx += k * x0; wy += k * y0;
    sx += x1; sy += y1;
    wx += (k + 1) * x1; wy += (k + 1) * y1;
    out[0] = make_double2(x0, y0);
    out[32] = make_double2(x1, y1);
    out += 64;
  }
  double* pp = part + static_cast<size_t>(item) * 128 + lane;
  pp[0] = sx; pp[32] = sy; pp[64] = wx; pp[96] = wy;
}

template <int WG>
__global__ void __launch_bounds__(32 * WG) gen_close_kernel(int32_t ppl, int32_t b0, int32_t M,
                                                            const double2* xi, const double* part,
                                                            float4* blocks, double* xy64,
                                                            int32_t n_loops) {
  __shared__ double sums[WG][32][4];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int bl = blockIdx.x;
  const int b = b0 + bl;
  const int32_t local = b * 32 + lane;
  const int R = ppl / WG;   // points of this warp (even, a multiple of M)
  const int k0 = w * R;
  const int C = ppl / M;
  double sx = 0.0, sy = 0.0, wx = 0.0, wy = 0.0;
  const double* pp = part + (static_cast<size_t>(bl) * C + k0 / M) * 128 + lane;
  for (int j = 0; j < R / M; ++j, pp += 128) {
    sx += pp[0]; sy += pp[32]; wx += pp[64]; wy += pp[96];
  }
  sums[w][lane][0] = sx; sums[w][lane][1] = sy;
  sums[w][lane][2] = wx; sums[w][lane][3] = wy;
  __syncthreads();
  double tx = 0.0, ty = 0.0, twx = 0.0, twy = 0.0, px = 0.0, py = 0.0;
  for (int v = 0; v < WG; ++v) {
    if (v == w) { px = tx; py = ty; }
    tx += sums[v][lane][0]; ty += sums[v][lane][1];
    twx += sums[v][lane][2]; twy += sums[v][lane][3];
  }
  const double N = ppl;
  const double mux = tx / N, muy = ty / N;
  // mean_k p_k = (1/N) sum_k (S_k - k mu) = (1/N) sum_j xi_j (N-1-j) - mu (N-1)/2
  const double cmx = ((N - 1.0) * tx - twx) / N - mux * (N - 1.0) * 0.5;
  const double cmy = ((N - 1.0) * ty - twy) / N - muy * (N - 1.0) * 0.5;
  // y_k = p_k - mean(p), carried from the warp's first point
  double yx = (px - k0 * mux) - cmx, yy = (py - k0 * muy) - cmy;

  const double2* in = xi + (static_cast<size_t>(bl) * ppl + k0) * 32 + lane;
  float4* row = blocks + (static_cast<size_t>(b) * (ppl / 2) + k0 / 2) * 32 + lane;
  double* ox = xy64 ? xy64 + static_cast<size_t>(local) * 2 * ppl : nullptr;
  const bool real = local < n_loops;
  for (int k = k0; k < k0 + R; k += 2) {
    const double2 a = in[0], c = in[32];
    in += 64;
    const double ax = yx, ay = yy;
    yx += a.x - mux; yy += a.y - muy;
    const double bx = yx, by = yy;
    yx += c.x - mux; yy += c.y - muy;
    *row = make_float4(__double2float_rn(ax), __double2float_rn(ay), __double2float_rn(bx),
                       __double2float_rn(by));
    row += 32;
    if (ox && real) {
      ox[k] = ax; ox[k + 1] = bx;
      ox[ppl + k] = ay; ox[ppl + k + 1] = by;
    }
  }
}

// d-loops (paper Sec. "Loop Generation", Eqs. yn2 and ynk): from the point
// y_N = y_0 = 0, level k (N_k = 2^k) adds the points q N/N_k, q odd, each
// Gaussian about the mean of its two neighbours of the previous level with
// variance 1/N_k per component; then the centre of mass is removed.
// Gaussian number m (in creation order) comes from Philox call m/2 with
// counter (m/2, loop, 1, 0): (u0,u1) for even m, (u2,u3) for odd m.  Number m
// belongs to level N_k = 2^(floor(log2(m + 1)) + 1), as its
// (m + 2 - N_k/2)-th new point: q = 2 (m + 1 - N_k/2) + 1.
//
// Two kernels over a slice of blocks (32 loops each, lane = loop), positions
// in double2 at g[block][point][lane]:
//  gen_dgauss_kernel: one warp per (block, M consecutive numbers m) draws
//   the Gaussians and stores sqrt(1/N_k) z at the point each one places (the
//   double-precision Box-Muller work, spread evenly over the SMs);
//  gen_dbuild_kernel: one CTA per block adds, level by level, the mean of
//   each new point's two neighbours (the level's points split over the
//   warps, a barrier between levels: every parent was written one level
//   earlier), removes the centre of mass and stores.
__global__ void __launch_bounds__(32 * kGenWarps) gen_dgauss_kernel(uint64_t seed, int64_t loop0,
                                                                   int32_t ppl, int32_t b0,
                                                                   int32_t n_items, int32_t M,
                                                                   double2* g) {
  const int lane = threadIdx.x & 31;
  const int item = static_cast<int>(blockIdx.x) * kGenWarps + static_cast<int>(threadIdx.x >> 5);
  if (item >= n_items) return;
  const int C = ppl / M;
  const int bl = item / C;
  const int m0 = (item - bl * C) * M;
  const uint32_t loop =
      static_cast<uint32_t>(loop0 + (static_cast<int64_t>(b0) + bl) * 32 + lane);
  const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  double2* G = g + static_cast<size_t>(bl) * ppl * 32 + lane;
  const int m1 = min(m0 + M, ppl - 1);   // numbers 0 .. N - 2 place points 1 .. N - 1
  uint4 u = make_uint4(0, 0, 0, 0);
  int level_n = 0;      // the N_k whose sigma is held (a chunk spans at most two levels)
  double sigma = 0.0;
  for (int m = m0; m < m1; ++m) {
    if ((m & 1) == 0) u = philox4x32_10(make_uint4(static_cast<uint32_t>(m >> 1), loop, 1u, 0u), k0, k1);
    const uint32_t ua = (m & 1) ? u.z : u.x, ub = (m & 1) ? u.w : u.y;
    const int Nk = 2 << (31 - __clz(m + 1));   // 2^(floor(log2(m + 1)) + 1)
    const int q = 2 * (m + 1 - Nk / 2) + 1;
    if (Nk != level_n) {   // the same on every lane
      level_n = Nk;
      sigma = sqrt(1.0 / Nk);
    }
    double sn, cs;
    const double r = sqrt(-2.0 * log(uniform_open(ua)));
    sincospi(2.0 * uniform_open(ub), &sn, &cs);
    G[static_cast<size_t>(q) * (ppl / Nk) * 32] = make_double2(sigma * (r * cs), sigma * (r * sn));
  }
}

template <int WG>
__global__ void __launch_bounds__(32 * WG) gen_dbuild_kernel(int32_t ppl, int32_t b0, double2* g,
                                                            float4* blocks, double* xy64,
                                                            int32_t n_loops) {
  __shared__ double cms[WG][32][2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int bl = blockIdx.x;
  const int b = b0 + bl;
  const int32_t local = b * 32 + lane;
  double2* W = g + static_cast<size_t>(bl) * ppl * 32 + lane;
  if (w == 0) W[0] = make_double2(0.0, 0.0);
  __syncthreads();
  constexpr int kBatch = WG >= 8 ? 4 : 8;   // new points of a warp handled together
  for (int32_t Nk = 2; Nk <= ppl; Nk *= 2) {
    // the level's new points split over the warps; the barrier below makes
    // them visible to every warp before the next level reads them as parents
    const int32_t stride = ppl / Nk, n_new = Nk / 2;
    const int32_t per = (n_new + WG - 1) / WG;
    const int32_t ja = w * per, jb = min(n_new, ja + per);
    for (int32_t j0 = ja; j0 < jb; j0 += kBatch) {
      // parents (the previous level) first, then the new points: within a
      // level no new point is another's parent
      double2 a[kBatch], c[kBatch], d[kBatch];
#pragma unroll
      for (int t = 0; t < kBatch; ++t) {
        if (j0 + t < jb) {
          const int32_t q = 2 * (j0 + t) + 1;
          a[t] = W[static_cast<size_t>((q - 1) * stride) * 32];
          c[t] = W[static_cast<size_t>(((q + 1) * stride) % ppl) * 32];
          d[t] = W[static_cast<size_t>(q * stride) * 32];
        }
      }
#pragma unroll
      for (int t = 0; t < kBatch; ++t) {
        if (j0 + t < jb) {
          const int32_t q = 2 * (j0 + t) + 1;
          W[static_cast<size_t>(q * stride) * 32] =
              make_double2(0.5 * (a[t].x + c[t].x) + d[t].x, 0.5 * (a[t].y + c[t].y) + d[t].y);
        }
      }
    }
    __syncthreads();
  }
  // centre of mass: each warp's points, then the warps' sums in warp order
  const int32_t R = ppl / WG;
  const int32_t k0 = w * R;
  double sx = 0.0, sy = 0.0;
  for (int32_t i = k0; i < k0 + R; ++i) {
    const double2 v = W[static_cast<size_t>(i) * 32];
    sx += v.x;
    sy += v.y;
  }
  cms[w][lane][0] = sx;
  cms[w][lane][1] = sy;
  __syncthreads();
  double cmx = 0.0, cmy = 0.0;
  for (int v = 0; v < WG; ++v) {
    cmx += cms[v][lane][0];
    cmy += cms[v][lane][1];
  }
  cmx /= ppl;
  cmy /= ppl;
  float4* row = blocks + (static_cast<size_t>(b) * (ppl / 2) + k0 / 2) * 32 + lane;
  double* ox = xy64 ? xy64 + static_cast<size_t>(local) * 2 * ppl : nullptr;
  const bool real = local < n_loops;
  for (int32_t k = k0; k < k0 + R; k += 2) {
    const double2 p0 = W[static_cast<size_t>(k) * 32], p1 = W[static_cast<size_t>(k + 1) * 32];
    const double ax = p0.x - cmx, ay = p0.y - cmy, bx = p1.x - cmx, by = p1.y - cmy;
    *row = make_float4(__double2float_rn(ax), __double2float_rn(ay), __double2float_rn(bx),
                       __double2float_rn(by));
    row += 32;
    if (ox && real) {
      ox[k] = ax; ox[k + 1] = bx;
      ox[ppl + k] = ay; ox[ppl + k + 1] = by;
    }
  }
}

__global__ void pack_kernel(const float* xy, float4* blocks, int32_t n_loops, int32_t ppl,
                            int32_t n_blocks) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t rows = ppl / 2;
  if (i >= static_cast<int64_t>(n_blocks) * rows * 32) return;
  const int lane = static_cast<int>(i & 31);
  const int64_t r = (i >> 5) % rows;
  const int64_t b = (i >> 5) / rows;
  const int64_t loop = b * 32 + lane;
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (loop < n_loops) {
    const float* p = xy + loop * 2 * ppl;
    v = make_float4(p[2 * r], p[ppl + 2 * r], p[2 * r + 1], p[ppl + 2 * r + 1]);
  }
  blocks[i] = v;
}

__global__ void unpack_kernel(const float4* blocks, float* xy, int32_t n_loops, int32_t ppl) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t rows = ppl / 2;
  if (i >= static_cast<int64_t>(n_loops) * rows) return;
  const int64_t loop = i / rows, r = i % rows;
  const float4 v = blocks[((loop >> 5) * rows + r) * 32 + (loop & 31)];
  float* p = xy + loop * 2 * ppl;
  p[2 * r] = v.x; p[2 * r + 1] = v.z;
  p[ppl + 2 * r] = v.y; p[ppl + 2 * r + 1] = v.w;
}

// Flags a loop with two cyclically consecutive equal points.
__global__ void degenerate_kernel(const float4* blocks, int32_t n_loops, int32_t ppl,
                                  int* flag) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t rows = ppl / 2;
  if (i >= static_cast<int64_t>(n_loops) * rows) return;
  const int64_t loop = i / rows, r = i % rows;
  const float4* base = blocks + (loop >> 5) * rows * 32 + (loop & 31);
  const float4 a = base[r * 32];
  const float4 b = base[((r + 1) % rows) * 32];
  const bool same01 = a.x == a.z && a.y == a.w;
  const bool same12 = a.z == b.x && a.w == b.y;
  if (same01 || same12) atomicOr(flag, 1);
}

// Per block of 32 loops: the longest segment (closing segment included) and
// the largest distance of a point from the loop's centre, over the block's
// valid loops.  The Wilson kernel bounds the angle its segments subtend at
// the field axis with them.  One CTA per block, a fixed reduction tree.
__global__ void block_stats_kernel(const float4* blocks, int32_t n_loops, int32_t ppl,
                                   float2* stats, float* maxlen) {
  __shared__ float sd[8], sr[8], sl[8][32];
  const int64_t rows = ppl / 2;
  const int64_t b = blockIdx.x;
  const float4* base = blocks + b * rows * 32;
  float d2 = 0.f, r2 = 0.f, len = 0.f;
  // thread t walks lane t & 31 (blockDim is a multiple of 32): the partial
  // lengths of one loop sit in the same lane of every warp
  for (int64_t i = threadIdx.x; i < rows * 32; i += blockDim.x) {
    const int lane = static_cast<int>(i & 31);
    const int64_t r = i >> 5;
    if (b * 32 + lane >= n_loops) continue;
    const float4 a = base[r * 32 + lane];
    const float4 c = base[((r + 1) % rows) * 32 + lane];
    const float ux = a.z - a.x, uy = a.w - a.y, vx = c.x - a.z, vy = c.y - a.w;
    const float du = ux * ux + uy * uy, dv = vx * vx + vy * vy;
    d2 = fmaxf(d2, fmaxf(du, dv));
    r2 = fmaxf(r2, fmaxf(a.x * a.x + a.y * a.y, a.z * a.z + a.w * a.w));
    len += sqrtf(du) + sqrtf(dv);
  }
  sl[threadIdx.x >> 5][threadIdx.x & 31] = len;
  for (int o = 16; o > 0; o >>= 1) {
    d2 = fmaxf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
    r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o));
  }
  if ((threadIdx.x & 31) == 0) { sd[threadIdx.x >> 5] = d2; sr[threadIdx.x >> 5] = r2; }
  __syncthreads();
  if (threadIdx.x < 32) {
    // one loop's length over the warps, then the longest loop of the block
    float l = 0.f;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) l += sl[w][threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) l = fmaxf(l, __shfl_xor_sync(0xffffffffu, l, o));
    if (threadIdx.x == 0) {
      for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w) {
        d2 = fmaxf(d2, sd[w]);
        r2 = fmaxf(r2, sr[w]);
      }
      // square roots and the length rounded up by a relative 2^-20 (the
      // length also by the float sum's rounding, ppl 2^-24): bounds, not estimates
      stats[b] = make_float2(sqrtf(d2) * (1.0f + 0x1p-20f), sqrtf(r2) * (1.0f + 0x1p-20f));
      maxlen[b] = l * (1.0f + 0x1p-20f + static_cast<float>(ppl) * 0x1p-24f);
    }
  }
}

// The block statistics per sub-block of kSubRows rows, one warp each: the
// longest segment starting in the rows (the last one ending at the next
// row's first point, cyclically) and the largest |y| of their points and of
// that next point, rounded up as the block's.  Every segment a chunk of at
// most kSubRows aligned rows walks, and its end points, are covered.
__global__ void sub_stats_kernel(const float4* blocks, int32_t n_loops, int32_t ppl,
                                 int32_t n_blocks, int32_t n_sub, float2* sub) {
  const int lane = threadIdx.x & 31;
  const int64_t item = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (item >= static_cast<int64_t>(n_blocks) * n_sub) return;
  const int64_t b = item / n_sub;
  const int c = static_cast<int>(item - b * n_sub);
  const int rows = ppl / 2;
  const int r0 = c * kSubRows, r1 = min(rows, r0 + kSubRows);
  const float4* base = blocks + b * rows * 32 + lane;
  float d2 = 0.f, r2 = 0.f;
  if (b * 32 + lane < n_loops) {
    for (int r = r0; r < r1; ++r) {
      const float4 a = base[static_cast<size_t>(r) * 32];
      const float4 n = base[static_cast<size_t>((r + 1) % rows) * 32];
      const float ux = a.z - a.x, uy = a.w - a.y, vx = n.x - a.z, vy = n.y - a.w;
      d2 = fmaxf(d2, fmaxf(ux * ux + uy * uy, vx * vx + vy * vy));
      r2 = fmaxf(r2, fmaxf(fmaxf(a.x * a.x + a.y * a.y, a.z * a.z + a.w * a.w),
                           n.x * n.x + n.y * n.y));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    d2 = fmaxf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
    r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o));
  }
  if (lane == 0) sub[item] = make_float2(sqrtf(d2) * (1.0f + 0x1p-20f), sqrtf(r2) * (1.0f + 0x1p-20f));
}

cudaError_t launch_block_stats(cudaStream_t s, const Ensemble& e) {
  block_stats_kernel<<<e.n_blocks, 256, 0, s>>>(e.blocks, e.n_loops, e.ppl, e.stats, e.maxlen);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const int64_t n = static_cast<int64_t>(e.n_blocks) * e.n_sub;
  sub_stats_kernel<<<static_cast<unsigned>((n + 7) / 8), 256, 0, s>>>(e.blocks, e.n_loops, e.ppl,
                                                                     e.n_blocks, e.n_sub, e.sub_stats);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_philox_stream(cudaStream_t s, uint64_t seed, int64_t loop0, int32_t n_loops,
                                 int32_t n_calls, uint32_t* out) {
  const int64_t n = static_cast<int64_t>(n_loops) * n_calls;
  if (n == 0) return cudaSuccess;
  philox_stream_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(
      seed, loop0, n_loops, n_calls, reinterpret_cast<uint4*>(out));
  return cudaGetLastError();
}

int gen_warps(int32_t ppl) { return ppl >= 16 ? 8 : ppl / 2; }
int gen_chunk(int32_t ppl) { return ppl / gen_warps(ppl) < kGenChunk ? ppl / gen_warps(ppl) : kGenChunk; }

int gen_slice_blocks(int32_t n_blocks, int32_t ppl) {
  const size_t per_block = static_cast<size_t>(ppl) * 32 * sizeof(double2) +
                           static_cast<size_t>(ppl / gen_chunk(ppl)) * 128 * sizeof(double);
  const size_t fit = kGenWorkBytes / per_block;
  const size_t slice = fit < 1 ? 1 : fit;
  return static_cast<int>(slice < static_cast<size_t>(n_blocks) ? slice : n_blocks);
}

size_t gen_loops_work_bytes(int32_t n_blocks, int32_t ppl) {
  const size_t slice = static_cast<size_t>(gen_slice_blocks(n_blocks, ppl));
  return slice * ppl * 32 * sizeof(double2) + slice * (ppl / gen_chunk(ppl)) * 128 * sizeof(double);
}

int gen_loops_launches(int32_t n_blocks, int32_t ppl) {
  const int slice = gen_slice_blocks(n_blocks, ppl);
  return 2 * ((n_blocks + slice - 1) / slice) + 3;
}

cudaError_t launch_gen_loops(cudaStream_t s, uint64_t seed, const Ensemble& e, void* work,
                             int* d_degenerate) {
  const int wg = gen_warps(e.ppl), M = gen_chunk(e.ppl);
  const int slice = gen_slice_blocks(e.n_blocks, e.ppl);
  double2* xi = static_cast<double2*>(work);
  double* part = reinterpret_cast<double*>(xi + static_cast<size_t>(slice) * e.ppl * 32);
  cudaError_t err = cudaSuccess;
  for (int b0 = 0; b0 < e.n_blocks && err == cudaSuccess; b0 += slice) {
    const int nb = e.n_blocks - b0 < slice ? e.n_blocks - b0 : slice;
    const int n_items = nb * (e.ppl / M);
    gen_increments_kernel<<<(n_items + kGenWarps - 1) / kGenWarps, 32 * kGenWarps, 0, s>>>(
        seed, e.loop0, e.ppl, b0, n_items, M, xi, part);
    switch (wg) {
      case 8: gen_close_kernel<8><<<nb, 256, 0, s>>>(e.ppl, b0, M, xi, part, e.blocks, e.xy64, e.n_loops); break;
      case 4: gen_close_kernel<4><<<nb, 128, 0, s>>>(e.ppl, b0, M, xi, part, e.blocks, e.xy64, e.n_loops); break;
      case 2: gen_close_kernel<2><<<nb, 64, 0, s>>>(e.ppl, b0, M, xi, part, e.blocks, e.xy64, e.n_loops); break;
      default: return cudaErrorInvalidValue;
    }
    err = cudaGetLastError();
  }
  if (err != cudaSuccess) return err;
  const int64_t n = static_cast<int64_t>(e.n_loops) * (e.ppl / 2);
  degenerate_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(e.blocks, e.n_loops,
                                                                          e.ppl, d_degenerate);
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  return launch_block_stats(s, e);
}

int gen_dslice_blocks(int32_t n_blocks, int32_t ppl) {
  const size_t per_block = static_cast<size_t>(ppl) * 32 * sizeof(double2);
  const size_t fit = kGenWorkBytes / per_block;
  const size_t slice = fit < 1 ? 1 : fit;
  return static_cast<int>(slice < static_cast<size_t>(n_blocks) ? slice : n_blocks);
}

size_t gen_dloops_work_bytes(int32_t n_blocks, int32_t ppl) {
  return static_cast<size_t>(gen_dslice_blocks(n_blocks, ppl)) * ppl * 32 * sizeof(double2);
}

int gen_dloops_launches(int32_t n_blocks, int32_t ppl) {
  const int slice = gen_dslice_blocks(n_blocks, ppl);
  return 2 * ((n_blocks + slice - 1) / slice) + 3;
}

cudaError_t launch_gen_dloops(cudaStream_t s, uint64_t seed, const Ensemble& e, void* work,
                              int* d_degenerate) {
  const int M = e.ppl < kGenChunk ? e.ppl : kGenChunk;
  const int slice = gen_dslice_blocks(e.n_blocks, e.ppl);
  double2* g = static_cast<double2*>(work);
  cudaError_t err = cudaSuccess;
  for (int b0 = 0; b0 < e.n_blocks && err == cudaSuccess; b0 += slice) {
    const int nb = e.n_blocks - b0 < slice ? e.n_blocks - b0 : slice;
    const int n_items = nb * (e.ppl / M);
    gen_dgauss_kernel<<<(n_items + kGenWarps - 1) / kGenWarps, 32 * kGenWarps, 0, s>>>(
        seed, e.loop0, e.ppl, b0, n_items, M, g);
    err = cudaGetLastError();
    if (err != cudaSuccess) break;
    switch (gen_warps(e.ppl)) {
      case 8: gen_dbuild_kernel<8><<<nb, 256, 0, s>>>(e.ppl, b0, g, e.blocks, e.xy64, e.n_loops); break;
      case 4: gen_dbuild_kernel<4><<<nb, 128, 0, s>>>(e.ppl, b0, g, e.blocks, e.xy64, e.n_loops); break;
      case 2: gen_dbuild_kernel<2><<<nb, 64, 0, s>>>(e.ppl, b0, g, e.blocks, e.xy64, e.n_loops); break;
      default: return cudaErrorInvalidValue;
    }
    err = cudaGetLastError();
  }
  if (err != cudaSuccess) return err;
  const int64_t n = static_cast<int64_t>(e.n_loops) * (e.ppl / 2);
  degenerate_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(e.blocks, e.n_loops,
                                                                          e.ppl, d_degenerate);
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  return launch_block_stats(s, e);
}

cudaError_t launch_pack_loops(cudaStream_t s, const float* xy, const Ensemble& e, int* d_degenerate) {
  const int64_t n = static_cast<int64_t>(e.n_blocks) * (e.ppl / 2) * 32;
  pack_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(xy, e.blocks, e.n_loops,
                                                                   e.ppl, e.n_blocks);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const int64_t m = static_cast<int64_t>(e.n_loops) * (e.ppl / 2);
  degenerate_kernel<<<static_cast<unsigned>((m + 255) / 256), 256, 0, s>>>(e.blocks, e.n_loops,
                                                                          e.ppl, d_degenerate);
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  return launch_block_stats(s, e);
}

cudaError_t launch_unpack_loops(cudaStream_t s, const Ensemble& e, float* xy) {
  const int64_t n = static_cast<int64_t>(e.n_loops) * (e.ppl / 2);
  unpack_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(e.blocks, xy, e.n_loops,
                                                                     e.ppl);
  return cudaGetLastError();
}

}  // namespace wln
