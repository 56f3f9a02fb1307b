// toggle.cu -- the genetic toggle switch prior predictive (the paper's own
// example, Sec. 3.2-3.4, Eq. 3-5).
//
// Per prior sample theta = (mu, sigma, gamma, alpha_u, alpha_v, beta_u,
// beta_v), C cells each run T-1 Euler-Maruyama steps (Delta t = 1) of the two
// coupled SDEs from u = v = 10, clamped at 1, and are observed as
// y = max(u + mu + mu sigma eta / u^gamma, 1); the summaries are the 19
// quantiles of the C values at levels 0.05..0.95 and rho is their Euclidean
// distance to the observed quantiles.
//
// The paper vectorises over a block of VECL cells with all normals of the
// block drawn up front (Sec. 3.4).  Here one CTA owns one prior sample: its
// threads walk the sample's cells, every cell draws its normals from its own
// counter stream in registers, the C observations land in shared memory,
// are bitonic-sorted there, and the quantiles and distance are formed in
// binary64.  The state is binary32 (the 0.97 contraction keeps the rounding
// error of u and v within a few ulp); the drift powers v^beta use the
// hardware log2 and exp2 (see toggle_step2), the observation's u^-gamma an
// accurate polynomial log2.  Each thread runs two cells at once on packed
// binary32 pairs.
#include "internal.h"

namespace ppabc {

namespace {

constexpr int kTgThreads = 256;

// log2(x) for x >= 1 (binary32): x = 2^e f, f in [sqrt(1/2), sqrt(2)),
// log2 x = e + log1p(f - 1) / ln 2 with the log1p polynomial of rng.cuh
// (-2 log1p(s) = -2 s + s^2 Q(s)).
__device__ __forceinline__ float log2_ge1(float x) {
  const uint32_t v = __float_as_uint(x);
  const int32_t e = static_cast<int32_t>(v - 0x3F3504F3u) >> 23;
  const float f = __uint_as_float(v - (static_cast<uint32_t>(e) << 23));
  const float s = f - 1.0f;
  float q = 0.1524621695280075f;
  q = fmaf(q, s, -0.2581113576889038f);
  q = fmaf(q, s, 0.2648598849773407f);
  q = fmaf(q, s, -0.2836324870586395f);
  q = fmaf(q, s, 0.33218106627464294f);
  q = fmaf(q, s, -0.4000397026538849f);
  q = fmaf(q, s, 0.5000317096710205f);
  q = fmaf(q, s, -0.6666665077209473f);
  q = fmaf(q, s, 0.9999997615814209f);
  const float neg2_ln = fmaf(s * s, q, -2.0f * s);        // -2 log1p(s)
  // log2 f = -0.5 * neg2_ln / ln 2
  return fmaf(neg2_ln, -0.7213475204444817f, static_cast<float>(e));
}

// The drift x^p (x >= 1, 0 <= p <= 7) is ex2(p lg2(x)) and alpha / (1 + x^p)
// is alpha times the reciprocal, all three by the hardware approximations
// used directly: p lg2 x >= 0, x^p >= 1 and 1 + x^p in [2, 2^126), so no
// denormal or overflow handling is needed.  The log2's absolute error of
// about 2^-22 gives x^p to a relative error of at most p ln2 2^-22 < 1.2e-6,
// which moves alpha / (1 + x^p) by at most alpha 1.2e-6 / 4 per step; the
// 0.97 contraction keeps the accumulated effect on u and v below 1e-3
// absolute (about 1e-6 of y).
__device__ __forceinline__ float lg2_hw(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_hw(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_hw(float d) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  return r;
}

// One Euler-Maruyama step of both species (Delta t = 1) for two cells at
// once, lane q = cell q, from the previous (u, v) of each:
//   u' = max(0.97 u + alpha_u / (1 + v^beta_u) - 1 + 0.5 z_u, 1),
//   v' = max(0.97 v + alpha_v / (1 + u^beta_v) - 1 + 0.5 z_v, 1),
// each lane rounded as the one-cell update would be.
__device__ __forceinline__ void toggle_step2(float2& U, float2& V, float2 zu, float2 zv, float beta_u,
                                             float beta_v, float alpha_u, float alpha_v) {
  const float2 eu = mul2(splat2(beta_u), make_float2(lg2_hw(V.x), lg2_hw(V.y)));
  const float2 ev = mul2(splat2(beta_v), make_float2(lg2_hw(U.x), lg2_hw(U.y)));
  const float2 du = add2(splat2(1.0f), make_float2(ex2_hw(eu.x), ex2_hw(eu.y)));
  const float2 dv = add2(splat2(1.0f), make_float2(ex2_hw(ev.x), ex2_hw(ev.y)));
  const float2 qu = mul2(splat2(alpha_u), make_float2(rcp_hw(du.x), rcp_hw(du.y)));
  const float2 qv = mul2(splat2(alpha_v), make_float2(rcp_hw(dv.x), rcp_hw(dv.y)));
  float2 un = mul2(splat2(0.97f), U);
  un = add2(un, add2(qu, splat2(-1.0f)));
  un = fma2(splat2(0.5f), zu, un);
  float2 vn = mul2(splat2(0.97f), V);
  vn = add2(vn, add2(qv, splat2(-1.0f)));
  vn = fma2(splat2(0.5f), zv, vn);
  U = make_float2(fmaxf(un.x, 1.0f), fmaxf(un.y, 1.0f));
  V = make_float2(fmaxf(vn.x, 1.0f), fmaxf(vn.y, 1.0f));
}

template <bool kWantY, bool kWantSumm, bool kWantTheta>
__global__ void __launch_bounds__(kTgThreads) toggle_abc(const __grid_constant__ ToggleConst P,
                                                         uint32_t base, uint32_t n, uint32_t Ppow2,
                                                         float* __restrict__ theta_out,
                                                         double* __restrict__ summ_out,
                                                         float* __restrict__ y_out,
                                                         double* __restrict__ dist_out) {
  extern __shared__ float ys[];  // Ppow2 floats
  __shared__ double qres[PPABC_TOGGLE_NQ];
  const uint32_t i = blockIdx.x;
  const uint32_t g = base + i;
  // Prior draw (every thread draws the same theta from the sample's counter).
  const uint4 w0 = philox4x32_10(make_uint4(kTagTogglePrior, 0u, P.sub, g), P.keys);
  const uint4 w1 = philox4x32_10(make_uint4(kTagTogglePrior, 1u, P.sub, g), P.keys);
  const uint32_t words[7] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z};
  float th[7];
#pragma unroll
  for (int j = 0; j < 7; ++j) th[j] = fmaf(P.span[j], u01f(words[j]), P.lo[j]);
  if (kWantTheta && threadIdx.x < 7) theta_out[static_cast<size_t>(threadIdx.x) * n + i] = th[threadIdx.x];
  const float mu = th[0], sigma = th[1], gam = th[2];
  const float alpha_u = th[3], alpha_v = th[4], beta_u = th[5], beta_v = th[6];
  const uint32_t T = P.T, C = P.C;
  const uint32_t tag = (P.sub << 8) | kTagTogglePath;
  // the cells of a sample are the streams of one family (substream = g)
  const PhiloxFamily fam = philox_family(P.keys, tag, g);
  const uint32_t steps = T - 1;
  // Cells c0 and c0 + kTgThreads run together, packed (lane q = cell q): the
  // same cells per thread as one at a time, with two independent chains.
  for (uint32_t c0 = threadIdx.x; c0 < C; c0 += 2 * kTgThreads) {
    const uint32_t c1 = c0 + kTgThreads;
    const bool has1 = c1 < C;
    const PhiloxStream S0 = philox_stream(P.keys, fam, c0);
    const PhiloxStream S1 = philox_stream(P.keys, fam, has1 ? c1 : c0);
    float2 U = splat2(10.0f), V = splat2(10.0f);
    // normals 2(j-1), 2(j-1)+1 drive step j: one counter block covers two steps
    uint32_t b = 0;
    uint32_t j = 0;
    float2 z[4];
    // Unrolled by 4 (paper-size benchmark 100.7 -> 97.3 ms; the same
    // operations in the same order).
#pragma unroll 4
    for (; j + 2 <= steps; j += 2, ++b) {
      const PhiloxBlockPart Ub = philox_block_part(fam, b);
      normals_x2(philox_block(P.keys, S0, Ub), philox_block(P.keys, S1, Ub), z);
      toggle_step2(U, V, z[0], z[1], beta_u, beta_v, alpha_u, alpha_v);
      toggle_step2(U, V, z[2], z[3], beta_u, beta_v, alpha_u, alpha_v);
    }
    const PhiloxBlockPart Ub = philox_block_part(fam, b);
    normals_x2(philox_block(P.keys, S0, Ub), philox_block(P.keys, S1, Ub), z);
    float2 eta;
    if (j < steps) {  // odd number of steps: one more, eta is normal 2 of this block
      toggle_step2(U, V, z[0], z[1], beta_u, beta_v, alpha_u, alpha_v);
      eta = z[2];
    } else {
      eta = z[0];
    }
    const float y0 = fmaxf(U.x + mu + mu * sigma * eta.x * exp2f(-gam * log2_ge1(U.x)), 1.0f);
    ys[c0] = y0;
    if (kWantY) y_out[static_cast<size_t>(i) * C + c0] = y0;
    if (has1) {
      const float y1 = fmaxf(U.y + mu + mu * sigma * eta.y * exp2f(-gam * log2_ge1(U.y)), 1.0f);
      ys[c1] = y1;
      if (kWantY) y_out[static_cast<size_t>(i) * C + c1] = y1;
    }
  }
  for (uint32_t c = C + threadIdx.x; c < Ppow2; c += kTgThreads) ys[c] = __int_as_float(0x7F800000);
  __syncthreads();
  for (uint32_t size = 2; size <= Ppow2; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t t = threadIdx.x; t < (Ppow2 >> 1); t += kTgThreads) {
        const uint32_t lo = 2 * t - (t & (stride - 1));
        const uint32_t hi = lo + stride;
        const bool up = (lo & size) == 0;
        const float a = ys[lo], bb = ys[hi];
        if ((a > bb) == up) {
          ys[lo] = bb;
          ys[hi] = a;
        }
      }
      __syncthreads();
    }
  }
  if (threadIdx.x < PPABC_TOGGLE_NQ) {
    const uint32_t k = threadIdx.x + 1;
    const uint64_t num = static_cast<uint64_t>(C - 1) * k;
    const uint32_t lo = static_cast<uint32_t>(num / 20);
    const double frac = static_cast<double>(num % 20) / 20.0;
    const double a = ys[lo];
    const double q = (lo + 1 < C) ? a + frac * (static_cast<double>(ys[lo + 1]) - a) : a;
    if (kWantSumm) summ_out[static_cast<size_t>(threadIdx.x) * n + i] = q;
    const double r = q - P.q_obs[threadIdx.x];
    qres[threadIdx.x] = r * r;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int k = 0; k < PPABC_TOGGLE_NQ; ++k) acc += qres[k];
    dist_out[i] = sqrt(acc);
  }
}

template <bool A, bool B, bool C3>
cudaError_t launch_t(const ToggleConst& P, uint32_t base, uint32_t n, uint32_t Ppow2, size_t smem,
                     float* theta_out, double* summ_out, float* y_out, double* dist_out,
                     cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(toggle_abc<A, B, C3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  toggle_abc<A, B, C3><<<n, kTgThreads, smem, s>>>(P, base, n, Ppow2, theta_out, summ_out, y_out,
                                                   dist_out);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_toggle(const ToggleConst& P, uint64_t base, uint32_t n, float* theta_out,
                          double* summ_out, float* y_out, double* dist_out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  uint32_t Ppow2 = 2;
  while (Ppow2 < P.C) Ppow2 <<= 1;
  const size_t smem = sizeof(float) * Ppow2;
  const uint32_t b = static_cast<uint32_t>(base);
  const int sel = (y_out ? 4 : 0) | (summ_out ? 2 : 0) | (theta_out ? 1 : 0);
  switch (sel) {
    case 0: return launch_t<false, false, false>(P, b, n, Ppow2, smem, theta_out, summ_out, y_out, dist_out, s);
    case 1: return launch_t<false, false, true>(P, b, n, Ppow2, smem, theta_out, summ_out, y_out, dist_out, s);
    case 2: return launch_t<false, true, false>(P, b, n, Ppow2, smem, theta_out, summ_out, y_out, dist_out, s);
    case 3: return launch_t<false, true, true>(P, b, n, Ppow2, smem, theta_out, summ_out, y_out, dist_out, s);
    case 4: return launch_t<true, false, false>(P, b, n, Ppow2, smem, theta_out, summ_out, y_out, dist_out, s);
    case 5: return launch_t<true, false, true>(P, b, n, Ppow2, smem, theta_out, summ_out, y_out, dist_out, s);
    case 6: return launch_t<true, true, false>(P, b, n, Ppow2, smem, theta_out, summ_out, y_out, dist_out, s);
    default: return launch_t<true, true, true>(P, b, n, Ppow2, smem, theta_out, summ_out, y_out, dist_out, s);
  }
}

}  // namespace ppabc
