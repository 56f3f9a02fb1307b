// bege.cu -- BEGE log-likelihood of many parameter vectors on one return
// series (Sec. 4.2: the BEGE model, its shape recursion, Eq. BEGE_LL,
// Eq. CDF_BEGE discretised as Eq. BEGE_LL_approx, P(a, x) of Eq. incompGamma).
//
// For particle i with theta = (p0, sp, rho_p, phi_p+, phi_p-, n0, sn, rho_n,
// phi_n+, phi_n-, mu) and returns r_1..r_T:
//   u_t = r_t - mu,  ll_i = sum_t log f(u_t; sp, sn, p_{t-1}, n_{t-1}),
//   p_t = p0 + rho_p p_{t-1} + phi_p^{+|-} u_t^2 / (2 sp^2), (p_0, n_0) = (p0, n0),
//   f(u) = (F(u + h) - F(u - h)) / (2h),
//   F(u) = sum_{j=1..100} [1 - P(n, (w_{j-1} - u + n sn) / sn)]
//                         [P(p, (w_j + p sp) / sp) - P(p, (w_{j-1} + p sp) / sp)],
//   w_j = w_0 + j dw, w_0 = 1e-4 - p sp, dw = (10 sp sqrt(p) - w_0) / 99.
//
// The paper vectorises P(a, x) over a block of V grid nodes on one core.
// Here four kernels split the work: the shape recursion (sequential in t,
// one thread per particle); the per-step constants (one thread per
// (particle, t): lgamma of both shapes and the node coordinates); the
// densities (one warp per (particle, t): the 101 grid nodes spread over the
// lanes, the grid differences taken with shuffles); and log f with a
// fixed-order sum over t per particle.
//
// Precision.  The inputs, the shapes, the node coordinates' constants and the
// sums over t are binary64.  GB300 retires a binary64 FMA about 32 times
// slower than a binary32 one, so the per-node work -- the incomplete gamma
// function (series and continued fraction), the prefactors
// exp(a ln x - x - lgamma(a)), the gamma densities of the Taylor nodes and
// the sum over the nodes -- runs in double-float (about 48 bits) on the
// binary32 pipes.  The prefactor's relative error is about 2^-48 times the
// size of its exponent (below 1e-11); the binary64 definition itself carries
// the rounding of F divided by 2h (eps F / h ~ 1e-11 relative).
#include "dfloat.cuh"
#include "internal.h"

namespace ppabc {

namespace {

constexpr int kBegeNw = PPABC_BEGE_NW;  // grid intervals
constexpr int kBegeWarpsPerCta = 8;
constexpr int kGammaMaxIter = 1000000;

inline size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Per-step constants of the density kernel (one record per (particle, t)).
// Positive-shock node j sits at x_j = xa + j xb (= (w_j + p sp) / sp =
// (1e-4 + j dw) / sp), negative-shock node j at x0_j = ya + (j - 1) yb
// (= (w_{j-1} - u + n sn) / sn).
struct BegeTask {
  DF xa, xb;    // 1e-4 / sp, dw / sp
  DF ya, yb;    // (w_0 - u + n sn) / sn, dw / sn
  DF p, lgp;    // positive shape and lgamma of it
  DF nm1, lgn;  // negative shape - 1 and lgamma of the shape
  DF two_delta;  // 2 h / sn
};


// Reciprocals 1 / (a + k), k < kRecip, of one shape (binary64, stored as
// double-float), shared by every node of a task: the series' ratio
// x / (a + k) becomes x * inv[k].
constexpr int kRecip = 256;

// The central difference of the negative-shock factor at node x0 comes from
// the Taylor expansion of P(n, .) about x0 to fifth order in delta = h / sn,
//   P(n, x0 + d) - P(n, x0 - d) = 2 d g [1 + (d^2/6) g2/g + (d^4/120) g4/g] + O(d^7 g6),
// (gk the k-th derivative of the gamma density g) where the node is far from
// the edge of the support on the scale of delta and ln g varies slowly
// across it: x0 >= kTaylorEdge delta max(1, |n - 1|) and delta <=
// kTaylorMaxDelta.  Then delta / x0 <= 0.01 and delta |d ln g / dx| <= 0.03,
// and the omitted terms are below 1e-12 of the value (checked against the
// exact difference at 600 digits over shapes 0.05..200); the two corrections,
// below 2e-4 of the leading term, are formed in binary32 (relative error
// below 1e-10 of the value).  Elsewhere both values are evaluated (in
// binary64).
constexpr float kTaylorEdge = 100.0f;
enum { kTaylor = 0, kTwoValues = 1, kNone = 2 };
constexpr float kTaylorMaxDelta = 0.02f;

// 1 / d for a positive double-float d: the binary32 reciprocal of d.hi and
// one Newton step r + r (1 - d r), the residual formed in double-float
// (relative error about 2^-46).
__device__ __forceinline__ DF df_recip(DF d) {
  const float r = 1.0f / d.hi;
  const DF dr = df_mul(d, DF{r, 0.0f});
  const DF res = df_add(DF{1.0f, 0.0f}, DF{-dr.hi, -dr.lo});
  return df_fast_two_sum(r, r * res.hi);
}

// sum_{j>=0} x^j / (a (a+1) ... (a+j)), ratios from the table
// inv[k] = 1 / (a + k) (computed per term beyond it), two terms per
// convergence check.  Terms at or above 2^-24 of the partial sum are formed and added in
// double-float; the rest of the tail -- terms that are all below one binary32
// ulp of the sum -- in binary32, until a term falls below 2^-49 of the sum
// (the format's own precision).  The binary32 tail's relative error (the
// rounding of its k products) times its size (below 2^-24 of the sum over
// 1 - x/(a+k)) stays far below 2^-40 of the sum.  All terms are positive; for
// x < a + 66 they stay below e^66 / a, inside the binary32 range.
__device__ DF series_df(DF a_df, DF x, const DF* __restrict__ inv) {
  DF term = inv[0], sum = term;
  int k = 1;
  bool small = false;  // the last term is below 2^-24 of the sum
  for (; k + 1 < kRecip; k += 2) {
    term = df_mul(term, df_mul(x, inv[k]));
    sum = df_add(sum, term);
    term = df_mul(term, df_mul(x, inv[k + 1]));
    sum = df_add(sum, term);
    if (term.hi < sum.hi * 0x1p-24f) {
      small = true;
      k += 2;
      break;
    }
  }
  if (!small) {  // past the table: ratios from binary64
    for (; k < kGammaMaxIter; k += 2) {
      term = df_mul(term, df_mul(x, df_recip(df_add_f(a_df, static_cast<float>(k)))));
      sum = df_add(sum, term);
      term = df_mul(term, df_mul(x, df_recip(df_add_f(a_df, static_cast<float>(k + 1)))));
      sum = df_add(sum, term);
      if (term.hi < sum.hi * 0x1p-24f) {
        k += 2;
        break;
      }
    }
  }
  if (term.hi < sum.hi * 0x1p-49f || term.hi == 0.0f) return sum;
  const float xf = x.hi, stop = sum.hi * 0x1p-49f;
  float tf = term.hi, tail = 0.0f;
  bool done = false;
  for (; k + 1 < kRecip; k += 2) {
    tf *= xf * inv[k].hi;
    tail += tf;
    tf *= xf * inv[k + 1].hi;
    tail += tf;
    if (tf < stop || tf == 0.0f) {
      done = true;
      break;
    }
  }
  if (!done) {
    for (; k < kGammaMaxIter; k += 2) {
      tf *= xf / (a_df.hi + static_cast<float>(k));
      tail += tf;
      tf *= xf / (a_df.hi + static_cast<float>(k + 1));
      tail += tf;
      if (tf < stop || tf == 0.0f) break;
    }
  }
  return df_add_f(sum, tail);
}

// The double-float log and exp tables, computed once per call by one CTA
// into the workspace (the density kernel's CTAs copy them into shared memory).
__global__ void __launch_bounds__(128) bege_tables(DfTables* __restrict__ out) {
  for (int i = threadIdx.x; i < 64; i += blockDim.x) out->exp2j[i] = df_split(exp2(static_cast<double>(i) / 64.0));
  for (int i = threadIdx.x; i < 128; i += blockDim.x) {
    const float c = static_cast<float>(1.0 / (1.0 + (static_cast<double>(i) + 0.5) / 128.0));
    out->log_c[i] = c;
    out->log_l[i] = df_split(-log(static_cast<double>(c)));
  }
}
static_assert(sizeof(DfTables) % 16 == 0, "the tables are copied as 16-byte words");

// 2^m x for a double-float x with x.hi below 2^100, in at most two exact
// power-of-two multiplies; results below 2^-126 lose bits or flush to 0
// (such values of P or of a node's difference enter the sum for f, of order
// 1e-5 and more, far below its rounding).
__device__ __forceinline__ DF df_scale(DF x, int m) {
  if (m < -250) return DF{0.0f, 0.0f};
  const int m1 = m < -126 ? -126 : m;
  const float s1 = __int_as_float((m1 + 127) << 23);
  x = DF{x.hi * s1, x.lo * s1};
  if (m != m1) {
    const float s2 = __int_as_float((m - m1 + 127) << 23);
    x = DF{x.hi * s2, x.lo * s2};
  }
  return x;
}

// Where the GPU sums the series (below) rather than the continued fraction.
constexpr float kSeriesPastShape = 65.0f;  // x < a + 1 + 65
constexpr float kCfTiny = 1e-30f;           // modified Lentz's floor for d and c

// Regularised lower incomplete gamma P(a, x), a > 0, given a, lgamma(a) and x
// as double-floats (af = a rounded to binary32), in double-float throughout.
// The power series the paper names,
//   P = exp(-x + a ln x - lgamma(a)) sum_j x^j / (a (a+1) ... (a+j)),
// converges for every x; past x ~ a its terms first grow (to about k = x - a,
// the largest about e^((x-a)^2 / 2a) / x, inside the binary32 range for
// x < a + 66) and then fall, so it needs about (x - a) + sqrt(78 x) terms.
// The series is used for every x < a + 1 and, past the shape, for
// x < a + 66; beyond, Legendre's continued fraction for Q = 1 - P (modified
// Lentz), which converges in a few terms there.  Where the tail bound
//   Q <= exp(-x + a ln x - lgamma(a)) / (x + 1 - max(a, 1))     (x > a - 1)
// is below 2^-56, 1 - Q rounds to 1 whatever Q is, and 1 is returned.  The
// branches are decided on binary32 copies of x and a.  Each loop is bounded
// by kGammaMaxIter terms.  Not inlined: its three call sites share one copy,
// which keeps the density kernel's code within the instruction cache.
__device__ __noinline__ DF gammainc_p_df(float af, DF a_df, DF lga, DF x, const DF* __restrict__ inv, const DfTables& dtab) {
  if (!(x.hi > 0.0f)) return DF{0.0f, 0.0f};
  const DF lead = df_add(df_mul(a_df, df_log(x, dtab)), df_neg(df_add(x, lga)));  // a ln x - x - lgamma(a)
  const float xf = x.hi;
  const bool upper = xf >= af + 1.0f;
  // Tail bound exp(lead) / (x + 1 - max(a, 1)) < 2^-56, in the log domain.
  if (upper && lead.hi < -38.816242f + __logf(xf + 1.0f - fmaxf(af, 1.0f))) return DF{1.0f, 0.0f};
  if (lead.hi < -700.0f) return DF{upper ? 1.0f : 0.0f, 0.0f};  // P < 1e-270 or 1 - P < 1e-270
  int m;
  const DF v = df_exp_scaled(lead, m, dtab);  // exp(lead) = 2^m v, v in [1, 2)
  if (!upper || xf < af + 1.0f + kSeriesPastShape) {
    // series x v: the series is at least 1/a and below e^66 / a, so the
    // product is a normal binary32 pair before the scaling.
    return df_scale(df_mul(series_df(a_df, x, inv), v), m);
  }
  // Q = exp(lead) / (x + 1 - a - 1 (1 - a) / (x + 3 - a - 2 (2 - a) / (x + 5 - a - ...))).
  DF b = df_add(df_add_f(x, 1.0f), df_neg(a_df));
  DF c = DF{1.0f / kCfTiny, 0.0f};
  DF d = df_recip(b);
  DF hq = d;
  for (int i = 1; i < kGammaMaxIter; ++i) {
    const DF an = df_mul_f(df_add_f(df_neg(a_df), static_cast<float>(i)), -static_cast<float>(i));  // -i (i - a)
    b = df_add_f(b, 2.0f);
    d = df_add(df_mul(an, d), b);
    if (fabsf(d.hi) < kCfTiny) d = DF{kCfTiny, 0.0f};
    c = df_add(b, df_mul(an, df_recip(c)));
    if (fabsf(c.hi) < kCfTiny) c = DF{kCfTiny, 0.0f};
    d = df_recip(d);
    const DF del = df_mul(d, c);
    hq = df_mul(hq, del);
    if (fabsf(df_add_f(del, -1.0f).hi) < 0x1p-47f) break;
  }
  const DF q = df_scale(df_mul(hq, v), m);
  return df_add_f(df_neg(q), 1.0f);
}

// Shapes used at each step, one thread per particle; first_bad[i] = the first
// step whose scale is not positive or whose shape is not a positive finite
// number (T if none).
__global__ void bege_shapes(const double* __restrict__ theta, uint32_t np, const double* __restrict__ r,
                            uint32_t T, double* __restrict__ shape_p, double* __restrict__ shape_n,
                            uint32_t* __restrict__ first_bad) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const double p0 = theta[i], sp = theta[np + i], rp = theta[2ull * np + i];
  const double fpp = theta[3ull * np + i], fpm = theta[4ull * np + i];
  const double n0 = theta[5ull * np + i], sn = theta[6ull * np + i], rn = theta[7ull * np + i];
  const double fnp = theta[8ull * np + i], fnm = theta[9ull * np + i], mu = theta[10ull * np + i];
  uint32_t bad = T;
  if (!(sp > 0.0) || !(sn > 0.0)) bad = 0;
  double p = p0, n = n0;
  const double inv2sp2 = 1.0 / (2.0 * sp * sp), inv2sn2 = 1.0 / (2.0 * sn * sn);
  for (uint32_t t = 0; t < T && bad == T; ++t) {
    if (!(p > 0.0) || !(n > 0.0) || !isfinite(p) || !isfinite(n)) {
      bad = t;
      break;
    }
    shape_p[static_cast<size_t>(i) * T + t] = p;
    shape_n[static_cast<size_t>(i) * T + t] = n;
    const double u = r[t] - mu;
    const double u2 = u * u;
    p = p0 + rp * p + (u >= 0.0 ? fpp : fpm) * inv2sp2 * u2;
    n = n0 + rn * n + (u >= 0.0 ? fnp : fnm) * inv2sn2 * u2;
  }
  first_bad[i] = bad;
}

// Per-step constants, one thread per (particle, t): lgamma of both shapes
// and the node coordinates' offsets and spacings, as double-floats.  The
// density kernel runs one warp per (particle, t); doing this binary64 work
// there would run it on a whole warp for one set of values.
__global__ void __launch_bounds__(256) bege_tasks(const double* __restrict__ theta, uint32_t np,
                                                  const double* __restrict__ r, uint32_t T, double h,
                                                  const double* __restrict__ shape_p,
                                                  const double* __restrict__ shape_n,
                                                  const uint32_t* __restrict__ first_bad, uint64_t n_tasks,
                                                  BegeTask* __restrict__ tasks) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t task = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; task < n_tasks;
       task += stride) {
    const uint32_t i = static_cast<uint32_t>(task / T);
    const uint32_t t = static_cast<uint32_t>(task % T);
    if (t >= first_bad[i]) continue;
    const double sp = theta[np + i], sn = theta[6ull * np + i], mu = theta[10ull * np + i];
    const double p = shape_p[task], n = shape_n[task];
    const double u = r[t] - mu;
    const double w0 = 1e-4 - p * sp;
    const double dw = (10.0 * sp * sqrt(p) - w0) / static_cast<double>(kBegeNw - 1);
    BegeTask k;
    k.xa = df_split(1e-4 / sp);
    k.xb = df_split(dw / sp);
    k.ya = df_split((w0 - u + n * sn) / sn);
    k.yb = df_split(dw / sn);
    k.p = df_split(p);
    k.lgp = df_split(lgamma(p));
    k.nm1 = df_split(n - 1.0);
    k.lgn = df_split(lgamma(n));
    k.two_delta = df_split(2.0 * h / sn);
    tasks[task] = k;
  }
}

// Negative-shock node j (1..100) of task K: its coordinate x0 and whether its
// difference comes from the Taylor form, from both values, or is zero (both
// values below 1e-297: P(n, x) <= e^(n ln x - x - lgamma(n)) (n + 1) / n for
// x < n).
__device__ __forceinline__ int node_kind(const BegeTask& K, int j, float delta_f, float nf, float lgn_f, DF& x0) {
  x0 = df_add(K.ya, df_mul_f(K.yb, static_cast<float>(j - 1)));
  const float xm = x0.hi + delta_f;
  if (delta_f <= kTaylorMaxDelta && x0.hi >= kTaylorEdge * delta_f * fmaxf(1.0f, fabsf(K.nm1.hi))) return kTaylor;
  if (!(xm > 0.0f) || (xm < nf && nf * __logf(xm) - xm - lgn_f < -700.0f)) return kNone;
  return kTwoValues;
}

// f(u_t) for task (i, t) per warp.  Lane l owns grid nodes j = l + 32 k,
// k = 0..3 (j <= 100): it evaluates P(p, .) at x_j and, for j >= 1, the
// central difference over u +- h of the node's factor [1 - P(n, .)]; the
// difference P(p, x_j) - P(p, x_{j-1}) takes x_{j-1}'s value from the
// neighbouring lane.  F(u + h) - F(u - h) is accumulated as one sum of
// per-node differences: the same quantity as the two sums differenced,
// without their cancellation.  Away from the edge of the negative shock's
// support the node's difference comes from the Taylor expansion of P(n, .)
// about the node (one density instead of two series); near the edge both
// values are evaluated.  f is written to fout (bege_finish takes its log).
__global__ void __launch_bounds__(32 * kBegeWarpsPerCta, 3)
bege_density(uint32_t np, uint32_t T, double inv_2h, const DfTables* __restrict__ tables,
             const BegeTask* __restrict__ tasks,
             const uint32_t* __restrict__ first_bad, double* __restrict__ fout) {
  __shared__ DF recip[kBegeWarpsPerCta][2][kRecip];
  __shared__ DfTables dtab;
  {
    const uint4* src = reinterpret_cast<const uint4*>(tables);
    uint4* dst = reinterpret_cast<uint4*>(&dtab);
    for (uint32_t q = threadIdx.x; q < sizeof(DfTables) / sizeof(uint4); q += blockDim.x) dst[q] = src[q];
  }
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u;
  DF* inv_p = recip[threadIdx.x >> 5][0];
  DF* inv_n = recip[threadIdx.x >> 5][1];
  const uint64_t n_tasks = static_cast<uint64_t>(np) * T;
  const uint64_t warp0 = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t n_warps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
  for (uint64_t task = warp0; task < n_tasks; task += n_warps) {
    const uint32_t i = static_cast<uint32_t>(task / T);
    const uint32_t t = static_cast<uint32_t>(task % T);
    if (t >= first_bad[i]) continue;  // the whole warp skips together
    const BegeTask K = tasks[task];
    const float delta_f = 0.5f * K.two_delta.hi;
    const float pf = K.p.hi;
    // The n table is needed only where some node of the warp takes both
    // values.
    bool near_edge = false;
    const float nf = K.nm1.hi + 1.0f, lgn_f = K.lgn.hi;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int j = static_cast<int>(lane) + 32 * k;
      DF x0;
      if (j >= 1 && j <= kBegeNw && node_kind(K, j, delta_f, nf, lgn_f, x0) == kTwoValues) near_edge = true;
    }
    const bool fill_n = __any_sync(0xFFFFFFFFu, near_edge);
    const DF n_df = df_add_f(K.nm1, 1.0f);
    __syncwarp();  // the previous task's readers are done with the tables
    for (int k = static_cast<int>(lane); k < kRecip; k += 32) {
      inv_p[k] = df_recip(df_add(K.p, DF{static_cast<float>(k), 0.0f}));
      if (fill_n) inv_n[k] = df_recip(df_add(n_df, DF{static_cast<float>(k), 0.0f}));
    }
    __syncwarp();
    DF acc = DF{0.0f, 0.0f};     // F(u + h) - F(u - h): a sum of non-negative terms
    DF F_last = DF{0.0f, 0.0f};  // F at node 32 k + 31 of the previous group (lane 31's value)
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {  // one copy of the node code: it is large
      const int j = static_cast<int>(lane) + 32 * k;
      const bool live = j <= kBegeNw;
      DF F = DF{0.0f, 0.0f};
      if (live) F = gammainc_p_df(pf, K.p, K.lgp, df_add(K.xa, df_mul_f(K.xb, static_cast<float>(j))), inv_p, dtab);
      DF F_prev = DF{__shfl_up_sync(0xFFFFFFFFu, F.hi, 1), __shfl_up_sync(0xFFFFFFFFu, F.lo, 1)};
      if (lane == 0) F_prev = F_last;
      F_last = DF{__shfl_sync(0xFFFFFFFFu, F.hi, 31), __shfl_sync(0xFFFFFFFFu, F.lo, 31)};
      if (live && j >= 1) {
        // [1 - P(n, x0 - delta)] - [1 - P(n, x0 + delta)], x0 = (w_{j-1} - u + n sn) / sn.
        DF x0;
        const int kind = node_kind(K, j, delta_f, nf, lgn_f, x0);
        DF dG;
        if (kind == kTaylor) {
          // Gamma density g = x^(n-1) e^-x / Gamma(n).  With the derivatives of
          // ln g, L1 = (n-1)/x - 1, L2 = -(n-1)/x^2, L3 = 2(n-1)/x^3 and
          // L4 = -6(n-1)/x^4: g2/g = L1^2 + L2 and
          // g4/g = L1^4 + 6 L1^2 L2 + 4 L1 L3 + 3 L2^2 + L4.
          const DF arg = df_add(df_mul(K.nm1, df_log(x0, dtab)), df_neg(df_add(x0, K.lgn)));
          if (arg.hi < -700.0f) {
            dG = DF{0.0f, 0.0f};
          } else {
            int m;
            const DF g = df_exp_scaled(arg, m, dtab);  // g = 2^m (hi + lo)
            const float ix = 1.0f / x0.hi;
            const float q = K.nm1.hi * ix;
            const float L1 = q - 1.0f, L2 = -q * ix;
            const float L3 = -2.0f * L2 * ix, L4 = -3.0f * L3 * ix;
            const float d2 = delta_f * delta_f;
            const float c2 = (d2 / 6.0f) * fmaf(L1, L1, L2);
            const float c4 = (d2 * d2 / 120.0f) *
                             (L1 * L1 * (L1 * L1 + 6.0f * L2) + 4.0f * L1 * L3 + 3.0f * L2 * L2 + L4);
            dG = df_scale(df_mul(g, df_add_f(K.two_delta, K.two_delta.hi * (c2 + c4))), m);
          }
        } else if (kind == kNone) {
          dG = DF{0.0f, 0.0f};
        } else {
          // Both values in double-float.  Their relative difference is at
          // least about 2 delta |d ln g / dx| > 0.02 here (the node failed the
          // Taylor test), so the difference keeps about 42 bits; where x0 - d
          // is outside the support it is P(n, x0 + d) itself.
          const DF half_delta = DF{0.5f * K.two_delta.hi, 0.5f * K.two_delta.lo};
          const DF xm = df_add(x0, half_delta), xp = df_add(x0, df_neg(half_delta));
          const DF Pm = gammainc_p_df(nf, n_df, K.lgn, xm, inv_n, dtab);
          dG = xp.hi > 0.0f ? df_add(Pm, df_neg(gammainc_p_df(nf, n_df, K.lgn, xp, inv_n, dtab))) : Pm;
        }
        acc = df_add(acc, df_mul(dG, df_add(F, df_neg(F_prev))));
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
      acc = df_add(acc, DF{__shfl_xor_sync(0xFFFFFFFFu, acc.hi, off), __shfl_xor_sync(0xFFFFFFFFu, acc.lo, off)});
    if (lane == 0) fout[task] = df_to_double(acc) * inv_2h;
  }
}

// log f per step (in place: f -> log f, -inf where f is not a positive
// finite number) and ll_i = sum_{t < T} log f in a fixed-order tree per
// particle; -inf if a step was invalid or a density was not positive.
__global__ void __launch_bounds__(256) bege_finish(double* __restrict__ logf, uint32_t T,
                                                   const uint32_t* __restrict__ first_bad,
                                                   double* __restrict__ ll) {
  __shared__ double part[256];
  const uint32_t i = blockIdx.x;
  const uint32_t t_end = first_bad[i] < T ? first_bad[i] : T;
  double s = 0.0;
  for (uint32_t t = threadIdx.x; t < t_end; t += 256) {
    const double f = logf[static_cast<size_t>(i) * T + t];
    const double lf = (f > 0.0 && isfinite(f)) ? log(f) : -INFINITY;
    logf[static_cast<size_t>(i) * T + t] = lf;
    s += lf;
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < static_cast<unsigned>(w)) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) ll[i] = (first_bad[i] < T || part[0] != part[0]) ? -INFINITY : part[0];
}

struct BegeLayout {
  size_t shape_p, shape_n, tasks, tables, first_bad, logf, total;
  BegeLayout(uint64_t np, uint64_t T) {
    size_t o = 0;
    shape_p = o;
    o = align256(o + sizeof(double) * np * T);
    shape_n = o;
    o = align256(o + sizeof(double) * np * T);
    tasks = o;
    o = align256(o + sizeof(BegeTask) * np * T);
    tables = o;
    o = align256(o + sizeof(DfTables));
    first_bad = o;
    o = align256(o + sizeof(uint32_t) * np);
    logf = o;
    o = align256(o + sizeof(double) * np * T);
    total = o;
  }
};

}  // namespace

}  // namespace ppabc

using namespace ppabc;

extern "C" {

size_t bege_loglik_workspace_bytes(uint64_t n_particles, uint32_t T) {
  return BegeLayout(n_particles ? n_particles : 1, T ? T : 1).total;
}

int bege_loglik(const double* theta, uint64_t n_particles, const double* r, uint32_t T, double h,
                double* ll_out, double* logf_out, void* workspace, size_t workspace_bytes, void* stream) {
  if (!theta || !r || !ll_out) return set_error(PPABC_EINVAL, "theta, r and ll_out must be non-NULL");
  if (n_particles == 0 || n_particles > PPABC_BEGE_MAX_PARTICLES)
    return set_error(PPABC_EINVAL, "n_particles must be in [1, %d]", PPABC_BEGE_MAX_PARTICLES);
  if (T == 0 || T > PPABC_BEGE_MAX_T) return set_error(PPABC_EINVAL, "T must be in [1, %d]", PPABC_BEGE_MAX_T);
  if (!(h > 0.0) || !(h < 1.0)) return set_error(PPABC_EINVAL, "h must be in (0, 1)");
  const BegeLayout L(n_particles, T);
  if (!workspace || workspace_bytes < L.total)
    return set_error(PPABC_ENOMEM, "workspace needs %zu bytes, got %zu", L.total, workspace_bytes);
  if (reinterpret_cast<uintptr_t>(workspace) & 255u) return set_error(PPABC_EINVAL, "workspace must be 256-byte aligned");
  int rc = require_device();
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(workspace);
  double* shape_p = reinterpret_cast<double*>(w + L.shape_p);
  double* shape_n = reinterpret_cast<double*>(w + L.shape_n);
  BegeTask* tasks = reinterpret_cast<BegeTask*>(w + L.tasks);
  DfTables* tables = reinterpret_cast<DfTables*>(w + L.tables);
  uint32_t* first_bad = reinterpret_cast<uint32_t*>(w + L.first_bad);
  double* logf = logf_out ? logf_out : reinterpret_cast<double*>(w + L.logf);
  const uint32_t np = static_cast<uint32_t>(n_particles);
  cudaError_t e = cudaSuccess;
  if (logf_out) {
    // Steps after the one that ended a particle keep NaN.
    e = cudaMemsetAsync(logf_out, 0xFF, sizeof(double) * n_particles * T, s);
  }
  if (e == cudaSuccess) {
    bege_tables<<<1, 128, 0, s>>>(tables);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    bege_shapes<<<(np + 127) / 128, 128, 0, s>>>(theta, np, r, T, shape_p, shape_n, first_bad);
    e = cudaGetLastError();
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t n_tasks = n_particles * T;
  if (e == cudaSuccess) {
    const uint64_t want = (n_tasks + 255) / 256, cap = static_cast<uint64_t>(sms > 0 ? sms : 1) * 8;
    bege_tasks<<<static_cast<unsigned>(want < cap ? want : cap), 256, 0, s>>>(theta, np, r, T, h, shape_p, shape_n,
                                                                                first_bad, n_tasks, tasks);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const uint64_t per_cta = kBegeWarpsPerCta;
    uint64_t blocks = (n_tasks + per_cta - 1) / per_cta;
    const uint64_t cap = static_cast<uint64_t>(sms > 0 ? sms : 1) * 64;
    if (blocks > cap) blocks = cap;
    bege_density<<<static_cast<unsigned>(blocks), 32 * kBegeWarpsPerCta, 0, s>>>(np, T, 0.5 / h, tables, tasks,
                                                                                 first_bad, logf);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    bege_finish<<<np, 256, 0, s>>>(logf, T, first_bad, ll_out);
    e = cudaGetLastError();
  }
  return check_cuda(e, "bege_loglik");
}

}  // extern "C"
