// bege.cu -- BEGE log-likelihood of many parameter vectors on one return
// series (Sec. 4.3: the BEGE model, its shape recursion, Eq. BEGE_LL,
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
// Here three kernels split the work: the shape recursion (sequential in t,
// one thread per particle), the densities (one warp per (particle, t): the
// 101 grid nodes spread over the lanes, lgamma of the two shapes computed
// once per warp, the grid differences taken with shuffles), and a fixed-order
// reduction of log f over t per particle.  Everything is binary64: the
// central difference divides the rounding of F by 2h.  GB300 issues about two
// binary64 FMAs per SM per clock, so the series avoids divisions: its ratios
// come from a per-warp table of 1 / (shape + k) in shared memory.
#include "internal.h"

namespace ppabc {

namespace {

constexpr int kBegeNw = PPABC_BEGE_NW;  // grid intervals
constexpr int kBegeWarpsPerCta = 8;
constexpr double kGammaEps = 1e-17;
constexpr double kGammaTiny = 1e-300;
constexpr int kGammaMaxIter = 1000000;

inline size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

struct BegeLayout {
  size_t shape_p, shape_n, first_bad, logf, total;
  BegeLayout(uint64_t np, uint64_t T) {
    size_t o = 0;
    shape_p = o;
    o = align256(o + sizeof(double) * np * T);
    shape_n = o;
    o = align256(o + sizeof(double) * np * T);
    first_bad = o;
    o = align256(o + sizeof(uint32_t) * np);
    logf = o;
    o = align256(o + sizeof(double) * np * T);
    total = o;
  }
};

// Reciprocals 1 / (a + k), k < kRecip, of one shape (binary64, stored as
// double-float), shared by every node of a task: the series' ratio
// x / (a + k) becomes x * inv[k].
constexpr int kRecip = 256;

// Nodes with x0 > kTaylorEdge * delta (delta = h / sn) take the central
// difference of the negative-shock factor from its Taylor expansion, whose
// relative truncation is about (delta / x0)^4 <= 1e-12; nearer the edge of
// the support, where the density is not smooth on the scale of delta, both
// values are evaluated.
constexpr double kTaylorEdge = 1001.0;

// Double-float arithmetic (a value is hi + lo, two binary32 numbers with
// |lo| <= ulp(hi) / 2; about 48 significant bits): Knuth's two-sum, the
// FMA two-product and Dekker's normalisation.  GB300 retires about one
// binary64 FMA per sub-partition every other clock, so a warp-wide binary64
// instruction holds the pipe about 64 clocks, while the binary32 pipes take
// a warp instruction per clock: the series below runs in double-float.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return DF{s, b - (s - a)};
}

__device__ __forceinline__ DF df_split(double x) {
  const float hi = __double2float_rn(x);
  return DF{hi, __double2float_rn(x - static_cast<double>(hi))};
}

__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = a.hi + b.hi;
  const float v = s - a.hi;
  float e = (a.hi - (s - v)) + (b.hi - v);
  e += a.lo + b.lo;
  return df_fast_two_sum(s, e);
}

// 1 / d for a positive double-float d: the binary32 reciprocal of d.hi and
// one Newton step r + r (1 - d r), the residual formed in double-float
// (relative error about 2^-46).
__device__ __forceinline__ DF df_recip(DF d) {
  const float r = 1.0f / d.hi;
  const DF dr = df_mul(d, DF{r, 0.0f});
  const DF res = df_add(DF{1.0f, 0.0f}, DF{-dr.hi, -dr.lo});
  return df_fast_two_sum(r, r * res.hi);
}

// sum_{j>=0} x^j / (a (a+1) ... (a+j)) in double-float, ratios from the
// table inv[k] = 1 / (a + k) (binary64 beyond it), two terms per
// convergence check, stopping when a term falls below 2^-49 of the sum (the
// format's own precision).  All terms are positive; for x < a + 66 they stay
// below e^66 / a, inside the binary32 range.
__device__ double series_df(double a, double x, const DF* __restrict__ inv) {
  const DF xd = df_split(x);
  DF term = inv[0], sum = term;
  for (int k = 1; k < kGammaMaxIter; k += 2) {
    term = df_mul(term, df_mul(xd, k < kRecip ? inv[k] : df_split(1.0 / (a + static_cast<double>(k)))));
    sum = df_add(sum, term);
    term = df_mul(term, df_mul(xd, k + 1 < kRecip ? inv[k + 1] : df_split(1.0 / (a + static_cast<double>(k + 1)))));
    sum = df_add(sum, term);
    if (term.hi < sum.hi * 0x1p-49f || term.hi == 0.0f) break;
  }
  return static_cast<double>(sum.hi) + static_cast<double>(sum.lo);
}

// Binary64 exp and log by Tang's table-driven method (ACM TOMS 15, 1989, and
// 16, 1990).  Every evaluation of P(a, .) needs exp(-x + a ln x - lgamma(a))
// and every Taylor node a density, so these two functions are most of the
// kernel's binary64 work; with the tables they take about ten binary64
// instructions each.  Accuracy (checked on the CPU with exact FMA): exp within
// 2.2e-16 relative for x >= -708 (0 below, where the value is < 1e-307 and
// only ever added to sums of order one), log within 4.2e-16 absolute for
// positive normal x.
struct BegeTables {
  double exp2j[64];   // 2^(j/64)
  double log_c[128];  // 1 / (1 + j/128), rounded
  double log_l[128];  // -log(log_c[j])
};

constexpr double kLn2Over64Hi = 0x1.62e42p-7;  // ln2/64 with 32 trailing zero bits
constexpr double kLn2Over64Lo = 0x1.fdf473de6af28p-28;
constexpr double k64OverLn2 = 0x1.71547652b82fep+6;
constexpr double kLn2Hi = 0x1.62e42p-1;
constexpr double kLn2Lo = 0x1.fdf473de6af28p-22;

__device__ void bege_fill_tables(BegeTables& tab) {
  for (int i = threadIdx.x; i < 64; i += blockDim.x) tab.exp2j[i] = exp2(static_cast<double>(i) / 64.0);
  for (int i = threadIdx.x; i < 128; i += blockDim.x) {
    const double c = 1.0 / (1.0 + static_cast<double>(i) / 128.0);
    tab.log_c[i] = c;
    tab.log_l[i] = -log(c);
  }
}

// exp(x) = 2^m 2^(j/64) exp(r), n = 64 m + j = round(64 x / ln2),
// r = x - n ln2/64 (Cody-Waite, |r| <= ln2/128), exp(r) - 1 to degree 5.
__device__ __forceinline__ double exp_tab(double x, const BegeTables& tab) {
  if (!(x >= -708.0)) return x != x ? x : 0.0;
  if (x > 709.0) return __longlong_as_double(0x7FF0000000000000ll);
  const double n = rint(x * k64OverLn2);
  double r = fma(-n, kLn2Over64Hi, x);
  r = fma(-n, kLn2Over64Lo, r);
  double p = fma(fma(fma(fma(1.0 / 120.0, r, 1.0 / 24.0), r, 1.0 / 6.0), r, 0.5), r, 1.0);
  p *= r;
  const int ni = static_cast<int>(n);
  const double t = tab.exp2j[ni & 63];
  const double v = fma(t, p, t);
  return __longlong_as_double(__double_as_longlong(v) + (static_cast<long long>(ni >> 6) << 52));
}

// log(x) = e ln2 + log(1/c_j) + log1p(r) for x = 2^e m, m in [1, 2), j the
// top seven bits of m's fraction, r = m c_j - 1 (|r| < 2^-7), log1p to
// degree 6.  Positive normal x only; anything else takes the library log.
__device__ __forceinline__ double log_tab(double x, const BegeTables& tab) {
  if (!(x >= 0x1p-1022) || !(x < __longlong_as_double(0x7FF0000000000000ll))) return log(x);
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const int e = static_cast<int>((b >> 52) & 0x7FF) - 1023;
  const double m = __longlong_as_double(static_cast<long long>((b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull));
  const int j = static_cast<int>((b >> 45) & 127);
  const double r = fma(m, tab.log_c[j], -1.0);
  const double p = fma(fma(fma(fma(fma(-1.0 / 6.0, r, 1.0 / 5.0), r, -0.25), r, 1.0 / 3.0), r, -0.5), r, 1.0);
  const double q = fma(p, r, tab.log_l[j]);
  const double ed = static_cast<double>(e);
  return fma(ed, kLn2Hi, fma(ed, kLn2Lo, q));
}

// Where the GPU sums the series (below) rather than the continued fraction.
constexpr double kSeriesPastShape = 65.0;  // x < a + 1 + 65
constexpr double kSeriesMaxX = 600.0;      // partial sums stay far below overflow

// Regularised lower incomplete gamma P(a, x), a > 0, with lga = lgamma(a).
// The power series the paper names,
//   P = exp(-x + a ln x - lga) sum_j x^j / (a (a+1) ... (a+j)),
// converges for every x; past x ~ a its terms first grow (to about k = x - a)
// and then fall, so it needs about (x - a) + sqrt(78 x) terms.  On this GPU a
// term is two multiplies and an add (table ratios), against about thirty
// binary64 instructions (two divisions) per step of the continued fraction, so
// the series is used for every x < a + 1 and, past the shape, for x < a + 66
// while x < 600 (keeping the growing partial sums far from overflow), and
// Legendre's continued fraction for Q = 1 - P (modified Lentz) beyond.  Both
// give P to about 1e-14.  Where the tail bound
//   Q <= exp(-x + a ln x - lga) / (x + 1 - max(a, 1))     (x > a - 1)
// is below 2^-56, 1 - Q rounds to 1 whatever Q is, and 1 is returned.  Each
// loop is bounded by kGammaMaxIter terms.
__device__ double gammainc_p(double a, double lga, double x, const DF* __restrict__ inv, const BegeTables& tab) {
  if (!(x > 0.0)) return 0.0;
  const double lead = -x + a * log_tab(x, tab) - lga;
  const double e = exp_tab(lead, tab);
  if (x >= a + 1.0 && e < 0x1p-56 * (x + 1.0 - fmax(a, 1.0))) return 1.0;
  if (x < a + 1.0 || (x < a + 1.0 + kSeriesPastShape && x < kSeriesMaxX)) return series_df(a, x, inv) * e;
  double b = x + 1.0 - a;
  double c = 1.0 / kGammaTiny;
  double d = 1.0 / b;
  double h = d;
  for (int i = 1; i < kGammaMaxIter; ++i) {
    const double an = -i * (i - a);
    b += 2.0;
    d = fma(an, d, b);
    if (fabs(d) < kGammaTiny) d = kGammaTiny;
    c = b + an / c;
    if (fabs(c) < kGammaTiny) c = kGammaTiny;
    d = 1.0 / d;
    const double del = d * c;
    h *= del;
    if (fabs(del - 1.0) < kGammaEps) break;
  }
  return 1.0 - e * h;
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

// log f(u_t) for task (i, t) per warp.  Lane l owns grid nodes j = l + 32 k,
// k = 0..3 (j <= 100): it evaluates P(p, .) at w_j and, for j >= 1, the
// central difference over u +- h of the node's factor [1 - P(n, .)]; the
// difference P(p, w_j) - P(p, w_{j-1}) takes w_{j-1}'s value from the
// neighbouring lane.  F(u + h) - F(u - h) is accumulated as one sum of
// per-node differences: the same quantity as the two sums differenced,
// without their cancellation.  Away from the edge of the negative shock's
// support the node's difference comes from the Taylor expansion of P(n, .)
// about the node (one density instead of two series); within kTaylorEdge
// delta of the edge both values are evaluated.
__global__ void __launch_bounds__(32 * kBegeWarpsPerCta)
bege_density(const double* __restrict__ theta, uint32_t np, const double* __restrict__ r, uint32_t T,
             double h, const double* __restrict__ shape_p, const double* __restrict__ shape_n,
             const uint32_t* __restrict__ first_bad, double* __restrict__ logf) {
  __shared__ DF recip[kBegeWarpsPerCta][2][kRecip];
  __shared__ BegeTables tab;
  bege_fill_tables(tab);
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
    const double sp = theta[np + i], sn = theta[6ull * np + i], mu = theta[10ull * np + i];
    const double p = shape_p[task], n = shape_n[task];
    const double u = r[t] - mu;
    // lgamma of the two shapes, once per warp.
    const double lg_own = lgamma(lane == 0 ? p : n);
    const double lgp = __shfl_sync(0xFFFFFFFFu, lg_own, 0);
    const double lgn = __shfl_sync(0xFFFFFFFFu, lg_own, 1);
    const double w0 = 1e-4 - p * sp;
    const double dw = (10.0 * sp * sqrt(p) - w0) / static_cast<double>(kBegeNw - 1);
    const double psp = p * sp, nsn = n * sn;
    const double up = u + h, um = u - h;
    const double isp = 1.0 / sp, isn = 1.0 / sn;  // per task: nodes multiply
    const double delta = h * isn;
    // Each node's decision between the Taylor form and the two values, made
    // once: the n table is needed only where some node of the warp lies
    // within kTaylorEdge delta of the negative shock's support edge.
    double x0s[4];
    bool taylor[4];
    bool near_edge = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int j = static_cast<int>(lane) + 32 * k;
      x0s[k] = (w0 + static_cast<double>(j - 1) * dw - u + nsn) * isn;
      taylor[k] = x0s[k] > kTaylorEdge * delta;
      if (j >= 1 && j <= kBegeNw) near_edge |= !taylor[k];
    }
    const bool fill_n = __any_sync(0xFFFFFFFFu, near_edge);
    __syncwarp();  // the previous task's readers are done with the tables
    const DF p_df = df_split(p), n_df = df_split(n);
    for (int k = static_cast<int>(lane); k < kRecip; k += 32) {
      inv_p[k] = df_recip(df_add(p_df, DF{static_cast<float>(k), 0.0f}));
      if (fill_n) inv_n[k] = df_recip(df_add(n_df, DF{static_cast<float>(k), 0.0f}));
    }
    __syncwarp();
    double acc = 0.0;     // F(u + h) - F(u - h)
    double F_last = 0.0;  // F at node 32 k + 31 of the previous group (lane 31's value)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int j = static_cast<int>(lane) + 32 * k;
      const bool live = j <= kBegeNw;
      double F = 0.0;
      if (live) F = gammainc_p(p, lgp, (w0 + static_cast<double>(j) * dw + psp) * isp, inv_p, tab);
      double F_prev = __shfl_up_sync(0xFFFFFFFFu, F, 1);
      if (lane == 0) F_prev = F_last;
      F_last = __shfl_sync(0xFFFFFFFFu, F, 31);
      if (live && j >= 1) {
        // [1 - P(n, x0 - delta)] - [1 - P(n, x0 + delta)], x0 = (w_{j-1} - u + n sn) / sn.
        const double wjm1 = w0 + static_cast<double>(j - 1) * dw;
        const double x0 = x0s[k];
        double dG;
        if (taylor[k]) {
          // P(n, x0 + d) - P(n, x0 - d) = 2 d g + (d^3 / 3) g2 + O(d^5), with the
          // gamma density g = x^(n-1) e^-x / Gamma(n) and its second derivative
          // g2 = g [((n-1)/x - 1)^2 - (n-1)/x^2].
          const double g = exp_tab((n - 1.0) * log_tab(x0, tab) - x0 - lgn, tab);
          const double q = (n - 1.0) / x0;
          const double g2 = g * ((q - 1.0) * (q - 1.0) - q / x0);
          dG = 2.0 * delta * g + (delta * delta * delta / 3.0) * g2;
        } else {
          const double xp = (wjm1 - up + nsn) * isn;
          const double xm = (wjm1 - um + nsn) * isn;
          dG = (xm > 0.0 ? gammainc_p(n, lgn, xm, inv_n, tab) : 0.0) -
               (xp > 0.0 ? gammainc_p(n, lgn, xp, inv_n, tab) : 0.0);
        }
        acc += dG * (F - F_prev);
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
    if (lane == 0) {
      const double f = acc / (2.0 * h);
      logf[task] = (f > 0.0 && isfinite(f)) ? log(f) : -INFINITY;
    }
  }
}

// ll_i = sum_{t < T} log f, fixed-order tree per particle; -inf if a step
// was invalid or a density was not positive.
__global__ void __launch_bounds__(256) bege_reduce(const double* __restrict__ logf, uint32_t T,
                                                   const uint32_t* __restrict__ first_bad,
                                                   double* __restrict__ ll) {
  __shared__ double part[256];
  const uint32_t i = blockIdx.x;
  if (first_bad[i] < T) {
    if (threadIdx.x == 0) ll[i] = -INFINITY;
    return;
  }
  double s = 0.0;
  for (uint32_t t = threadIdx.x; t < T; t += 256) s += logf[static_cast<size_t>(i) * T + t];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < static_cast<unsigned>(w)) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) ll[i] = part[0] != part[0] ? -INFINITY : part[0];
}

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
  uint32_t* first_bad = reinterpret_cast<uint32_t*>(w + L.first_bad);
  double* logf = logf_out ? logf_out : reinterpret_cast<double*>(w + L.logf);
  const uint32_t np = static_cast<uint32_t>(n_particles);
  cudaError_t e = cudaSuccess;
  if (logf_out) {
    // Steps after the one that ended a particle keep NaN.
    e = cudaMemsetAsync(logf_out, 0xFF, sizeof(double) * n_particles * T, s);
  }
  if (e == cudaSuccess) {
    bege_shapes<<<(np + 127) / 128, 128, 0, s>>>(theta, np, r, T, shape_p, shape_n, first_bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t tasks = n_particles * T;
    const uint64_t per_cta = kBegeWarpsPerCta;
    uint64_t blocks = (tasks + per_cta - 1) / per_cta;
    const uint64_t cap = static_cast<uint64_t>(sms > 0 ? sms : 1) * 64;
    if (blocks > cap) blocks = cap;
    bege_density<<<static_cast<unsigned>(blocks), 32 * kBegeWarpsPerCta, 0, s>>>(
        theta, np, r, T, h, shape_p, shape_n, first_bad, logf);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    bege_reduce<<<np, 256, 0, s>>>(logf, T, first_bad, ll_out);
    e = cudaGetLastError();
  }
  return check_cuda(e, "bege_loglik");
}

}  // extern "C"
