// dfloat.cuh -- double-float arithmetic and its log and exp.
//
// A double-float value is hi + lo, two binary32 numbers with |lo| <= ulp(hi)/2
// (about 48 significant bits).  GB300 retires about one binary64 FMA per SM
// sub-partition every other clock, so a warp-wide binary64 instruction holds
// that pipe about 64 clocks, while the binary32 pipes take a warp instruction
// per clock: where 48 bits are enough, a double-float operation of four to
// ten binary32 instructions is far cheaper than one binary64 instruction.
//
// The error-free transformations are Knuth's two-sum, Dekker's fast two-sum
// and the FMA two-product.  Their additions and multiplications are written
// with the round-to-nearest intrinsics so that the compiler does not fuse a
// product into the following addition (which would change the rounding the
// transformations rely on).
#pragma once

#include <math.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define PPABC_DF_FN __host__ __device__ __forceinline__
#else
#define PPABC_DF_FN inline
#endif

namespace ppabc {

struct DF {
  float hi, lo;
};

PPABC_DF_FN float df_add_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}

PPABC_DF_FN float df_mul_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}

PPABC_DF_FN uint32_t df_bits(float x) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(x);
#else
  uint32_t u;
  __builtin_memcpy(&u, &x, 4);
  return u;
#endif
}

PPABC_DF_FN float df_from_bits(uint32_t u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float x;
  __builtin_memcpy(&x, &u, 4);
  return x;
#endif
}

// s + e = a + b exactly, for |a| >= |b| (or a = 0).
PPABC_DF_FN DF df_fast_two_sum(float a, float b) {
  const float s = df_add_rn(a, b);
  return DF{s, df_add_rn(b, -df_add_rn(s, -a))};
}

// s + e = a + b exactly.
PPABC_DF_FN DF df_two_sum(float a, float b) {
  const float s = df_add_rn(a, b);
  const float v = df_add_rn(s, -a);
  return DF{s, df_add_rn(df_add_rn(a, -df_add_rn(s, -v)), df_add_rn(b, -v))};
}

// p + e = a b exactly.
PPABC_DF_FN DF df_two_prod(float a, float b) {
  const float p = df_mul_rn(a, b);
  return DF{p, fmaf(a, b, -p)};
}

PPABC_DF_FN DF df_split(double x) {
  const float hi = static_cast<float>(x);
  return DF{hi, static_cast<float>(x - static_cast<double>(hi))};
}

PPABC_DF_FN double df_to_double(DF a) { return static_cast<double>(a.hi) + static_cast<double>(a.lo); }

PPABC_DF_FN DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

PPABC_DF_FN DF df_mul(DF a, DF b) {
  const float p = df_mul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}

// a b for a double-float a and a binary32 b.
PPABC_DF_FN DF df_mul_f(DF a, float b) {
  const float p = df_mul_rn(a.hi, b);
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  return df_fast_two_sum(p, e);
}

PPABC_DF_FN DF df_sqr(DF a) {
  const float p = df_mul_rn(a.hi, a.hi);
  float e = fmaf(a.hi, a.hi, -p);
  e = fmaf(df_add_rn(a.hi, a.hi), a.lo, e);
  return df_fast_two_sum(p, e);
}

PPABC_DF_FN DF df_add(DF a, DF b) {
  const DF s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, df_add_rn(s.lo, df_add_rn(a.lo, b.lo)));
}

// a + b for a double-float a and a binary32 b.
PPABC_DF_FN DF df_add_f(DF a, float b) {
  const DF s = df_two_sum(a.hi, b);
  return df_fast_two_sum(s.hi, df_add_rn(s.lo, a.lo));
}

// Tables of the double-float log and exp (filled once per CTA).
struct alignas(16) DfTables {
  float log_c[128];  // c_j = 1 / (1 + (j + 1/2) / 128), rounded to binary32
  DF log_l[128];     // -log(c_j) for that rounded c_j
  DF exp2j[64];      // 2^(j / 64)
};

// log(x) by the table-driven reduction of Tang (ACM TOMS 16, 1990) in
// double-float: x = 2^e m, m in [1, 2), j = the top seven bits of m's
// fraction, r = m c_j - 1 (|r| <= 2^-8), and
//   log x = e ln2 - log(c_j) + log1p(r),
//   log1p(r) = r - r^2 / 2 + r^3 (1/3 - r/4 + r^2/5 - r^3/6 + r^4/7),
// the first two terms in double-float, the rest (below 2^-25) in binary32.
// x.hi must be a positive normal binary32 number below 2^126.  Absolute error
// about 2^-47 (2^-48 from the binary32 tail, the rest from the additions).
PPABC_DF_FN DF df_log(DF x, const DfTables& T) {
  const uint32_t b = df_bits(x.hi);
  const int e = static_cast<int>(b >> 23) - 127;
  const int j = static_cast<int>((b >> 16) & 127u);
  const float sc = df_from_bits(static_cast<uint32_t>(127 - e) << 23);  // 2^-e
  const float mh = df_mul_rn(x.hi, sc), ml = df_mul_rn(x.lo, sc);      // exact
  const float c = T.log_c[j];
  const float ph = df_mul_rn(mh, c);
  const float pl = fmaf(ml, c, fmaf(mh, c, -ph));
  const DF r = df_two_sum(df_add_rn(ph, -1.0f), pl);  // ph - 1 is exact
  const float t = r.hi;
  const float poly = fmaf(fmaf(fmaf(fmaf(1.0f / 7.0f, t, -1.0f / 6.0f), t, 0.2f), t, -0.25f), t, 1.0f / 3.0f);
  const float c3 = df_mul_rn(df_mul_rn(df_mul_rn(t, t), t), poly);
  const DF r2 = df_sqr(r);
  DF L = df_add(r, DF{-0.5f * r2.hi, -0.5f * r2.lo});
  L = df_add_f(L, c3);
  L = df_add(L, T.log_l[j]);
  // e ln2 with ln2 = H + M + L3 (H has 16 significant bits, so e H is exact).
  const float ef = static_cast<float>(e);
  const DF eln2 = df_add_f(df_add(DF{df_mul_rn(ef, 0x1.62e4p-1f), 0.0f}, df_two_prod(ef, 0x1.7f7d1cp-20f)),
                           df_mul_rn(ef, 0x1.ef357ap-45f));
  return df_add(eln2, L);
}

// exp(y) = 2^m v with v in [1, 2) returned as a double-float and m through
// the reference, for y.hi >= -745 and below 709.7: n = round(64 y / ln2),
// r = y - n ln2/64 with ln2/64 = C1 + C2 + C3 (C1 = 0x1.64p-7 has 7
// significant bits, so n C1 is exact; C2 = -0x1.1bd01p-15, C3 =
// -0x1.718432p-41), and
//   v = 2^(j/64) (1 + r + r^2/2 + r^3 (1/6 + r/24 + r^2/120 + r^3/720)),
// n = 64 m + j.  Relative error about 2^-47, plus what y's own double-float
// rounding carries (up to ulp(y.hi) 2^-24 absolute: 2e-12 at |y| = 700).
PPABC_DF_FN DF df_exp_scaled(DF y, int& m, const DfTables& T) {
  const float nf = rintf(df_mul_rn(y.hi, 0x1.715476p+6f));
  const int n = static_cast<int>(nf);
  const float rh = df_add_rn(y.hi, -df_mul_rn(nf, 0x1.64p-7f));  // exact
  const DF p2 = df_two_prod(nf, 0x1.1bd01p-15f);                   // -n C2, exactly
  const DF s = df_two_sum(rh, p2.hi);
  const float corr = df_add_rn(df_add_rn(y.lo, p2.lo), df_mul_rn(nf, 0x1.718432p-41f));  // + y.lo - n C3
  const DF r = df_fast_two_sum(s.hi, df_add_rn(s.lo, corr));
  const float t = r.hi;
  const float poly = fmaf(fmaf(fmaf(1.0f / 720.0f, t, 1.0f / 120.0f), t, 1.0f / 24.0f), t, 1.0f / 6.0f);
  const float c3 = df_mul_rn(df_mul_rn(df_mul_rn(t, t), t), poly);
  const DF r2 = df_sqr(r);
  DF q = df_add(r, DF{0.5f * r2.hi, 0.5f * r2.lo});
  q = df_add_f(q, c3);
  const DF tj = T.exp2j[n & 63];
  m = n >> 6;  // arithmetic shift: floor(n / 64)
  return df_add(tj, df_mul(tj, q));
}

// 2^m d for a double d in [2^-30, 2^100) and m >= -1000 (a normal result),
// by adding m to the exponent field.
PPABC_DF_FN double df_ldexp_normal(double d, int m) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double(__double_as_longlong(d) + (static_cast<long long>(m) << 52));
#else
  long long u;
  __builtin_memcpy(&u, &d, 8);
  u += static_cast<long long>(m) << 52;
  double r;
  __builtin_memcpy(&r, &u, 8);
  return r;
#endif
}

}  // namespace ppabc
