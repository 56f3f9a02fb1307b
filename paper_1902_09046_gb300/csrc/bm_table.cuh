// bm_table.cuh -- table-driven Box-Muller for the OU path kernels.
//
// The transform is the one rng.cuh names (Sec. 3.4, the Box-Muller method of
// the paper's MKL calls): r = sqrt(-2 ln u1), (z0, z1) = r (cos 2 pi u2,
// sin 2 pi u2), on the generator's uniforms u = (m + 1/2) 2^-23.  Here both
// functions read tables from shared memory instead of evaluating
// polynomials, which moves most of their arithmetic off the FMA pipe that
// the Philox multiplies saturate:
//
//  * -2 ln u by Tang's table-driven method (ACM TOMS 16(4), 1990): u = 2^e f
//    with f in [3/4, 3/2), bucket j = the top 8 bits of f's field, r =
//    fma(f, c_j, -1) with |r| <= 2^-9, t = -2 r + r^2 (1 - 2r/3) for
//    -2 log1p(r), and -2 ln u = fma(e, K, A_j + t), where A_j = 2 ln c_j
//    (c_j chosen by Gal's accurate-table method so that A_j is within 2^-12
//    ulp of its binary32 value) and K = RN(-2 ln 2).  Within 0.95 ulp on all
//    2^23 inputs.
//  * (cos, sin)(2 pi u): m = 2^11 i + k, 2 pi u = a_i + b_k with a_i =
//    2 pi i / 4096 and b_k = 2 pi (k + 1/2) 2^-23, and
//      cos = C_i + fma(C_i, cm_k, -S_i s_k),  sin = S_i + fma(S_i, cm_k, C_i s_k)
//    with cm_k = cos b_k - 1.  Within 2^-24 absolute on all 2^23 inputs.
//  * sqrt by the hardware reciprocal square root and one Newton step
//    (rng.cuh's sqrt_pos).
//
// make_bm_tables.py writes the tables (bm_tables.h) and checks both bounds
// by emulating this arithmetic on every input.  The two-stream forms perform
// the scalar operations in the same order, on f32x2 pairs where both operands
// already sit in register pairs and per lane where they come from two table
// entries, so every lane is bit for bit the scalar result.
//
// Shared memory: the two angle tables (48 KB, read at random indices) and
// the log table, either compact (2 KB) or lane-replicated (16 copies
// interleaved entry by entry, 32 KB), where lane l reads copy l % 16: the 16
// lanes of a half-warp then hit 16 different bank pairs whatever their
// entries, and a 64-bit table read costs the minimum two wavefronts instead
// of about four and a half at random.  Kernels with short-lived CTAs read
// the compact layout from global memory instead (bm_tab_global).  All forms
// hold the same values.
#pragma once

#include <stdint.h>

#include "bm_tables.h"
#include "rng.cuh"

namespace ppabc {

constexpr size_t kBmScBytes = (static_cast<size_t>(kBmScHi) + kBmScLo) * sizeof(float2);

template <bool kRepLog>
constexpr size_t bm_smem_bytes() {
  return kBmScBytes + static_cast<size_t>(kBmLogBuckets) * sizeof(float2) * (kRepLog ? 16 : 1);
}

// The tables of one CTA in shared memory, as seen by one lane: the angle
// tables at fixed offsets from `base`, the log table after them, and this
// lane's copy of the log table (an OR into a 128-byte-aligned entry offset).
struct BmTab {
  const unsigned char* base;
  uint32_t lane8;  // 8 (lane % 16) for the replicated log table, 0 for the compact one
};

// Copies the tables into smem (16-byte aligned, bm_smem_bytes<kRepLog>()
// bytes) with all threads of the CTA; the caller synchronises before use.
template <bool kRepLog>
__device__ __forceinline__ void bm_load(unsigned char* smem) {
  const uint4* sc = reinterpret_cast<const uint4*>(kBmTablesBits);
  uint4* d = reinterpret_cast<uint4*>(smem);
  constexpr int nsc = (kBmScHi + kBmScLo) / 2;  // two float2 per uint4
  for (int t = threadIdx.x; t < nsc; t += blockDim.x) d[t] = sc[t];
  const uint2* lg = reinterpret_cast<const uint2*>(kBmTablesBits) + kBmScHi + kBmScLo;
  uint2* dl = reinterpret_cast<uint2*>(smem + kBmScBytes);
  if (kRepLog) {
    for (int t = threadIdx.x; t < kBmLogBuckets * 16; t += blockDim.x) dl[t] = lg[t >> 4];
  } else {
    for (int t = threadIdx.x; t < kBmLogBuckets; t += blockDim.x) dl[t] = lg[t];
  }
}

template <bool kRepLog>
__device__ __forceinline__ BmTab bm_tab(const unsigned char* smem) {
  BmTab T;
  T.base = smem;
  T.lane8 = kRepLog ? 8u * (threadIdx.x & 15u) : 0u;
  return T;
}

// The same tables read where the library keeps them in global memory (the
// compact layout, cached in L1): for kernels whose CTAs live too briefly, or
// are too small, to pay for a copy into shared memory.  Same values, so the
// same results bit for bit.
__device__ __forceinline__ BmTab bm_tab_global() {
  BmTab T;
  T.base = reinterpret_cast<const unsigned char*>(kBmTablesBits);
  T.lane8 = 0u;
  return T;
}

__device__ __forceinline__ float2 bm_ld2(const unsigned char* p) { return *reinterpret_cast<const float2*>(p); }

// Table entry (c_j, A_j) of the log bucket of bits Bp = bits(u) + 2^22,
// j = (Bp >> 15) & 255: entry j of this lane's copy, at 128 bytes per entry
// (replicated) or 8 (compact).
template <bool kRepLog>
__device__ __forceinline__ float2 bm_log_entry(const BmTab& T, uint32_t Bp) {
  const uint32_t off = kRepLog ? (((Bp >> 8) & 0x7F80u) | T.lane8) : ((Bp >> 12) & 0x7F8u);
  return bm_ld2(T.base + kBmScBytes + off);
}

// u = 2^e f split of the uniform of word w: returns the bits Bp of u + 2^22
// (exponent field and bucket) and sets f in [3/4, 3/2).
__device__ __forceinline__ uint32_t bm_log_split(uint32_t B, float& f) {
  const uint32_t Bp = B + 0x00400000u;
  f = __uint_as_float(B - (Bp & 0xFF800000u) + 0x3F800000u);
  return Bp;
}

// e as binary32 from Bp (exact): 2^23 + (e + 127) minus 2^23 + 127.
__device__ __forceinline__ float bm_log_e(uint32_t Bp) {
  return __uint_as_float((Bp >> 23) + 0x4B000000u) - 8388735.0f;
}

// -2 ln u(w).
template <bool kRepLog>
__device__ __forceinline__ float neg2_log_tab(const BmTab& T, uint32_t w) {
  const float u = u01f(w);
  float f;
  const uint32_t Bp = bm_log_split(__float_as_uint(u), f);
  const float ef = bm_log_e(Bp);
  const float2 cA = bm_log_entry<kRepLog>(T, Bp);
  const float r = fmaf(f, cA.x, -1.0f);
  const float q = fmaf(r, -0x1.555556p-1f, 1.0f);
  const float t = fmaf(r * q, r, -2.0f * r);
  return fmaf(ef, __uint_as_float(kBmLogK), cA.y + t);
}

// (sin, cos)(2 pi u(w)): C, S from entry w >> 20 of the 4096-entry table,
// cm, s from entry (w >> 9) & 2047 of the 2048-entry one.
__device__ __forceinline__ void sincos_2pi_tab(const BmTab& T, uint32_t w, float& s, float& c) {
  const float2 H = bm_ld2(T.base + ((w >> 17) & 0x7FF8u));
  const float2 L = bm_ld2(T.base + kBmScHi * sizeof(float2) + ((w >> 6) & 0x3FF8u));
  c = H.x + fmaf(H.x, L.x, -(H.y * L.y));
  s = H.y + fmaf(H.y, L.x, H.x * L.y);
}

// Scalar Box-Muller on one word pair.
template <bool kRepLog>
__device__ __forceinline__ void box_muller_tab(const BmTab& T, uint32_t w_even, uint32_t w_odd, float& z_even,
                                               float& z_odd) {
  const float r = sqrt_pos(neg2_log_tab<kRepLog>(T, w_even));
  float s, c;
  sincos_2pi_tab(T, w_odd, s, c);
  z_even = r * c;
  z_odd = r * s;
}

// neg2_log_tab on two words.  The arithmetic runs on packed pairs except
// where it takes table values: those two operations run per lane, because
// packing values read from two table entries would first need register moves
// on the FMA pipe.  Each lane is bit for bit neg2_log_tab.
template <bool kRepLog>
__device__ __forceinline__ float2 neg2_log_tab2(const BmTab& T, uint32_t wa, uint32_t wb) {
  const float2 u = add2(make_float2(__uint_as_float((wa >> 9) + 0x3F800000u),
                                    __uint_as_float((wb >> 9) + 0x3F800000u)),
                        splat2(-0x1.fffffep-1f));
  float fa, fb;
  const uint32_t Bpa = bm_log_split(__float_as_uint(u.x), fa);
  const uint32_t Bpb = bm_log_split(__float_as_uint(u.y), fb);
  const float2 ef = add2(make_float2(__uint_as_float((Bpa >> 23) + 0x4B000000u),
                                     __uint_as_float((Bpb >> 23) + 0x4B000000u)),
                         splat2(-8388735.0f));
  const float2 ca = bm_log_entry<kRepLog>(T, Bpa), cb = bm_log_entry<kRepLog>(T, Bpb);
  const float2 r = make_float2(fmaf(fa, ca.x, -1.0f), fmaf(fb, cb.x, -1.0f));
  const float2 q = fma2(r, splat2(-0x1.555556p-1f), splat2(1.0f));
  const float2 t = fma2(mul2(r, q), r, mul2(splat2(-2.0f), r));
  return fma2(ef, splat2(__uint_as_float(kBmLogK)), make_float2(ca.y + t.x, cb.y + t.y));
}

// The four normals of one counter block, the two radii side by side, the
// angles per lane (bit-identical to two box_muller_tab calls).
template <bool kRepLog>
__device__ __forceinline__ float4 tnormals_of(const BmTab& T, uint4 w) {
  const float2 r = sqrt_pos2(neg2_log_tab2<kRepLog>(T, w.x, w.z));
  float s0, c0, s1, c1;
  sincos_2pi_tab(T, w.y, s0, c0);
  sincos_2pi_tab(T, w.w, s1, c1);
  const float2 zc = mul2(r, make_float2(c0, c1)), zs = mul2(r, make_float2(s0, s1));
  return make_float4(zc.x, zs.x, zc.y, zs.y);
}

// scale * (the four normals of w), the scale applied to each radius.
template <bool kRepLog>
__device__ __forceinline__ float4 scaled_tnormals_of(const BmTab& T, uint4 w, float scale) {
  const float2 r = mul2(splat2(scale), sqrt_pos2(neg2_log_tab2<kRepLog>(T, w.x, w.z)));
  float s0, c0, s1, c1;
  sincos_2pi_tab(T, w.y, s0, c0);
  sincos_2pi_tab(T, w.w, s1, c1);
  const float2 zc = mul2(r, make_float2(c0, c1)), zs = mul2(r, make_float2(s0, s1));
  return make_float4(zc.x, zs.x, zc.y, zs.y);
}

// The four normals of blocks w0 and w1 of two streams, packed across the
// streams: z[l] = (normal l of w0, normal l of w1), each lane bit for bit
// tnormals_of of its stream.
template <bool kRepLog>
__device__ __forceinline__ void tnormals_x2(const BmTab& T, uint4 w0, uint4 w1, float2 z[4]) {
  const float2 rA = sqrt_pos2(neg2_log_tab2<kRepLog>(T, w0.x, w1.x));
  const float2 rB = sqrt_pos2(neg2_log_tab2<kRepLog>(T, w0.z, w1.z));
  float s0, c0, s1, c1, s2, c2, s3, c3;
  sincos_2pi_tab(T, w0.y, s0, c0);
  sincos_2pi_tab(T, w1.y, s1, c1);
  sincos_2pi_tab(T, w0.w, s2, c2);
  sincos_2pi_tab(T, w1.w, s3, c3);
  z[0] = mul2(rA, make_float2(c0, c1));
  z[1] = mul2(rA, make_float2(s0, s1));
  z[2] = mul2(rB, make_float2(c2, c3));
  z[3] = mul2(rB, make_float2(s2, s3));
}

// The four normals of blocks w0 and w1 of two streams, packed across the
// streams and scaled per stream: z[l] = (c.x normal l of w0, c.y normal l of
// w1), each lane bit for bit scaled_tnormals_of of its stream.
template <bool kRepLog>
__device__ __forceinline__ void scaled_tnormals_x2(const BmTab& T, uint4 w0, uint4 w1, float2 c, float2 z[4]) {
  const float2 rA = mul2(c, sqrt_pos2(neg2_log_tab2<kRepLog>(T, w0.x, w1.x)));
  const float2 rB = mul2(c, sqrt_pos2(neg2_log_tab2<kRepLog>(T, w0.z, w1.z)));
  float s0, c0, s1, c1, s2, c2, s3, c3;
  sincos_2pi_tab(T, w0.y, s0, c0);
  sincos_2pi_tab(T, w1.y, s1, c1);
  sincos_2pi_tab(T, w0.w, s2, c2);
  sincos_2pi_tab(T, w1.w, s3, c3);
  z[0] = mul2(rA, make_float2(c0, c1));
  z[1] = mul2(rA, make_float2(s0, s1));
  z[2] = mul2(rB, make_float2(c2, c3));
  z[3] = mul2(rB, make_float2(s2, s3));
}

}  // namespace ppabc
