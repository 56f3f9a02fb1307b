// ou_path.cuh -- one OU prior-predictive sample per thread, fused end to end.
//
// For global sample index g (Sec. 3.1, Eq. 2 and Algorithm 1 with N fixed):
//   theta ~ U(lo, hi)        counter (PRIOR, 0, sub, g), words 0..2;
//   X_s = X_{s-1} + th1 dt (th2 - X_{s-1}) + th3 sqrt(dt) xi_{s-1}
//                            Euler-Maruyama (Eq. 5) on the OU SDE, with xi_j
//                            lane j%4 of counter (PATH, j/4, sub, g);
//   acc += (X_{s_j} - y_j)^2 at the observation steps s_j;  rho = sqrt(acc).
//
// Precision: the state is binary32 with Kahan compensation (X - comp is the
// running value to about 2^-48 relative), the normals are binary32, and the
// residuals and their sum are binary64.  Uncompensated binary32 loses about
// sqrt(1 / (th1 dt)) ulps over a path, which at dt = 1e-3 is far above the
// 1e-6 relative band the accept sets are compared in.
//
// Nothing is read from or written to global memory inside the step loop: the
// Philox words, the normals and the state live in registers, and the
// Box-Muller tables (bm_table.cuh) in shared memory.
#pragma once

#include <stdint.h>

#include "../../include/ppabc.h"
#include "bm_table.cuh"
#include "rng.cuh"

namespace ppabc {

// Launch-invariant constants of one OU job (binary32 prior box and step
// constants, observation steps, observed summaries, Philox key).
struct OUConst {
  float lo[3];
  float span[3];  // hi - lo
  float dt;
  float sqrt_dt;
  float x0;
  uint32_t n_steps;
  uint32_t n_obs;
  uint32_t sub;
  PhiloxKeys keys;
  uint32_t s_obs[PPABC_MAX_OBS];
  double y[PPABC_MAX_OBS];
};

// Prior draw of sample g: th_j = lo_j + span_j u(w_j).
__device__ __forceinline__ void ou_prior(const OUConst& P, uint32_t g, float& th1, float& th2,
                                         float& th3) {
  const uint4 w = philox4x32_10(make_uint4(kTagPrior, 0u, P.sub, g), P.keys);
  th1 = fmaf(P.span[0], u01f(w.x), P.lo[0]);
  th2 = fmaf(P.span[1], u01f(w.y), P.lo[1]);
  th3 = fmaf(P.span[2], u01f(w.z), P.lo[2]);
}

// One Euler-Maruyama step on the centred state Y = X - th2 with Kahan
// compensation: Y <- Y - k Y + c xi, with c xi already folded into `cz`;
// Y - comp is the running value and comp holds the rounding error.
__device__ __forceinline__ void em_step(float& Y, float& comp, float k, float cz) {
  const float y = fmaf(-k, Y, cz) - comp;
  const float t = Y + y;
  comp = (t - Y) - y;
  Y = t;
}

// Four Euler-Maruyama steps at once, for blocks with no observation inside:
// the recursion is linear, Y_4 = a^4 Y_0 + a^3 cz_0 + a^2 cz_1 + a cz_2 + cz_3
// with a = 1 - k, so one compensated update carries
//   inc = -K4 Y + ((a cz_0 + cz_1) a + cz_2) a + cz_3,   K4 = 1 - a^4,
// where K4 comes from binary64 (a^4 itself is too close to 1 to carry the
// mean reversion in binary32).  Same mathematics as four em_step calls, with
// one rounding of the state instead of four.
//
// Runs of whole blocks are taken two blocks (eight steps) at a time, with
//   inc = -K8 Y + (..((a cz_0 + cz_1) a + cz_2) a + .. ) a + cz_7,  K8 = 1 - a^8,
// and an odd last block of a run alone; every kernel groups the blocks of a
// run the same way, so their results stay bit-identical.
struct Em4 {
  float a;   // 1 - k, binary32
  float K4;  // 1 - a^4 from binary64
  float K8;  // 1 - a^8 from binary64
};

__device__ __forceinline__ Em4 em4_constants(float k) {
  const double ad = 1.0 - static_cast<double>(k);
  const double a2 = ad * ad;
  const double a4 = a2 * a2;
  Em4 E;
  E.a = static_cast<float>(ad);
  E.K4 = static_cast<float>(1.0 - a4);
  E.K8 = static_cast<float>(1.0 - a4 * a4);
  return E;
}

__device__ __forceinline__ void em_block4(float& Y, float& comp, const Em4& E, float4 cz) {
  const float s4 = fmaf(fmaf(fmaf(E.a, cz.x, cz.y), E.a, cz.z), E.a, cz.w);
  const float y = fmaf(-E.K4, Y, s4) - comp;
  const float t = Y + y;
  comp = (t - Y) - y;
  Y = t;
}

// Two consecutive blocks (eight steps) as one compensated update.
__device__ __forceinline__ void em_block8(float& Y, float& comp, const Em4& E, float4 c0, float4 c1) {
  float s8 = fmaf(fmaf(fmaf(E.a, c0.x, c0.y), E.a, c0.z), E.a, c0.w);
  s8 = fmaf(fmaf(fmaf(fmaf(s8, E.a, c1.x), E.a, c1.y), E.a, c1.z), E.a, c1.w);
  const float y = fmaf(-E.K8, Y, s8) - comp;
  const float t = Y + y;
  comp = (t - Y) - y;
  Y = t;
}

// em_block4 on two samples at once (lane q is sample q), with the same
// operations in the same order: each lane is bit for bit em_block4's result.
// x - y is formed as fma(y, -1, x), which rounds identically.
__device__ __forceinline__ void em_block4_2(float2& Y, float2& comp, float2 a, float2 negK4, const float2 z[4]) {
  const float2 s4 = fma2(fma2(fma2(a, z[0], z[1]), a, z[2]), a, z[3]);
  const float2 y = fma2(comp, splat2(-1.0f), fma2(negK4, Y, s4));
  const float2 t = add2(Y, y);
  comp = fma2(y, splat2(-1.0f), fma2(Y, splat2(-1.0f), t));
  Y = t;
}

// em_block8 on two samples at once, the same operations in the same order.
__device__ __forceinline__ void em_block8_2(float2& Y, float2& comp, float2 a, float2 negK8, const float2 z0[4],
                                            const float2 z1[4]) {
  float2 s8 = fma2(fma2(fma2(a, z0[0], z0[1]), a, z0[2]), a, z0[3]);
  s8 = fma2(fma2(fma2(fma2(s8, a, z1[0]), a, z1[1]), a, z1[2]), a, z1[3]);
  const float2 y = fma2(comp, splat2(-1.0f), fma2(negK8, Y, s8));
  const float2 t = add2(Y, y);
  comp = fma2(y, splat2(-1.0f), fma2(Y, splat2(-1.0f), t));
  Y = t;
}

// Simulate sample g and return rho; the summaries go to summ[j * summ_stride]
// when summ is non-null.  X_s = th2 + Y_s with Y_0 = x0 - th2 split exactly
// into (Y, -comp); observation steps are handled between runs of whole
// 4-step counter blocks, which take no per-step test.
template <bool kWantSumm, bool kRepLog>
__device__ __forceinline__ double ou_path(const OUConst& P, const BmTab& T, uint32_t g, float th1, float th2,
                                          float th3, double* summ, uint32_t summ_stride) {
  const float k = th1 * P.dt;
  const float c = th3 * P.sqrt_dt;
  const uint32_t S = P.n_steps;
  const uint32_t n_obs = P.n_obs;
  // Y0 = x0 - th2 exactly as Y - comp (Knuth's two-sum).
  float Y = P.x0 - th2;
  float comp;
  {
    const float bb = Y - P.x0;
    const float err = (P.x0 - (Y - bb)) + (-th2 - bb);
    comp = -err;
  }
  const double th2d = static_cast<double>(th2);
  double acc = 0.0;
  const Em4 E4 = em4_constants(k);
  const PhiloxFamily fam = philox_family(P.keys, kTagPath, P.sub);
  const PhiloxStream stream = philox_stream(P.keys, fam, g);
  uint32_t s = 0;  // steps taken (4 b except inside the last block)
  uint32_t b = 0;  // next counter block
  uint32_t j = 0;  // next observation
  while (j < n_obs) {
    uint32_t s_next = P.s_obs[j];  // > s
    // Whole blocks (steps s+1 .. s+4) that end before the observation step;
    // the count is the same for every thread of a launch.
    const uint32_t b_end = b + (s_next > s + 4u ? (s_next - s - 1u) >> 2 : 0u);
    s += (b_end - b) << 2;
#pragma unroll 2
    for (; b + 1 < b_end; b += 2) {
      const float4 z0 = scaled_tnormals_of<kRepLog>(T, philox_block(P.keys, fam, stream, b), c);
      const float4 z1 = scaled_tnormals_of<kRepLog>(T, philox_block(P.keys, fam, stream, b + 1), c);
      em_block8(Y, comp, E4, z0, z1);
    }
    if (b < b_end) {
      em_block4(Y, comp, E4, scaled_tnormals_of<kRepLog>(T, philox_block(P.keys, fam, stream, b), c));
      ++b;
    }
    // The block holding step s_next (and possibly later observation steps).
    const float4 z = scaled_tnormals_of<kRepLog>(T, philox_block(P.keys, fam, stream, b), c);
    ++b;
    const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      if (s < S) {
        em_step(Y, comp, k, zz[l]);
        ++s;
        if (s == s_next) {
          const double x = th2d + (static_cast<double>(Y) - static_cast<double>(comp));
          const double r = x - P.y[j];
          acc = fma(r, r, acc);
          if (kWantSumm) summ[static_cast<size_t>(j) * summ_stride] = x;
          ++j;
          s_next = (j < n_obs) ? P.s_obs[j] : 0xFFFFFFFFu;
        }
      }
    }
  }
  return sqrt(acc);
}

// Two samples per thread, interleaved step by step: the same arithmetic as
// ou_path on each sample (bit-identical results), with two independent
// dependency chains so a warp has work for the FP32 pipes while the other
// chain's Philox wide multiplies occupy the integer multiplier.  Both samples
// share the launch's step count and observation steps, so the control flow
// is the same as for one sample.
template <bool kWantSumm, bool kRepLog>
__device__ __forceinline__ void ou_path2(const OUConst& P, const BmTab& T, const uint32_t g[2], const float th1[2],
                                         const float th2[2], const float th3[2], double* summ0,
                                         double* summ1, uint32_t summ_stride, double out[2]) {
  float k[2], Y0[2], comp0[2];
  double th2d[2], acc[2];
  const PhiloxFamily fam = philox_family(P.keys, kTagPath, P.sub);
  PhiloxStream stream[2];
  Em4 E4[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    k[q] = th1[q] * P.dt;
    Y0[q] = P.x0 - th2[q];
    const float bb = Y0[q] - P.x0;
    const float err = (P.x0 - (Y0[q] - bb)) + (-th2[q] - bb);
    comp0[q] = -err;
    th2d[q] = static_cast<double>(th2[q]);
    acc[q] = 0.0;
    stream[q] = philox_stream(P.keys, fam, g[q]);
    E4[q] = em4_constants(k[q]);
  }
  const float2 c = make_float2(th3[0] * P.sqrt_dt, th3[1] * P.sqrt_dt);
  const float2 a2 = make_float2(E4[0].a, E4[1].a);
  const float2 negK4 = make_float2(-E4[0].K4, -E4[1].K4);
  const float2 negK8 = make_float2(-E4[0].K8, -E4[1].K8);
  float2 Y = make_float2(Y0[0], Y0[1]), comp = make_float2(comp0[0], comp0[1]);
  const uint32_t S = P.n_steps;
  const uint32_t n_obs = P.n_obs;
  uint32_t s = 0, b = 0, j = 0;
  while (j < n_obs) {
    uint32_t s_next = P.s_obs[j];
    const uint32_t b_end = b + (s_next > s + 4u ? (s_next - s - 1u) >> 2 : 0u);
    s += (b_end - b) << 2;
    // Unrolled by 4: without it the schedule of this loop swings by 7% with
    // unrelated changes (such as adding a sample offset to the index).
#pragma unroll 4
    for (; b + 1 < b_end; b += 2) {
      float2 z0[4], z1[4];
      const PhiloxBlockPart U0 = philox_block_part(fam, b);  // shared by both streams
      scaled_tnormals_x2<kRepLog>(T, philox_block(P.keys, stream[0], U0), philox_block(P.keys, stream[1], U0), c, z0);
      const PhiloxBlockPart U1 = philox_block_part(fam, b + 1);
      scaled_tnormals_x2<kRepLog>(T, philox_block(P.keys, stream[0], U1), philox_block(P.keys, stream[1], U1), c, z1);
      em_block8_2(Y, comp, a2, negK8, z0, z1);
    }
    if (b < b_end) {
      float2 z[4];
      const PhiloxBlockPart U = philox_block_part(fam, b);
      scaled_tnormals_x2<kRepLog>(T, philox_block(P.keys, stream[0], U), philox_block(P.keys, stream[1], U), c, z);
      em_block4_2(Y, comp, a2, negK4, z);
      ++b;
    }
    float2 z[4];
    const PhiloxBlockPart U = philox_block_part(fam, b);
    scaled_tnormals_x2<kRepLog>(T, philox_block(P.keys, stream[0], U), philox_block(P.keys, stream[1], U), c, z);
    ++b;
    float Ys[2] = {Y.x, Y.y}, Cs[2] = {comp.x, comp.y};
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      if (s < S) {
        em_step(Ys[0], Cs[0], k[0], z[l].x);
        em_step(Ys[1], Cs[1], k[1], z[l].y);
        ++s;
        if (s == s_next) {
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const double x = th2d[q] + (static_cast<double>(Ys[q]) - static_cast<double>(Cs[q]));
            const double r = x - P.y[j];
            acc[q] = fma(r, r, acc[q]);
            if (kWantSumm) (q ? summ1 : summ0)[static_cast<size_t>(j) * summ_stride] = x;
          }
          ++j;
          s_next = (j < n_obs) ? P.s_obs[j] : 0xFFFFFFFFu;
        }
      }
    }
    Y = make_float2(Ys[0], Ys[1]);
    comp = make_float2(Cs[0], Cs[1]);
  }
  out[0] = sqrt(acc[0]);
  out[1] = sqrt(acc[1]);
}

}  // namespace ppabc
