// ou_path.cuh -- one OU prior-predictive sample per thread, fused end to end.
//
// For global sample index g (Sec. 3.1, Eq. 2 and Algorithm 1 with N fixed):
//   theta ~ U(lo, hi)        counter (0, g, sub, PRIOR), words 0..2;
//   X_s = X_{s-1} + th1 dt (th2 - X_{s-1}) + th3 sqrt(dt) xi_{s-1}
//                            Euler-Maruyama (Eq. 5) on the OU SDE, with xi_j
//                            lane j%4 of counter block (j/4, g, sub, PATH);
//   acc += (X_{s_j} - y_j)^2 at the observation steps s_j;  rho = sqrt(acc).
//
// Precision: the state is binary32 with Kahan compensation (X - comp is the
// running value to about 2^-48 relative), the normals are binary32, and the
// residuals and their sum are binary64.  Uncompensated binary32 loses about
// sqrt(1 / (th1 dt)) ulps over a path, which at dt = 1e-3 is far above the
// 1e-6 relative band the accept sets are compared in.
//
// Nothing is read from or written to global memory inside the step loop: the
// Philox words, the normals and the state live in registers.
#pragma once

#include <stdint.h>

#include "../../include/ppabc.h"
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
  uint32_t key0, key1;
  uint32_t sub;
  uint32_t s_obs[PPABC_MAX_OBS];
  double y[PPABC_MAX_OBS];
};

// Prior draw of sample g: th_j = lo_j + span_j u(w_j).
__device__ __forceinline__ void ou_prior(const OUConst& P, uint32_t g, float& th1, float& th2,
                                         float& th3) {
  const uint4 w = philox4x32_10(make_uint4(0u, g, P.sub, kTagPrior), P.key0, P.key1);
  th1 = fmaf(P.span[0], u01f(w.x), P.lo[0]);
  th2 = fmaf(P.span[1], u01f(w.y), P.lo[1]);
  th3 = fmaf(P.span[2], u01f(w.z), P.lo[2]);
}

// One Euler-Maruyama step with a Kahan-compensated state:
// inc = k (th2 - X) + c xi, then X <- X + inc with the rounding error kept in comp.
__device__ __forceinline__ void em_step(float& X, float& comp, float k, float th2, float c,
                                        float xi) {
  const float inc = fmaf(k, th2 - X, c * xi);
  const float y = inc - comp;
  const float t = X + y;
  comp = (t - X) - y;
  X = t;
}

// Simulate sample g and return rho; the summaries go to summ[j * summ_stride]
// when summ is non-null.
template <bool kWantSumm>
__device__ __forceinline__ double ou_path(const OUConst& P, uint32_t g, float th1, float th2,
                                          float th3, double* summ, uint32_t summ_stride) {
  const float k = th1 * P.dt;
  const float c = th3 * P.sqrt_dt;
  const uint32_t S = P.n_steps;
  const uint32_t n_obs = P.n_obs;
  float X = P.x0;
  float comp = 0.0f;
  double acc = 0.0;
  uint32_t j = 0;
  uint32_t s_next = P.s_obs[0];
  uint32_t s = 0;  // steps taken
  for (uint32_t b = 0; s < S; ++b) {
    const float4 z = block_normals(b, g, P.sub, kTagPath, P.key0, P.key1);
    if (s + 4u < s_next) {
      // No observation among steps s+1 .. s+4 (uniform across the launch).
      em_step(X, comp, k, th2, c, z.x);
      em_step(X, comp, k, th2, c, z.y);
      em_step(X, comp, k, th2, c, z.z);
      em_step(X, comp, k, th2, c, z.w);
      s += 4u;
    } else {
      const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        if (s < S) {
          em_step(X, comp, k, th2, c, zz[l]);
          ++s;
          if (s == s_next) {
            const double x = static_cast<double>(X) - static_cast<double>(comp);
            const double r = x - P.y[j];
            acc = fma(r, r, acc);
            if (kWantSumm) summ[static_cast<size_t>(j) * summ_stride] = x;
            ++j;
            s_next = (j < n_obs) ? P.s_obs[j] : 0xFFFFFFFFu;
          }
        }
      }
    }
  }
  return sqrt(acc);
}

}  // namespace ppabc
