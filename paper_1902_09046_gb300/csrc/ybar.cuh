// ybar.cuh -- mean of one prior-predictive data set of the conjugate model.
//
// y_i ~ N(mu, 1), i = 1..n, mu ~ N(0, lambda^2): with z_t the normals of the
// data set's stream (lane t%4 of counter block t/4), mu = lambda z_0 and
// ybar = mu + (1/n) sum_{t=1..n} z_t.  The normals are binary32 and summed
// with Kahan compensation; ybar itself is binary64.
#pragma once

#include "rng.cuh"

namespace ppabc {

__device__ __forceinline__ void kahan_add(float& s, float& comp, float x) {
  const float y = x - comp;
  const float t = s + y;
  comp = (t - s) - y;
  s = t;
}

__device__ __forceinline__ double dataset_ybar(const PhiloxKeys& K, double lam, uint32_t n_obs,
                                               double inv_n, uint32_t c1, uint32_t c2,
                                               uint32_t tag) {
  const PhiloxStream S = philox_stream(K, c1, c2, tag);
  const uint32_t n_full = (n_obs + 1) >> 2;  // counter blocks whose 4 normals are all used
  const uint32_t rem = (n_obs + 1) & 3u;     // normals used from the last block
  float z0 = 0.0f, s = 0.0f, comp = 0.0f;
  for (uint32_t b = 0; b < n_full; ++b) {
    const float4 z = normals_of(philox_block(S, K, b));
    if (b == 0) {
      z0 = z.x;
    } else {
      kahan_add(s, comp, z.x);
    }
    kahan_add(s, comp, z.y);
    kahan_add(s, comp, z.z);
    kahan_add(s, comp, z.w);
  }
  if (rem) {
    const float4 z = normals_of(philox_block(S, K, n_full));
    if (n_full == 0) {
      z0 = z.x;
    } else {
      kahan_add(s, comp, z.x);
    }
    if (rem > 1) kahan_add(s, comp, z.y);
    if (rem > 2) kahan_add(s, comp, z.z);
  }
  const double sum = static_cast<double>(s) - static_cast<double>(comp);
  return fma(lam, static_cast<double>(z0), sum * inv_n);
}

}  // namespace ppabc
