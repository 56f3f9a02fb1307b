// ybar.cuh -- mean of one prior-predictive data set of the conjugate model.
//
// y_i ~ N(mu, 1), i = 1..n, mu ~ N(0, lambda^2): with z_t the normals of the
// data set's stream (lane t%4 of counter block t/4), mu = lambda z_0 and
// ybar = mu + (1/n) sum_{t=1..n} z_t.  The normals are binary32 and summed
// with Kahan compensation; ybar itself is binary64.
#pragma once

#include "bm_table.cuh"
#include "rng.cuh"

namespace ppabc {

// Two data sets at once (lane q = data set q, streams S0 and S1 of the same
// length): the normals come packed across the sets (normals_x2); the four
// normals of a counter block are summed pairwise and the block sums are
// added with Kahan compensation on packed binary32 pairs:
//   y = x - comp;  t = s + y;  comp = (t - s) - y;  s = t
// (x - y formed as fma(y, -1, x), which rounds identically), then
// ybar = lambda z_0 + (s - comp) / n in binary64.  kTable selects the
// table-driven Box-Muller of bm_table.cuh (tables in shared memory, T) or
// the polynomial one of rng.cuh (T unused).
__device__ __forceinline__ void kahan_add2(float2& s, float2& comp, float2 x) {
  const float2 y = fma2(comp, splat2(-1.0f), x);
  const float2 t = add2(s, y);
  comp = fma2(y, splat2(-1.0f), fma2(s, splat2(-1.0f), t));
  s = t;
}

template <bool kTable, bool kRepLog>
__device__ __forceinline__ void ybar_normals_x2(const BmTab& T, uint4 w0, uint4 w1, float2 z[4]) {
  if (kTable)
    tnormals_x2<kRepLog>(T, w0, w1, z);
  else
    normals_x2(w0, w1, z);
}

template <bool kTable, bool kRepLog>
__device__ __forceinline__ double2 dataset_ybar2(const BmTab& T, const PhiloxKeys& K, double lam, uint32_t n_obs,
                                                 double inv_n, uint32_t c1a, uint32_t c1b, uint32_t c2,
                                                 uint32_t tag) {
  const PhiloxFamily F = philox_family(K, tag, c2);
  const PhiloxStream S0 = philox_stream(K, F, c1a);
  const PhiloxStream S1 = philox_stream(K, F, c1b);
  const uint32_t n_full = (n_obs + 1) >> 2;
  const uint32_t rem = (n_obs + 1) & 3u;
  float2 z0 = splat2(0.0f), s = splat2(0.0f), comp = splat2(0.0f);
  float2 z[4];
  // A block's normals summed pairwise, then one compensated add; block 0
  // also holds z_0.  The loop over the other blocks is unrolled by 4 (3.7%
  // faster sweeps than the rolled loop with block 0 tested inside it).
  if (n_full > 0) {
    const PhiloxBlockPart U = philox_block_part(F, 0u);
    ybar_normals_x2<kTable, kRepLog>(T, philox_block(K, S0, U), philox_block(K, S1, U), z);
    z0 = z[0];
    kahan_add2(s, comp, add2(add2(z[1], z[2]), z[3]));
  }
#pragma unroll 4
  for (uint32_t b = 1; b < n_full; ++b) {
    const PhiloxBlockPart U = philox_block_part(F, b);
    ybar_normals_x2<kTable, kRepLog>(T, philox_block(K, S0, U), philox_block(K, S1, U), z);
    kahan_add2(s, comp, add2(add2(z[0], z[1]), add2(z[2], z[3])));
  }
  if (rem) {
    const PhiloxBlockPart U = philox_block_part(F, n_full);
    ybar_normals_x2<kTable, kRepLog>(T, philox_block(K, S0, U), philox_block(K, S1, U), z);
    if (n_full == 0) {
      z0 = z[0];
    } else {
      kahan_add2(s, comp, z[0]);
    }
    if (rem > 1) kahan_add2(s, comp, z[1]);
    if (rem > 2) kahan_add2(s, comp, z[2]);
  }
  const double sum0 = static_cast<double>(s.x) - static_cast<double>(comp.x);
  const double sum1 = static_cast<double>(s.y) - static_cast<double>(comp.y);
  return make_double2(fma(lam, static_cast<double>(z0.x), sum0 * inv_n),
                      fma(lam, static_cast<double>(z0.y), sum1 * inv_n));
}

}  // namespace ppabc
