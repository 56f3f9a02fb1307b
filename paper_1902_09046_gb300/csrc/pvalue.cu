// pvalue.cu -- prior-predictive p-value sweep with exact tail counts.
//
// For lambda index k and data set m (Sec. 4.1, Eq. 6 and Eq. 8, conjugate
// model y_i ~ N(mu, 1), mu ~ N(0, lambda_k^2)):
//   z_t = normal t of stream (seed, m, k, PATH), t = 0..n_obs,
//   ybar = lambda_k z_0 + (1/n_obs) sum_{t>=1} z_t,
//   counts[k] += [|ybar| >= |ybar_obs|].
// One thread walks a strided set of data sets of one lambda (blockIdx.y) and
// keeps its count in a register; a warp reduction and one 64-bit atomic per
// warp add it to counts[k].  The normals are binary32 and summed with Kahan
// compensation; ybar and the comparison are binary64 (a handful of binary64
// operations per data set, against 51 normals of binary32 work).
#include "internal.h"

namespace ppabc {

namespace {

constexpr int kPvThreads = 256;

__device__ __forceinline__ void kahan_add(float& s, float& comp, float x) {
  const float y = x - comp;
  const float t = s + y;
  comp = (t - s) - y;
  s = t;
}

template <bool kWantYbar>
__global__ void __launch_bounds__(kPvThreads) pvalue_tail(const double* __restrict__ lambda,
                                                          uint32_t n_obs, double inv_n,
                                                          uint32_t m_sets, uint32_t set_base,
                                                          double abs_ybar_obs,
                                                          uint32_t k0, uint32_t k1,
                                                          unsigned long long* __restrict__ counts,
                                                          double* __restrict__ ybar_out) {
  const uint32_t k = blockIdx.y;
  const double lam = lambda[k];
  const uint32_t n_full = (n_obs + 1) >> 2;  // counter blocks whose 4 normals are all used
  const uint32_t rem = (n_obs + 1) & 3u;     // normals used from the last block
  unsigned int count = 0;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kPvThreads;
  for (uint64_t m0 = static_cast<uint64_t>(blockIdx.x) * kPvThreads; m0 < m_sets; m0 += stride) {
    const uint64_t m = m0 + threadIdx.x;
    if (m < m_sets) {
      float z0 = 0.0f, s = 0.0f, comp = 0.0f;
      for (uint32_t b = 0; b < n_full; ++b) {
        const float4 z = block_normals(b, set_base + static_cast<uint32_t>(m), k, kTagPath, k0, k1);
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
        const float4 z = block_normals(n_full, set_base + static_cast<uint32_t>(m), k, kTagPath, k0, k1);
        if (n_full == 0) {
          z0 = z.x;
        } else {
          kahan_add(s, comp, z.x);
        }
        if (rem > 1) kahan_add(s, comp, z.y);
        if (rem > 2) kahan_add(s, comp, z.z);
      }
      const double sum = static_cast<double>(s) - static_cast<double>(comp);
      const double ybar = fma(lam, static_cast<double>(z0), sum * inv_n);
      if (kWantYbar) ybar_out[static_cast<size_t>(k) * m_sets + m] = ybar;
      count += (fabs(ybar) >= abs_ybar_obs) ? 1u : 0u;
    }
  }
  count = __reduce_add_sync(0xFFFFFFFFu, count);
  if ((threadIdx.x & 31) == 0 && count)
    atomicAdd(counts + k, static_cast<unsigned long long>(count));
}

__global__ void pvalue_finalize(const unsigned long long* counts, uint32_t n_lambda,
                                double m_sets, double* p_out) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n_lambda) p_out[k] = static_cast<double>(counts[k]) / m_sets;
}

}  // namespace

cudaError_t launch_pvalue(const double* lambda, uint32_t n_lambda, uint32_t n_obs,
                          uint32_t m_sets, uint32_t set_base, double ybar_obs, uint64_t seed,
                          uint64_t* counts, double* p_out, double* ybar_out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(uint64_t) * n_lambda, s);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  // About four waves of 8 resident CTAs per SM over the whole sweep.
  const uint64_t target = static_cast<uint64_t>(sms) * 8u * 4u;
  uint64_t bx = (target + n_lambda - 1) / n_lambda;
  const uint64_t need = (static_cast<uint64_t>(m_sets) + kPvThreads - 1) / kPvThreads;
  if (bx > need) bx = need;
  if (bx < 1) bx = 1;
  const dim3 grid(static_cast<unsigned>(bx), n_lambda);
  const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  const double inv_n = 1.0 / static_cast<double>(n_obs);
  const double a = fabs(ybar_obs);
  auto* c = reinterpret_cast<unsigned long long*>(counts);
  if (ybar_out)
    pvalue_tail<true><<<grid, kPvThreads, 0, s>>>(lambda, n_obs, inv_n, m_sets, set_base, a, k0, k1, c,
                                                   ybar_out);
  else
    pvalue_tail<false><<<grid, kPvThreads, 0, s>>>(lambda, n_obs, inv_n, m_sets, set_base, a, k0, k1, c,
                                                    ybar_out);
  e = cudaGetLastError();
  if (e != cudaSuccess || !p_out) return e;
  pvalue_finalize<<<(n_lambda + 127) / 128, 128, 0, s>>>(c, n_lambda, static_cast<double>(m_sets), p_out);
  return cudaGetLastError();
}

}  // namespace ppabc
