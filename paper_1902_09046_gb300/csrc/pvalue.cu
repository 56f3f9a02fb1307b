// pvalue.cu -- prior-predictive p-value sweep with exact tail counts.
//
// For lambda index k and data set m (Sec. 4.1, Eq. 6 and Eq. 8, conjugate
// model y_i ~ N(mu, 1), mu ~ N(0, lambda_k^2)):
//   z_t = normal t of stream (seed, m, k, PATH), t = 0..n_obs,
//   ybar = lambda_k z_0 + (1/n_obs) sum_{t>=1} z_t,
//   counts[k] += [|ybar| >= |ybar_obs|].
// One thread walks a strided set of data-set pairs of one lambda (blockIdx.y)
// and keeps its count in a register; a warp reduction and one 64-bit atomic per
// warp add it to counts[k].  ybar comes from dataset_ybar2 (binary32 normals
// from the table-driven Box-Muller, Kahan-compensated sum, binary64 ybar);
// the comparison is binary64.  512-thread CTAs, two per SM, hold the
// Box-Muller tables (80 KB) in shared memory.
#include <atomic>

#include "internal.h"
#include "ybar.cuh"

namespace ppabc {

namespace {

constexpr int kPvThreads = 512;
constexpr size_t kPvSmem = bm_smem_bytes<true>();

template <bool kWantYbar>
__global__ void __launch_bounds__(kPvThreads, 2) pvalue_tail(const double* __restrict__ lambda,
                                                          uint32_t n_obs, double inv_n,
                                                          uint32_t m_sets, uint32_t set_base,
                                                          double abs_ybar_obs,
                                                          const __grid_constant__ PhiloxKeys K,
                                                          unsigned long long* __restrict__ counts,
                                                          double* __restrict__ ybar_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  bm_load<true>(smem);
  __syncthreads();
  const BmTab T = bm_tab<true>(smem);
  const uint32_t k = blockIdx.y;
  const double lam = lambda[k];
  unsigned int count = 0;
  // Each thread takes data sets m and m + kPvThreads of a 2 kPvThreads chunk,
  // evaluated together (dataset_ybar2); past the end the second lane repeats
  // the first and is not counted.
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * (2 * kPvThreads);
  for (uint64_t m0 = static_cast<uint64_t>(blockIdx.x) * (2 * kPvThreads); m0 < m_sets; m0 += stride) {
    const uint64_t ma = m0 + threadIdx.x;
    const uint64_t mb = ma + kPvThreads;
    if (ma < m_sets) {
      const uint64_t mb_eff = mb < m_sets ? mb : ma;
      const double2 yb = dataset_ybar2<true, true>(T, K, lam, n_obs, inv_n, set_base + static_cast<uint32_t>(ma),
                                                   set_base + static_cast<uint32_t>(mb_eff), k, kTagPath);
      if (kWantYbar) ybar_out[static_cast<size_t>(k) * m_sets + ma] = yb.x;
      count += (fabs(yb.x) >= abs_ybar_obs) ? 1u : 0u;
      if (mb < m_sets) {
        if (kWantYbar) ybar_out[static_cast<size_t>(k) * m_sets + mb] = yb.y;
        count += (fabs(yb.y) >= abs_ybar_obs) ? 1u : 0u;
      }
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
  static std::atomic<unsigned long long> ready{0ull};
  int dev0 = 0;
  cudaError_t e = cudaGetDevice(&dev0);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev0 < 64 ? (1ull << dev0) : 0ull;
  if (!bit || !(ready.load(std::memory_order_acquire) & bit)) {
    e = cudaFuncSetAttribute(pvalue_tail<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kPvSmem));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(pvalue_tail<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(kPvSmem));
    if (e != cudaSuccess) return e;
    if (bit) ready.fetch_or(bit, std::memory_order_acq_rel);
  }
  e = cudaMemsetAsync(counts, 0, sizeof(uint64_t) * n_lambda, s);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  // About four waves of 2 resident CTAs per SM over the whole sweep.
  const uint64_t target = static_cast<uint64_t>(sms) * 2u * 4u;
  uint64_t bx = (target + n_lambda - 1) / n_lambda;
  const uint64_t need = (static_cast<uint64_t>(m_sets) + 2 * kPvThreads - 1) / (2 * kPvThreads);
  if (bx > need) bx = need;
  if (bx < 1) bx = 1;
  const dim3 grid(static_cast<unsigned>(bx), n_lambda);
  const PhiloxKeys K = philox_keys(seed);
  const double inv_n = 1.0 / static_cast<double>(n_obs);
  const double a = fabs(ybar_obs);
  auto* c = reinterpret_cast<unsigned long long*>(counts);
  if (ybar_out)
    pvalue_tail<true><<<grid, kPvThreads, kPvSmem, s>>>(lambda, n_obs, inv_n, m_sets, set_base, a, K, c,
                                                         ybar_out);
  else
    pvalue_tail<false><<<grid, kPvThreads, kPvSmem, s>>>(lambda, n_obs, inv_n, m_sets, set_base, a, K, c,
                                                          ybar_out);
  e = cudaGetLastError();
  if (e != cudaSuccess || !p_out) return e;
  pvalue_finalize<<<(n_lambda + 127) / 128, 128, 0, s>>>(c, n_lambda, static_cast<double>(m_sets), p_out);
  return cudaGetLastError();
}

}  // namespace ppabc
