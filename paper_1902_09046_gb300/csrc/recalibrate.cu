// recalibrate.cu -- ABC recalibration of an accepted sample (the
// post-processing the paper's Discussion, Sec. 5, proposes to accelerate).
//
// Every accepted theta_a is recalibrated with a further ABC posterior built
// from all stored prior-predictive pairs (theta_j, S_j), taking its own
// simulated summaries S_a as the observation: the k pairs nearest to S_a
// give the marginal distribution functions at theta_a,
//   u_d = #{neighbours j : theta_j,d <= theta_a,d} / k,
// and the recalibrated value is the u_d-quantile of the accepted sample's own
// marginal (the ABC posterior given the real observation).
//
// Per accepted sample the GPU forms the n binary64 distances (summaries are
// [n_obs][n], so a warp reads consecutive pairs), selects the k nearest
// exactly with the abc_select kernels (ties to the smaller index), and counts
// u; a last kernel sorts each accepted marginal in shared memory and maps
// every u to its quantile.  Work is O(q n) -- meant for n up to ~10^6 and q
// up to a few thousand.
#include <algorithm>

#include "internal.h"

namespace ppabc {

namespace {

inline size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

struct RcLayout {
  size_t dist, idx, rec, nacc, select, total;
  RcLayout(uint64_t n, uint64_t k) {
    size_t o = 0;
    dist = o;
    o = align256(o + sizeof(double) * n);
    idx = o;
    o = align256(o + sizeof(uint32_t) * k);
    rec = o;
    o = align256(o + 16 * k);
    nacc = o;
    o = align256(o + sizeof(unsigned long long));
    select = o;
    o = align256(o + select_workspace_bytes(n));
    total = o;
  }
};

__global__ void summary_distance(const double* __restrict__ summ, uint32_t n, uint32_t n_obs,
                                 const uint32_t* __restrict__ acc, uint32_t i,
                                 double* __restrict__ dist) {
  const uint32_t a = acc[i];
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t j = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += stride) {
    if (a >= n) {  // invalid accepted index: NaN distances, NaN u
      dist[j] = __longlong_as_double(0x7FF8000000000000ll);
      continue;
    }
    double s = 0.0;
    for (uint32_t m = 0; m < n_obs; ++m) {
      const double r = summ[static_cast<size_t>(m) * n + j] - __ldg(summ + static_cast<size_t>(m) * n + a);
      s = fma(r, r, s);
    }
    dist[j] = sqrt(s);
  }
}

// u for accepted i from the neighbours' theta (columns 0..2 of the records).
__global__ void recal_u(const float4* __restrict__ rec_nn, uint32_t k, const float* __restrict__ theta,
                        uint32_t n, const uint32_t* __restrict__ acc, uint32_t i, uint32_t q,
                        double* __restrict__ u_out) {
  __shared__ unsigned int cnt[3];
  if (threadIdx.x < 3) cnt[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t a = acc[i];
  if (a >= n) {
    if (threadIdx.x < 3) u_out[static_cast<size_t>(threadIdx.x) * q + i] = __longlong_as_double(0x7FF8000000000000ll);
    return;
  }
  const float t0 = theta[a], t1 = theta[static_cast<size_t>(n) + a], t2 = theta[2 * static_cast<size_t>(n) + a];
  unsigned int c0 = 0, c1 = 0, c2 = 0;
  for (uint32_t t = threadIdx.x; t < k; t += blockDim.x) {
    const float4 r = rec_nn[t];
    c0 += r.x <= t0;
    c1 += r.y <= t1;
    c2 += r.z <= t2;
  }
  c0 = __reduce_add_sync(0xFFFFFFFFu, c0);
  c1 = __reduce_add_sync(0xFFFFFFFFu, c1);
  c2 = __reduce_add_sync(0xFFFFFFFFu, c2);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&cnt[0], c0);
    atomicAdd(&cnt[1], c1);
    atomicAdd(&cnt[2], c2);
  }
  __syncthreads();
  if (threadIdx.x < 3) u_out[static_cast<size_t>(threadIdx.x) * q + i] = static_cast<double>(cnt[threadIdx.x]) / k;
}

// One CTA per coordinate: sort the accepted marginal, map each u = c / k to
// its ceil(c q / k)-th smallest value.
__global__ void __launch_bounds__(1024) recal_quantiles(const float* __restrict__ theta, uint32_t n,
                                                        const uint32_t* __restrict__ acc, uint32_t q,
                                                        uint32_t k, uint32_t P, const double* __restrict__ u,
                                                        float* __restrict__ theta_rc) {
  extern __shared__ float v[];
  const uint32_t d = blockIdx.x;
  for (uint32_t t = threadIdx.x; t < P; t += blockDim.x)
    v[t] = (t < q && acc[t] < n) ? theta[static_cast<size_t>(d) * n + acc[t]] : __int_as_float(0x7F800000);
  __syncthreads();
  for (uint32_t size = 2; size <= P; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
        const uint32_t lo = 2 * t - (t & (stride - 1));
        const uint32_t hi = lo + stride;
        const bool up = (lo & size) == 0;
        const float a = v[lo], b = v[hi];
        if ((a > b) == up) {
          v[lo] = b;
          v[hi] = a;
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < q; i += blockDim.x) {
    const double ui = u[static_cast<size_t>(d) * q + i];
    if (ui != ui) {
      theta_rc[static_cast<size_t>(d) * q + i] = __int_as_float(0x7FC00000);
      continue;
    }
    // u = c / k: the rank ceil(u q) = ceil(c q / k) from the count, in
    // integers (the binary64 product u q can round above an integer).
    const uint64_t c = static_cast<uint64_t>(llrint(ui * static_cast<double>(k)));
    uint64_t r = (c * q + k - 1) / k;
    if (r < 1) r = 1;
    if (r > q) r = q;
    theta_rc[static_cast<size_t>(d) * q + i] = v[r - 1];
  }
}

}  // namespace

}  // namespace ppabc

using namespace ppabc;

extern "C" {

size_t abc_recalibrate_workspace_bytes(uint64_t n, uint64_t k) { return RcLayout(n ? n : 1, k ? k : 1).total; }

int abc_recalibrate(const double* summ, const float* theta, uint64_t n, uint32_t n_obs,
                    const uint32_t* acc_idx, uint64_t q, uint64_t k, double* u_out, float* theta_rc_out,
                    void* workspace, size_t workspace_bytes, void* stream) {
  if (!summ || !theta || !acc_idx || !u_out || !theta_rc_out)
    return set_error(PPABC_EINVAL, "summ, theta, acc_idx, u_out and theta_rc_out must be non-NULL");
  if (n == 0 || n > 0xFFFFFFFFull) return set_error(PPABC_EINVAL, "n must be in [1, 2^32)");
  if (n_obs < 1 || n_obs > PPABC_MAX_OBS) return set_error(PPABC_EINVAL, "n_obs must be in [1, %d]", PPABC_MAX_OBS);
  if (q == 0 || q > PPABC_RECAL_MAX_Q) return set_error(PPABC_EINVAL, "q must be in [1, %d]", PPABC_RECAL_MAX_Q);
  if (k == 0 || k > n) return set_error(PPABC_EINVAL, "k must be in [1, n]");
  const RcLayout L(n, k);
  if (!workspace || workspace_bytes < L.total)
    return set_error(PPABC_ENOMEM, "workspace needs %zu bytes, got %zu", L.total, workspace_bytes);
  if (reinterpret_cast<uintptr_t>(workspace) & 255u) return set_error(PPABC_EINVAL, "workspace must be 256-byte aligned");
  int rc = require_device();
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(workspace);
  double* dist = reinterpret_cast<double*>(w + L.dist);
  uint32_t* idx = reinterpret_cast<uint32_t*>(w + L.idx);
  float* rec = reinterpret_cast<float*>(w + L.rec);
  uint64_t* nacc = reinterpret_cast<uint64_t*>(w + L.nacc);
  OUConst P;
  memset(&P, 0, sizeof(P));
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned blocks = static_cast<unsigned>(std::min<uint64_t>((n + 255) / 256, static_cast<uint64_t>(sms > 0 ? sms : 1) * 16));
  cudaError_t e = cudaSuccess;
  for (uint64_t i = 0; i < q && e == cudaSuccess; ++i) {
    summary_distance<<<blocks, 256, 0, s>>>(summ, static_cast<uint32_t>(n), n_obs, acc_idx,
                                            static_cast<uint32_t>(i), dist);
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = launch_select(dist, static_cast<uint32_t>(n), k, 0.0, P, 0, theta, idx, rec, k, nacc, nullptr,
                        nullptr, w + L.select, s);
    if (e == cudaSuccess) {
      recal_u<<<1, 256, 0, s>>>(reinterpret_cast<const float4*>(rec), static_cast<uint32_t>(k), theta,
                                static_cast<uint32_t>(n), acc_idx, static_cast<uint32_t>(i),
                                static_cast<uint32_t>(q), u_out);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) {
    uint32_t Pq = 2;
    while (Pq < q) Pq <<= 1;
    const size_t smem = sizeof(float) * Pq;
    e = cudaFuncSetAttribute(recal_quantiles, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e == cudaSuccess) {
      recal_quantiles<<<3, 1024, smem, s>>>(theta, static_cast<uint32_t>(n), acc_idx, static_cast<uint32_t>(q),
                                            static_cast<uint32_t>(k), Pq, u_out, theta_rc_out);
      e = cudaGetLastError();
    }
  }
  return check_cuda(e, "abc_recalibrate");
}

}  // extern "C"
