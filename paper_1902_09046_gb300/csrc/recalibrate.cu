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
// Up to kKnnMaxN stored pairs one launch does all accepted samples, one CTA
// each (distances, radix select and counts in shared memory, recal_knn_u).
// Beyond that, per accepted sample the GPU forms the n binary64 distances
// (summaries are [n_obs][n], so a warp reads consecutive pairs), selects the
// k nearest exactly with the abc_select kernels (ties to the smaller index),
// and counts u.  A last kernel sorts each accepted marginal in shared memory
// and maps every u to its quantile.  Work is O(q n).
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

// One CTA per accepted sample, for n <= kKnnMaxN stored pairs: the n
// binary64 distances (the same fma order as summary_distance, so the same
// values) are kept in shared memory as their bit patterns, which order as the
// non-negative distances do (a NaN sorts after every number); an 8-pass radix
// select over those keys finds the k-th smallest key K and how many keys
// equal to K belong to the k nearest; the neighbours are every key below K
// and the first such keys equal to K in index order (the same set as the
// selection kernels give); u is counted from their theta.
constexpr int kKnnThreads = 512;
constexpr uint32_t kKnnMaxN = 24576;

__global__ void __launch_bounds__(kKnnThreads) recal_knn_u(const double* __restrict__ summ, uint32_t n,
                                                           uint32_t n_obs, const float* __restrict__ theta,
                                                           const uint32_t* __restrict__ acc, uint32_t q,
                                                           uint32_t k, double* __restrict__ u_out) {
  extern __shared__ unsigned long long keys[];  // n
  __shared__ unsigned int hist[256];
  __shared__ unsigned int warp_sums[kKnnThreads / 32];
  __shared__ unsigned long long s_prefix;
  __shared__ unsigned int s_rem;
  __shared__ unsigned int s_cnt[3];
  const uint32_t i = blockIdx.x;
  const uint32_t a = acc[i];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  if (a >= n) {  // invalid accepted index: NaN u (the whole CTA leaves here)
    if (threadIdx.x < 3) u_out[static_cast<size_t>(threadIdx.x) * q + i] = __longlong_as_double(0x7FF8000000000000ll);
    return;
  }
  // 1. Distances to pair a, as keys.
  for (uint32_t j = threadIdx.x; j < n; j += kKnnThreads) {
    double s2 = 0.0;
    for (uint32_t m = 0; m < n_obs; ++m) {
      const double r = summ[static_cast<size_t>(m) * n + j] - __ldg(summ + static_cast<size_t>(m) * n + a);
      s2 = fma(r, r, s2);
    }
    keys[j] = static_cast<unsigned long long>(__double_as_longlong(sqrt(s2)));
  }
  if (threadIdx.x < 3) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  // 2. Radix select of the k-th smallest key, 8 bits per pass from the top.
  unsigned long long prefix = 0, mask = 0;
  unsigned int rem = k;
  for (int pass = 7; pass >= 0; --pass) {
    const int shift = 8 * pass;
    for (uint32_t b = threadIdx.x; b < 256; b += kKnnThreads) hist[b] = 0;
    __syncthreads();
    const uint32_t rounds = (n + kKnnThreads - 1) / kKnnThreads;
    for (uint32_t r = 0; r < rounds; ++r) {
      const uint32_t j = r * kKnnThreads + threadIdx.x;
      unsigned int bin = 256;  // no bin
      if (j < n) {
        const unsigned long long key = keys[j];
        if ((key & mask) == prefix) bin = static_cast<unsigned int>((key >> shift) & 255u);
      }
      // Lanes with the same bin add once (most keys share the top bytes).
      const unsigned int peers = __match_any_sync(0xFFFFFFFFu, bin);
      if (bin < 256 && lane == static_cast<unsigned int>(__ffs(peers) - 1)) atomicAdd(&hist[bin], __popc(peers));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned int cum = 0;
      for (unsigned int d = 0; d < 256; ++d) {
        if (cum + hist[d] >= rem) {
          rem -= cum;
          prefix |= static_cast<unsigned long long>(d) << shift;
          break;
        }
        cum += hist[d];
      }
      s_prefix = prefix;
      s_rem = rem;
    }
    __syncthreads();
    prefix = s_prefix;
    rem = s_rem;
    mask |= 255ull << shift;
  }
  // 3. Count theta_j <= theta_a over the neighbours: keys below K, and the
  // first `rem` keys equal to K in index order.
  const unsigned long long K = prefix;
  const float t0 = theta[a], t1 = theta[static_cast<size_t>(n) + a], t2 = theta[2 * static_cast<size_t>(n) + a];
  unsigned int c0 = 0, c1 = 0, c2 = 0, eq_before = 0;
  for (uint32_t base = 0; base < n; base += kKnnThreads) {
    const uint32_t j = base + threadIdx.x;
    const unsigned long long key = j < n ? keys[j] : ~0ull;
    const bool less = key < K;
    const bool eq = j < n && key == K;
    bool take = less;
    const unsigned int n_eq = static_cast<unsigned int>(__syncthreads_count(eq));
    if (n_eq > 0) {  // rank of this equal key among the chunk's equal keys, in index order
      const unsigned int ballot = __ballot_sync(0xFFFFFFFFu, eq);
      if (lane == 0) warp_sums[warp] = __popc(ballot);
      __syncthreads();
      unsigned int before = __popc(ballot & ((1u << lane) - 1u));
      for (uint32_t w = 0; w < warp; ++w) before += warp_sums[w];
      take = take || (eq && eq_before + before < rem);
      __syncthreads();
      eq_before += n_eq;
    }
    if (take) {
      c0 += theta[j] <= t0;
      c1 += theta[static_cast<size_t>(n) + j] <= t1;
      c2 += theta[2 * static_cast<size_t>(n) + j] <= t2;
    }
  }
  c0 = __reduce_add_sync(0xFFFFFFFFu, c0);
  c1 = __reduce_add_sync(0xFFFFFFFFu, c1);
  c2 = __reduce_add_sync(0xFFFFFFFFu, c2);
  if (lane == 0) {
    atomicAdd(&s_cnt[0], c0);
    atomicAdd(&s_cnt[1], c1);
    atomicAdd(&s_cnt[2], c2);
  }
  __syncthreads();
  if (threadIdx.x < 3) u_out[static_cast<size_t>(threadIdx.x) * q + i] = static_cast<double>(s_cnt[threadIdx.x]) / k;
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
  if (n <= kKnnMaxN) {  // one launch, one CTA per accepted sample
    const size_t smem = sizeof(unsigned long long) * n;
    e = cudaFuncSetAttribute(recal_knn_u, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e == cudaSuccess) {
      recal_knn_u<<<static_cast<unsigned>(q), kKnnThreads, smem, s>>>(summ, static_cast<uint32_t>(n), n_obs, theta,
                                                                       acc_idx, static_cast<uint32_t>(q),
                                                                       static_cast<uint32_t>(k), u_out);
      e = cudaGetLastError();
    }
  }
  for (uint64_t i = 0; n > kKnnMaxN && i < q && e == cudaSuccess; ++i) {
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
