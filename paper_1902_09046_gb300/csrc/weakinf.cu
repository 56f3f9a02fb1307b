// weakinf.cu -- weak-informativity test (Algorithm 2) for the conjugate model.
//
// For each hyperparameter lambda_k (Sec. 4.1, Eq. 8 and Eq. 9), Algorithm 2
// draws N data sets from the base prior predictive (lambda_0) and N from the
// lambda_k prior predictive, estimates the p-value of every base data set
// under lambda_k as the fraction of lambda_k data sets whose prior-predictive
// density is no larger, and returns the alpha quantile of those p-values.
// With the sufficient statistic ybar (density falling in |ybar|) the count
// for base set i is #{j : |ybar_k^j| >= |ybar_0^i|}.
//
// Two kernels.  The first draws every |ybar| of both kinds for every lambda
// over the whole GPU (two data sets per thread, packed as in the p-value
// sweep) into the caller's workspace.  The second runs one CTA per lambda_k:
// the N values |ybar_k^j| are bitonic-sorted in shared memory, every base
// set's count is a binary search, and the ceil(alpha N)-th smallest count
// comes from a shared histogram of the counts.  The paper's N^2 indicator sum
// becomes N log N work per lambda.
#include "internal.h"
#include "ybar.cuh"

namespace ppabc {

namespace {

constexpr int kWiThreads = 1024;
constexpr int kWiMaxPerThread = PPABC_WEAKINF_MAX_SETS / kWiThreads;

// |ybar| of data sets (kind, k, j), kind 0 = lambda_k sets (stream tag PATH,
// lambda[k]), kind 1 = base sets (tag BASE, lambda0), into abs_out[kind][k][j].
// Thread t of the grid-stride takes the pair j0 = 2 (t mod ceil(N/2)) and
// j0 + 1 of one (kind, k).
__global__ void __launch_bounds__(256) weakinf_ybar(const double* __restrict__ lambda, uint32_t n_lambda,
                                                    double lambda0, uint32_t n_obs, double inv_n, uint32_t N,
                                                    const __grid_constant__ PhiloxKeys K,
                                                    double* __restrict__ abs_out) {
  const uint32_t half = (N + 1) >> 1;
  const uint64_t items = 2ull * n_lambda * half;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t t = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < items; t += stride) {
    const uint32_t jj = static_cast<uint32_t>(t % half);
    const uint64_t kk = t / half;  // kind * n_lambda + k
    const uint32_t kind = static_cast<uint32_t>(kk / n_lambda);
    const uint32_t k = static_cast<uint32_t>(kk % n_lambda);
    const uint32_t j0 = 2 * jj, j1 = j0 + 1 < N ? j0 + 1 : j0;
    const double lam = kind ? lambda0 : lambda[k];
    const double2 yb = dataset_ybar2<false, false>(BmTab{}, K, lam, n_obs, inv_n, j0, j1, k,
                                                   kind ? kTagBase : kTagPath);
    double* out = abs_out + (static_cast<size_t>(kind) * n_lambda + k) * N;
    out[j0] = fabs(yb.x);
    if (j0 + 1 < N) out[j0 + 1] = fabs(yb.y);
  }
}

// Register-blocked bitonic sort of kWiRegKeys = 16 * kWiThreads keys (one
// lambda's padded sets when N > 8192): thread t holds the run 16 t .. 16 t +
// 15 in registers.  Merges whose stride is below 16 stay inside a run and run
// in registers; the wider ones go through shared memory, where element e of
// run t sits at 16 t + 2 ((e / 2 mod 8) xor (t mod 8)) + e mod 2, so that
// the runs' 16-byte chunks, read and written a chunk per lane, spread over
// all banks.  55 shared-memory stages and barriers instead of 105.
constexpr uint32_t kWiRegKeys = 16u * kWiThreads;

__device__ __forceinline__ uint32_t wi_phys(uint32_t e) {
  return (e & ~15u) | (((((e >> 1) & 7u) ^ ((e >> 4) & 7u))) << 1) | (e & 1u);
}

__device__ __forceinline__ void wi_cas(unsigned long long& a, unsigned long long& b, bool up) {
  const unsigned long long lo = a < b ? a : b, hi = a < b ? b : a;
  a = up ? lo : hi;
  b = up ? hi : lo;
}

// In-register stages of one merge size, strides `first` .. 1 (first <= 8).
__device__ __forceinline__ void wi_reg_stages(unsigned long long (&r)[16], uint32_t t, uint32_t size,
                                              uint32_t first) {
#pragma unroll
  for (uint32_t st = 8; st > 0; st >>= 1) {
    if (st > first) continue;
#pragma unroll
    for (uint32_t i = 0; i < 16; ++i) {
      if (i & st) continue;
      wi_cas(r[i], r[i + st], ((16u * t + i) & size) == 0u);
    }
  }
}

__device__ __forceinline__ void wi_store_run(unsigned long long* smem, const unsigned long long (&r)[16],
                                             uint32_t t) {
#pragma unroll
  for (uint32_t c = 0; c < 8; ++c) {
    ulonglong2 v;
    v.x = r[2 * c];
    v.y = r[2 * c + 1];
    *reinterpret_cast<ulonglong2*>(smem + 16u * t + 2u * (c ^ (t & 7u))) = v;
  }
}

__device__ __forceinline__ void wi_load_run(const unsigned long long* smem, unsigned long long (&r)[16],
                                            uint32_t t) {
#pragma unroll
  for (uint32_t c = 0; c < 8; ++c) {
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(smem + 16u * t + 2u * (c ^ (t & 7u)));
    r[2 * c] = v.x;
    r[2 * c + 1] = v.y;
  }
}

// Sorts the kWiRegKeys keys src[0..N) (+inf beyond) ascending into smem, in
// the layout wi_phys describes.
__device__ void wi_sort_blocked(const double* __restrict__ src, uint32_t N, unsigned long long* smem) {
  const uint32_t t = threadIdx.x;
  unsigned long long r[16];
#pragma unroll
  for (uint32_t i = 0; i < 16; ++i) {
    const uint32_t e = 16u * t + i;
    r[i] = e < N ? static_cast<unsigned long long>(__double_as_longlong(src[e])) : 0x7FF0000000000000ull;
  }
#pragma unroll
  for (uint32_t size = 2; size <= 16; size <<= 1) wi_reg_stages(r, t, size, size >> 1);
  for (uint32_t size = 32; size <= kWiRegKeys; size <<= 1) {
    wi_store_run(smem, r, t);
    __syncthreads();
    for (uint32_t stride = size >> 1; stride >= 16; stride >>= 1) {
#pragma unroll
      for (uint32_t u = 0; u < kWiRegKeys / 2 / kWiThreads; ++u) {
        const uint32_t tt = t + u * kWiThreads;
        const uint32_t lo = 2 * tt - (tt & (stride - 1));
        const uint32_t plo = wi_phys(lo), phi = wi_phys(lo + stride);
        unsigned long long a = smem[plo], b = smem[phi];
        if ((a > b) == ((lo & size) == 0)) {
          smem[plo] = b;
          smem[phi] = a;
        }
      }
      __syncthreads();
    }
    wi_load_run(smem, r, t);
    wi_reg_stages(r, t, size, 8);
  }
  wi_store_run(smem, r, t);
  __syncthreads();
}

__global__ void __launch_bounds__(kWiThreads) weakinf_kernel(
    const double* __restrict__ lam_abs /* [n_lambda][N] */, const double* __restrict__ base_abs,
    uint32_t N, uint32_t P /* power of two >= N */, uint32_t rank /* ceil(alpha N), 1-based */,
    double* __restrict__ gamma_out, uint32_t* __restrict__ counts_out) {
  // The values are |ybar| >= 0 (and +inf padding), whose binary64 bit
  // patterns order exactly as the numbers: the sort and the searches compare
  // them as 64-bit integers, on the integer pipes (binary64 compares would
  // queue on this GPU's narrow FP64 pipe).
  extern __shared__ __align__(16) unsigned long long smem[];  // P keys; later reused as N+1 histogram bins
  __shared__ unsigned int scan_smem[kWiThreads / 32];
  __shared__ unsigned int s_answer;
  const uint32_t k = blockIdx.x;
  const bool blocked = P == kWiRegKeys;  // the register-blocked sort and its layout
  if (blocked) {
    wi_sort_blocked(lam_abs + static_cast<size_t>(k) * N, N, smem);
  } else {
    // 1. |ybar| of the lambda_k data sets, padded with +inf to P entries.
    for (uint32_t j = threadIdx.x; j < P; j += kWiThreads)
      smem[j] = j < N ? static_cast<unsigned long long>(__double_as_longlong(lam_abs[static_cast<size_t>(k) * N + j]))
                      : 0x7FF0000000000000ull;
    __syncthreads();
    // 2. Bitonic sort, ascending.  At a stride of at most 32 the pairs of warp
    // w's thread t (t = 32 w + lane + 1024 m) lie in the 64-element block
    // starting at 64 (w + 32 m), the same block at every such stride, so
    // between two such stages only the warp has to synchronise.
    for (uint32_t size = 2; size <= P; size <<= 1) {
      for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
        for (uint32_t t = threadIdx.x; t < (P >> 1); t += kWiThreads) {
          const uint32_t lo = 2 * t - (t & (stride - 1));
          const uint32_t hi = lo + stride;
          const bool up = (lo & size) == 0;
          const unsigned long long a = smem[lo], b = smem[hi];
          if ((a > b) == up) {
            smem[lo] = b;
            smem[hi] = a;
          }
        }
        const uint32_t next = stride > 1 ? stride >> 1 : size;  // the next stage's stride
        if (stride <= 32 && next <= 32)
          __syncwarp();
        else
          __syncthreads();
      }
    }
    __syncthreads();
  }
  // 3. Counts of the base data sets: N - (first index with value >= |ybar_0|).
  uint32_t my_counts[kWiMaxPerThread];
#pragma unroll
  for (int q = 0; q < kWiMaxPerThread; ++q) {
    const uint32_t i = threadIdx.x + q * kWiThreads;
    my_counts[q] = 0;
    if (i < N) {
      const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(base_abs[static_cast<size_t>(k) * N + i]));
      uint32_t lo = 0, hi = N;  // search in [0, N)
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (smem[blocked ? wi_phys(mid) : mid] < b)
          lo = mid + 1;
        else
          hi = mid;
      }
      my_counts[q] = N - lo;
      if (counts_out) counts_out[static_cast<size_t>(k) * N + i] = N - lo;
    }
  }
  __syncthreads();
  // 4. Histogram of the counts (values 0..N) in the same shared memory.
  unsigned int* hist = reinterpret_cast<unsigned int*>(smem);
  for (uint32_t v = threadIdx.x; v <= N; v += kWiThreads) hist[v] = 0u;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kWiMaxPerThread; ++q) {
    const uint32_t i = threadIdx.x + q * kWiThreads;
    if (i < N) atomicAdd(&hist[my_counts[q]], 1u);
  }
  __syncthreads();
  // 5. The rank-th smallest count: each thread owns a contiguous run of bins.
  const uint32_t bins = N + 1;
  const uint32_t per = (bins + kWiThreads - 1) / kWiThreads;
  const uint32_t v0 = threadIdx.x * per;
  unsigned int mine = 0;
  for (uint32_t v = v0; v < v0 + per && v < bins; ++v) mine += hist[v];
  // block exclusive scan of `mine`
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned int x = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) scan_smem[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned int w = scan_smem[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= o) w += y;
    }
    scan_smem[lane] = w;
  }
  __syncthreads();
  const unsigned int before = (warp ? scan_smem[warp - 1] : 0u) + x - mine;
  if (before < rank && rank <= before + mine) {
    unsigned int run = before;
    for (uint32_t v = v0; v < v0 + per && v < bins; ++v) {
      run += hist[v];
      if (run >= rank) {
        s_answer = v;
        break;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) gamma_out[k] = static_cast<double>(s_answer) / static_cast<double>(N);
}

}  // namespace

size_t weakinf_workspace_bytes(uint64_t n_lambda, uint64_t n_sets) {
  return 2 * sizeof(double) * n_lambda * n_sets;
}

cudaError_t launch_weakinf(const double* lambda, uint32_t n_lambda, double lambda0, uint32_t n_obs,
                           uint32_t n_sets, double alpha, uint64_t seed, double* gamma_out,
                           uint32_t* counts_out, void* workspace, cudaStream_t s) {
  uint32_t P = 1;
  while (P < n_sets) P <<= 1;
  if (P < 2) P = 2;
  const size_t smem = sizeof(double) * (P > n_sets + 1 ? P : n_sets + 1);
  cudaError_t e = cudaFuncSetAttribute(weakinf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  uint64_t rank = static_cast<uint64_t>(ceil(alpha * static_cast<double>(n_sets)));
  if (rank < 1) rank = 1;
  if (rank > n_sets) rank = n_sets;
  double* abs_all = static_cast<double*>(workspace);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t items = 2ull * n_lambda * ((n_sets + 1) / 2);
  uint64_t blocks = (items + 255) / 256;
  const uint64_t cap = static_cast<uint64_t>(sms > 0 ? sms : 1) * 8 * 4;
  if (blocks > cap) blocks = cap;
  weakinf_ybar<<<static_cast<unsigned>(blocks), 256, 0, s>>>(lambda, n_lambda, lambda0, n_obs,
                                                             1.0 / static_cast<double>(n_obs), n_sets,
                                                             philox_keys(seed), abs_all);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  weakinf_kernel<<<n_lambda, kWiThreads, smem, s>>>(abs_all, abs_all + static_cast<size_t>(n_lambda) * n_sets,
                                                    n_sets, P, static_cast<uint32_t>(rank), gamma_out, counts_out);
  return cudaGetLastError();
}

}  // namespace ppabc
