// em_ou.cu -- fused prior-predictive OU kernels and the raw RNG kernels.
//
// Prior draw, Euler-Maruyama path, summaries and discrepancy all happen in
// registers; the only global traffic is the optional theta / summary write
// and one binary64 distance per sample.  This replaces the paper's
// block-of-VECL SIMD loop with pre-generated normals (Sec. 3.4): on the GPU a
// warp is the SIMD vector, the sample index is the lane, and the normals
// never touch memory.  Two kernels, chosen by the launch size, give the same
// results bit for bit:
//   em_ou_fused_x2: two interleaved paths per thread (ou_path2), for large
//     launches;
//   em_ou_pipe: a warp-specialised pipeline over 32 samples per CTA, for
//     small ones.
// Both write theta ([3][n]) and the summaries ([n_obs][n]) when asked.
#include <atomic>

#include "internal.h"

namespace ppabc {

// The two-path kernel keeps the Box-Muller tables in shared memory (80 KB
// with the lane-replicated log table): 512-thread CTAs, two per SM, 32 warps.
constexpr int kEmThreads = 512;
constexpr size_t kEmSmem = bm_smem_bytes<true>();

// Samples i and i + kEmThreads of each CTA's 2 kEmThreads range, interleaved
// (ou_path2).  Past the end of the launch the second path repeats the first
// (same index, so the same values) and writes nothing of its own: its
// summary row pointer is the first path's.
template <bool kWantTheta, bool kWantSumm>
__global__ void __launch_bounds__(kEmThreads, 2) em_ou_fused_x2(const __grid_constant__ OUConst P,
                                                                uint32_t base, uint32_t n,
                                                                float* __restrict__ theta_out,
                                                                double* __restrict__ summ_out,
                                                                double* __restrict__ dist_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  bm_load<true>(smem);
  __syncthreads();
  const BmTab T = bm_tab<true>(smem);
  const uint32_t i0 = blockIdx.x * (2 * kEmThreads) + threadIdx.x;
  const uint32_t i1 = i0 + kEmThreads;
  if (i0 >= n) return;
  const bool has1 = i1 < n;
  const uint32_t gi[2] = {base + i0, base + (has1 ? i1 : i0)};
  float th1[2], th2[2], th3[2];
  ou_prior(P, gi[0], th1[0], th2[0], th3[0]);
  ou_prior(P, gi[1], th1[1], th2[1], th3[1]);
  if (kWantTheta) {
    theta_out[i0] = th1[0];
    theta_out[static_cast<size_t>(n) + i0] = th2[0];
    theta_out[2 * static_cast<size_t>(n) + i0] = th3[0];
    if (has1) {
      theta_out[i1] = th1[1];
      theta_out[static_cast<size_t>(n) + i1] = th2[1];
      theta_out[2 * static_cast<size_t>(n) + i1] = th3[1];
    }
  }
  double d[2];
  ou_path2<kWantSumm, true>(P, T, gi, th1, th2, th3, kWantSumm ? summ_out + i0 : nullptr,
                            kWantSumm ? summ_out + (has1 ? i1 : i0) : nullptr, n, d);
  dist_out[i0] = d[0];
  if (has1) dist_out[i1] = d[1];
}

// Small launches (n up to kPipeMaxN samples): a warp-specialised pipeline.
// With few samples the two-path kernel leaves most of the GPU idle and each
// warp waits on its own dependency chain.  Here a CTA owns 32 samples: warps
// 1..kPipeProducers draw the scaled normals of every counter block for those
// samples (lane = sample) into a double-buffered ring in shared memory, kPipeRound
// blocks per round, while warp 0 runs the samples' Euler-Maruyama paths
// (lane = sample) over the previous round's blocks.  The path arithmetic is
// ou_path's, block by block in the same order, so the distances are bit for
// bit those of the other kernels (the compact copy of the log table holds the
// same values as the replicated one).  Rounds end at a CTA barrier; nothing
// spins.
constexpr int kPipeProducers = 6;
constexpr int kPipeRound = 24;
constexpr int kPipeThreads = 32 * (1 + kPipeProducers);
static_assert(kPipeRound % kPipeProducers == 0, "every producer draws the same number of blocks a round");
// A CTA lives for one short pass over its 32 samples, so the producers read
// the Box-Muller tables from global memory (L1-cached; bm_tab_global) rather
// than copying 50 KB into shared memory per CTA.
template <bool kWantTheta, bool kWantSumm>
__global__ void __launch_bounds__(kPipeThreads) em_ou_pipe(const __grid_constant__ OUConst P, uint32_t base,
                                                           uint32_t n, float* __restrict__ theta_out,
                                                           double* __restrict__ summ_out,
                                                           double* __restrict__ dist_out) {
  __shared__ float4 ring[2][kPipeRound][32];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t i = blockIdx.x * 32 + lane;
  const bool valid = i < n;
  const uint32_t g = base + (valid ? i : n - 1);
  float th1, th2, th3;
  ou_prior(P, g, th1, th2, th3);
  const float c = th3 * P.sqrt_dt;
  const uint32_t S = P.n_steps, n_obs = P.n_obs;
  const uint32_t n_blocks = (P.s_obs[n_obs - 1] + 3u) >> 2;  // blocks up to the last observation
  const uint32_t rounds = (n_blocks + kPipeRound - 1) / kPipeRound;
  if (warp > 0) {
    const BmTab T = bm_tab_global();
    const PhiloxFamily fam = philox_family(P.keys, kTagPath, P.sub);
    const PhiloxStream stream = philox_stream(P.keys, fam, g);
    for (uint32_t r = 0; r <= rounds; ++r) {
      if (r < rounds) {
        // Blocks q = warp - 1 + kPipeProducers h of the round: a fixed count,
        // so the two chains interleave (5% faster at N = 10^4).
#pragma unroll
        for (uint32_t h = 0; h < static_cast<uint32_t>(kPipeRound / kPipeProducers); ++h) {
          const uint32_t q = warp - 1 + h * kPipeProducers;
          const uint32_t b = r * kPipeRound + q;
          if (b < n_blocks)
            ring[r & 1u][q][lane] = scaled_tnormals_of<false>(T, philox_block(P.keys, fam, stream, b), c);
        }
      }
      __syncthreads();
    }
    return;
  }
  // Warp 0: ou_path's walk, one counter block at a time.
  if (kWantTheta && valid) {
    theta_out[i] = th1;
    theta_out[static_cast<size_t>(n) + i] = th2;
    theta_out[2 * static_cast<size_t>(n) + i] = th3;
  }
  const float k = th1 * P.dt;
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
  uint32_t s = 0, b = 0, j = 0, s_next = 0, b_end = 0;
  bool seg = true;       // a new run of whole blocks starts at block b
  bool pending = false;  // zp holds the first block of a pair of the run
  float4 zp = make_float4(0.f, 0.f, 0.f, 0.f);
  for (uint32_t r = 0; r <= rounds; ++r) {
    if (r > 0) {
      const float4(&rd)[kPipeRound][32] = ring[(r - 1) & 1u];
      const uint32_t done = (r - 1) * kPipeRound;  // < n_blocks
      const uint32_t qend = n_blocks - done < static_cast<uint32_t>(kPipeRound) ? n_blocks - done
                                                                                : static_cast<uint32_t>(kPipeRound);
      uint32_t q = 0;
      while (q < qend && j < n_obs) {
        // Four whole blocks of the current run: the pair updates that the
        // block-at-a-time code below makes, in the same order, with the four
        // ring reads issued first.  Without a pending block the pairs are
        // (b, b+1), (b+2, b+3); with one, (zp, b), (b+1, b+2), and b+3 becomes
        // the pending block, which needs a block after it in the run.
        if (!seg && q + 4 <= qend && (pending ? b + 4 < b_end : b + 4 <= b_end)) {
          const float4 z0 = rd[q][lane], z1 = rd[q + 1][lane], z2 = rd[q + 2][lane], z3 = rd[q + 3][lane];
          if (pending) {
            em_block8(Y, comp, E4, zp, z0);
            em_block8(Y, comp, E4, z1, z2);
            zp = z3;
          } else {
            em_block8(Y, comp, E4, z0, z1);
            em_block8(Y, comp, E4, z2, z3);
          }
          b += 4;
          q += 4;
          continue;
        }
        const float4 z = rd[q][lane];
        ++q;
        if (seg) {
          s_next = P.s_obs[j];
          b_end = b + (s_next > s + 4u ? (s_next - s - 1u) >> 2 : 0u);
          s += (b_end - b) << 2;
          seg = false;
        }
        if (b < b_end) {  // the run's blocks in pairs, an odd last one alone (as ou_path)
          if (pending) {
            em_block8(Y, comp, E4, zp, z);
            pending = false;
          } else if (b + 1 < b_end) {
            zp = z;
            pending = true;
          } else {
            em_block4(Y, comp, E4, z);
          }
          ++b;
          continue;
        }
        ++b;  // the block holding step s_next (and possibly later observation steps)
        const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          if (s < S) {
            em_step(Y, comp, k, zz[l]);
            ++s;
            if (s == s_next) {
              const double x = th2d + (static_cast<double>(Y) - static_cast<double>(comp));
              const double rr = x - P.y[j];
              acc = fma(rr, rr, acc);
              if (kWantSumm && valid) summ_out[static_cast<size_t>(j) * n + i] = x;
              ++j;
              s_next = (j < n_obs) ? P.s_obs[j] : 0xFFFFFFFFu;
            }
          }
        }
        seg = true;
      }
    }
    __syncthreads();
  }
  if (valid) dist_out[i] = sqrt(acc);
}

constexpr uint32_t kPipeMaxN = 98304;  // above about this the two-path kernel is faster

cudaError_t bm_hooks_prepare();

cudaError_t em_prepare() {
  static std::atomic<unsigned long long> ready{0ull};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (ready.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  const int big = static_cast<int>(kEmSmem);
  e = cudaFuncSetAttribute(em_ou_fused_x2<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(em_ou_fused_x2<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(em_ou_fused_x2<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(em_ou_fused_x2<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = bm_hooks_prepare();
  if (e == cudaSuccess && bit) ready.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

namespace {

template <bool kWantTheta, bool kWantSumm>
cudaError_t launch_em_ou_as(const OUConst& P, uint32_t base, uint32_t n, float* theta_out, double* summ_out,
                            double* dist_out, cudaStream_t s) {
  if (n <= kPipeMaxN) {
    em_ou_pipe<kWantTheta, kWantSumm><<<(n + 31) / 32, kPipeThreads, 0, s>>>(P, base, n, theta_out, summ_out,
                                                                             dist_out);
  } else {
    const dim3 grid((n + 2 * kEmThreads - 1) / (2 * kEmThreads));
    em_ou_fused_x2<kWantTheta, kWantSumm><<<grid, kEmThreads, kEmSmem, s>>>(P, base, n, theta_out, summ_out,
                                                                            dist_out);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_em_ou(const OUConst& P, uint64_t base, uint32_t n, float* theta_out,
                         double* summ_out, double* dist_out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  cudaError_t e = em_prepare();
  if (e != cudaSuccess) return e;
  const uint32_t b = static_cast<uint32_t>(base);
  if (theta_out && summ_out) return launch_em_ou_as<true, true>(P, b, n, theta_out, summ_out, dist_out, s);
  if (theta_out) return launch_em_ou_as<true, false>(P, b, n, theta_out, summ_out, dist_out, s);
  if (summ_out) return launch_em_ou_as<false, true>(P, b, n, theta_out, summ_out, dist_out, s);
  return launch_em_ou_as<false, false>(P, b, n, theta_out, summ_out, dist_out, s);
}

// ---------------------------------------------------------------------------
// Raw generator outputs (parity hooks for the RNG itself).
// ---------------------------------------------------------------------------
__global__ void philox_raw_kernel(const __grid_constant__ PhiloxKeys K, const uint4* __restrict__ ctr,
                                  uint64_t n, uint4* __restrict__ out) {
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] = philox4x32_10(ctr[i], K);
}

// method 0 (PPABC_BM_POLY): the polynomial transform of rng.cuh, used by the
// p-value, Algorithm 2 and toggle kernels; method 1 (PPABC_BM_TABLE): the
// table-driven transform of bm_table.cuh, used by the OU path kernels.
constexpr size_t kHookSmem = bm_smem_bytes<false>();

template <int kMethod>
__global__ void normals_kernel(const __grid_constant__ PhiloxKeys K, uint32_t c1, uint32_t c2,
                               uint32_t tag, uint64_t j0, uint64_t n, float* __restrict__ z) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (kMethod == 1) {
    bm_load<false>(smem);
    __syncthreads();
  }
  const uint64_t t = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const uint64_t j = j0 + t;
  const PhiloxFamily F = philox_family(K, tag, c2);
  const PhiloxStream S = philox_stream(K, F, c1);
  const uint4 w = philox_block(K, F, S, static_cast<uint32_t>(j >> 2));
  const float4 q = kMethod == 1 ? tnormals_of<false>(bm_tab<false>(smem), w) : normals_of(w);
  const uint32_t lane = static_cast<uint32_t>(j & 3u);
  z[t] = lane == 0 ? q.x : lane == 1 ? q.y : lane == 2 ? q.z : q.w;
}

template <int kMethod>
__global__ void box_muller_kernel(const uint2* __restrict__ w, uint64_t n, float2* __restrict__ z) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (kMethod == 1) {
    bm_load<false>(smem);
    __syncthreads();
  }
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint2 p = w[i];
  float2 q;
  if (kMethod == 1)
    box_muller_tab<false>(bm_tab<false>(smem), p.x, p.y, q.x, q.y);
  else
    box_muller(p.x, p.y, q.x, q.y);
  z[i] = q;
}

cudaError_t bm_hooks_prepare() {
  cudaError_t e = cudaFuncSetAttribute(normals_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(kHookSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(box_muller_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kHookSmem));
  return e;
}

cudaError_t launch_box_muller(const uint32_t* w, uint64_t n, uint32_t method, float* z, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  cudaError_t e = em_prepare();
  if (e != cudaSuccess) return e;
  const unsigned blocks = static_cast<unsigned>((n + 1023) / 1024);
  const uint2* w2 = reinterpret_cast<const uint2*>(w);
  float2* z2 = reinterpret_cast<float2*>(z);
  if (method == 1)
    box_muller_kernel<1><<<blocks, 1024, kHookSmem, s>>>(w2, n, z2);
  else
    box_muller_kernel<0><<<blocks, 1024, 0, s>>>(w2, n, z2);
  return cudaGetLastError();
}

cudaError_t launch_philox_raw(uint64_t seed, const uint32_t* ctr, uint64_t n, uint32_t* out,
                              cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const unsigned blocks = static_cast<unsigned>((n + 255) / 256);
  philox_raw_kernel<<<blocks, 256, 0, s>>>(philox_keys(seed), reinterpret_cast<const uint4*>(ctr), n,
                                           reinterpret_cast<uint4*>(out));
  return cudaGetLastError();
}

cudaError_t launch_normals(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t tag, uint64_t j0,
                           uint64_t n, uint32_t method, float* z, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  cudaError_t e = em_prepare();
  if (e != cudaSuccess) return e;
  const unsigned blocks = static_cast<unsigned>((n + 1023) / 1024);
  if (method == 1)
    normals_kernel<1><<<blocks, 1024, kHookSmem, s>>>(philox_keys(seed), c1, c2, tag, j0, n, z);
  else
    normals_kernel<0><<<blocks, 1024, 0, s>>>(philox_keys(seed), c1, c2, tag, j0, n, z);
  return cudaGetLastError();
}

}  // namespace ppabc
