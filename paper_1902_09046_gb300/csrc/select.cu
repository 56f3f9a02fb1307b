// select.cu -- accepted set of ABC rejection and posterior moments.
//
// The paper fixes N and then picks epsilon a posteriori from the empirical
// distribution of the discrepancy (Sec. 3.1): accepting the k nearest means
// epsilon is the k-th smallest distance.  This file finds it with an exact
// MSD radix select over the order-preserving 64-bit image of each binary64
// distance (6 histogram passes of 11/11/11/11/11/9 bits; the last CTA of a
// pass picks the digit, so no host round trip), then writes the accepted
// samples in index order with a two-level scan, and reduces the posterior
// mean and variance with Chan's pairwise update in a fixed order.
//
// Threshold mode (k = 0) skips the radix passes: the key of epsilon itself is
// the cut.  Ties at the cut go to the smaller index in both modes.
#include <math.h>
#include <string.h>

#include "internal.h"

namespace ppabc {

namespace {

constexpr int kHistThreads = 256;
constexpr int kBins = 2048;          // 11-bit digits
constexpr int kTileThreads = 256;
constexpr int kPerThread = 16;
constexpr int kTile = kTileThreads * kPerThread;  // elements per compaction tile
constexpr int kNumPasses = 6;
__constant__ int kPassShift[kNumPasses] = {53, 42, 31, 20, 9, 0};
__constant__ int kPassBits[kNumPasses] = {11, 11, 11, 11, 11, 9};

struct SelState {
  unsigned long long prefix;  // key bits fixed so far
  unsigned long long mask;    // which bits of prefix are fixed
  unsigned long long krem;    // rank still to reach among keys matching prefix
  unsigned int ticket;        // CTAs done in the current pass
  unsigned int pad;
  unsigned long long n_acc;
};

struct MomentPart {  // per-tile (count, mean, M2) of the accepted theta
  double count;
  double mean[3];
  double m2[3];
  double pad;
};

inline size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

struct WsLayout {
  size_t state, hist, tile_less, tile_eq, tile_off, parts, total;
  explicit WsLayout(uint64_t n) {
    const size_t tiles = static_cast<size_t>((n + kTile - 1) / kTile);
    size_t o = 0;
    state = o;
    o = align256(o + sizeof(SelState));
    hist = o;
    o = align256(o + kBins * sizeof(unsigned int));
    tile_less = o;
    o = align256(o + tiles * sizeof(unsigned int));
    tile_eq = o;
    o = align256(o + tiles * sizeof(unsigned int));
    tile_off = o;
    o = align256(o + tiles * sizeof(unsigned int));
    parts = o;
    o = align256(o + tiles * sizeof(MomentPart));
    total = o;
  }
};

// Order-preserving image of a binary64 value: -0 maps to +0 and every NaN to
// the largest key.
__device__ __forceinline__ unsigned long long dist_key(double d) {
  if (isnan(d)) return 0xFFFFFFFFFFFFFFFFull;
  unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(d));
  if (b == 0x8000000000000000ull) b = 0ull;
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double key_to_double(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double(static_cast<long long>(b));
}

__global__ void select_init(SelState* st, unsigned int* hist, unsigned long long k) {
  for (int b = threadIdx.x; b < kBins; b += blockDim.x) hist[b] = 0u;
  if (threadIdx.x == 0) {
    st->prefix = 0ull;
    st->mask = 0ull;
    st->krem = k;
    st->ticket = 0u;
    st->n_acc = 0ull;
  }
}

// Block-wide exclusive scan of one unsigned value per thread (any blockDim.x
// that is a multiple of 32, up to 1024; smem holds one value per warp).
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* total, T* smem /* >= warps */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = (lane < (blockDim.x >> 5)) ? smem[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < (blockDim.x >> 5)) smem[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  const T warp_base = warp ? smem[warp - 1] : T(0);
  *total = smem[(blockDim.x >> 5) - 1];
  __syncthreads();
  return warp_base + x - v;
}

// One radix pass: histogram of the digit at `pass` over keys that match the
// prefix fixed so far; the last CTA to finish picks the digit holding rank
// krem and narrows the prefix.
__global__ void __launch_bounds__(kHistThreads) select_hist(const double* __restrict__ dist,
                                                            uint32_t n, int pass, SelState* st,
                                                            unsigned int* hist) {
  __shared__ unsigned int h[kBins];
  __shared__ bool is_last;
  __shared__ unsigned int scan_smem[8];
  const int shift = kPassShift[pass];
  const unsigned long long dmask = (1ull << kPassBits[pass]) - 1ull;
  for (int b = threadIdx.x; b < kBins; b += kHistThreads) h[b] = 0u;
  const unsigned long long prefix = st->prefix;
  const unsigned long long mask = st->mask;
  __syncthreads();
  // The loop bound is uniform across the CTA so every lane reaches the match.
  const int lane = threadIdx.x & 31;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kHistThreads;
  for (uint64_t b0 = static_cast<uint64_t>(blockIdx.x) * kHistThreads; b0 < n; b0 += stride) {
    const uint64_t i = b0 + threadIdx.x;
    unsigned int bin = 0xFFFFFFFFu;
    if (i < n) {
      const unsigned long long key = dist_key(__ldg(dist + i));
      if ((key & mask) == prefix) bin = static_cast<unsigned int>((key >> shift) & dmask);
    }
    // Distances crowd into few bins on the early passes: one shared atomic
    // per distinct bin in the warp.
    const unsigned int peers = __match_any_sync(0xFFFFFFFFu, bin);
    if (bin != 0xFFFFFFFFu && lane == __ffs(peers) - 1) atomicAdd(&h[bin], __popc(peers));
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kBins; b += kHistThreads)
    if (h[b]) atomicAdd(&hist[b], h[b]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(&st->ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // Each thread owns 8 consecutive bins.
  constexpr int kPer = kBins / kHistThreads;
  unsigned int c[kPer];
  unsigned int mine = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    c[q] = atomicExch(&hist[threadIdx.x * kPer + q], 0u);  // read and clear for the next pass
    mine += c[q];
  }
  unsigned int total;
  const unsigned int before = block_exclusive_scan<unsigned int>(mine, &total, scan_smem);
  const unsigned long long krem = st->krem;
  __syncthreads();
  if (before < krem && krem <= static_cast<unsigned long long>(before) + mine) {
    unsigned long long run = before;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      if (run < krem && krem <= run + c[q]) {
        const unsigned long long digit = static_cast<unsigned long long>(threadIdx.x * kPer + q);
        st->prefix = prefix | (digit << shift);
        st->mask = mask | (dmask << shift);
        st->krem = krem - run;
      }
      run += c[q];
    }
  }
  if (threadIdx.x == 0) st->ticket = 0u;
}

// Per-tile counts of keys below and at the cut.
__global__ void __launch_bounds__(kTileThreads) select_count(const double* __restrict__ dist,
                                                             uint32_t n, const SelState* st,
                                                             bool threshold,
                                                             unsigned long long cut_thr,
                                                             unsigned int* tile_less,
                                                             unsigned int* tile_eq) {
  __shared__ unsigned int s_less[kTileThreads / 32], s_eq[kTileThreads / 32];
  const unsigned long long cut = threshold ? cut_thr : st->prefix;
  const uint32_t t0 = blockIdx.x * kTile;
  unsigned int less = 0, eq = 0;
#pragma unroll 4
  for (int q = 0; q < kPerThread; ++q) {
    const uint32_t i = t0 + q * kTileThreads + threadIdx.x;  // coalesced
    if (i < n) {
      const unsigned long long key = dist_key(__ldg(dist + i));
      less += key < cut;
      eq += key == cut;
    }
  }
  less = __reduce_add_sync(0xFFFFFFFFu, less);
  eq = __reduce_add_sync(0xFFFFFFFFu, eq);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_less[warp] = less;
    s_eq[warp] = eq;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int a = 0, b = 0;
    for (int w = 0; w < kTileThreads / 32; ++w) {
      a += s_less[w];
      b += s_eq[w];
    }
    tile_less[blockIdx.x] = a;
    tile_eq[blockIdx.x] = b;
  }
}

// Single CTA: per tile, how many equal keys it may take and where its
// accepted samples start; total accepted and epsilon.
__global__ void __launch_bounds__(kTileThreads) select_scan(
    SelState* st, bool threshold, unsigned long long cut_thr, double eps_thr,
    const unsigned int* tile_less, unsigned int* tile_eq /* in: equal count, out: equal base */,
    unsigned int* tile_off, uint32_t tiles, unsigned long long* n_acc_out, double* eps_out) {
  __shared__ unsigned long long smem[8];
  __shared__ unsigned long long carry_eq, carry_acc;
  const unsigned long long krem = threshold ? 0xFFFFFFFFFFFFFFFFull : st->krem;
  if (threadIdx.x == 0) {
    carry_eq = 0ull;
    carry_acc = 0ull;
  }
  __syncthreads();
  for (uint32_t base = 0; base < tiles; base += kTileThreads) {
    const uint32_t t = base + threadIdx.x;
    const unsigned long long eq = t < tiles ? tile_eq[t] : 0u;
    const unsigned long long less = t < tiles ? tile_less[t] : 0u;
    unsigned long long tot_eq;
    const unsigned long long eq_before = carry_eq + block_exclusive_scan<unsigned long long>(eq, &tot_eq, smem);
    unsigned long long take_eq = 0;
    if (krem > eq_before) take_eq = (krem - eq_before < eq) ? (krem - eq_before) : eq;
    const unsigned long long acc = less + take_eq;
    unsigned long long tot_acc;
    const unsigned long long acc_before = carry_acc + block_exclusive_scan<unsigned long long>(acc, &tot_acc, smem);
    if (t < tiles) {
      tile_eq[t] = static_cast<unsigned int>(eq_before > 0xFFFFFFFFull ? 0xFFFFFFFFull : eq_before);
      tile_off[t] = static_cast<unsigned int>(acc_before);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry_eq += tot_eq;
      carry_acc += tot_acc;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    st->n_acc = carry_acc;
    *n_acc_out = carry_acc;
    if (eps_out) *eps_out = threshold ? eps_thr : key_to_double(st->prefix);
  }
}

// Writes the accepted samples of one tile in index order and the tile's
// (count, mean, M2) of theta.
template <bool kTheta>
__global__ void __launch_bounds__(kTileThreads) select_write(
    const double* __restrict__ dist, uint32_t n, const SelState* st, bool threshold,
    unsigned long long cut_thr, const unsigned int* __restrict__ tile_eq_base,
    const unsigned int* __restrict__ tile_off, const __grid_constant__ OUConst P, uint32_t base,
    const float* __restrict__ theta, uint32_t* __restrict__ idx_out, float4* __restrict__ rec_out,
    unsigned long long cap, MomentPart* __restrict__ parts) {
  __shared__ unsigned int scan_smem[8];
  __shared__ double red[3][kTileThreads / 32];
  __shared__ double s_mean[3];
  const unsigned long long cut = threshold ? cut_thr : st->prefix;
  const unsigned long long krem = threshold ? 0xFFFFFFFFFFFFFFFFull : st->krem;
  const uint32_t t0 = blockIdx.x * kTile + threadIdx.x * kPerThread;  // contiguous per thread
  // pass 1: flags and per-thread counts
  unsigned int flags = 0, eqmask = 0, my_eq = 0;
#pragma unroll
  for (int q = 0; q < kPerThread; ++q) {
    const uint32_t i = t0 + q;
    if (i < n) {
      const unsigned long long key = dist_key(dist[i]);
      if (key < cut) flags |= 1u << q;
      if (key == cut) {
        eqmask |= 1u << q;
        ++my_eq;
      }
    }
  }
  unsigned int tot;
  const unsigned int eq_rank0 = block_exclusive_scan<unsigned int>(my_eq, &tot, scan_smem);
  const unsigned long long eq_base = tile_eq_base[blockIdx.x];
  {
    unsigned long long r = eq_base + eq_rank0;
#pragma unroll
    for (int q = 0; q < kPerThread; ++q) {
      if (eqmask & (1u << q)) {
        if (r < krem) flags |= 1u << q;
        ++r;
      }
    }
  }
  const unsigned int my_acc = __popc(flags);
  const unsigned int pos0 = block_exclusive_scan<unsigned int>(my_acc, &tot, scan_smem);
  const unsigned long long off = tile_off[blockIdx.x];
  double sum[3] = {0.0, 0.0, 0.0};
  float th[kPerThread][3];
  {
    unsigned long long pos = off + pos0;
#pragma unroll
    for (int q = 0; q < kPerThread; ++q) {
      if (flags & (1u << q)) {
        const uint32_t i = t0 + q;
        float a, b, c;
        if (kTheta) {
          a = theta[i];
          b = theta[static_cast<size_t>(n) + i];
          c = theta[2 * static_cast<size_t>(n) + i];
        } else {
          ou_prior(P, base + i, a, b, c);
        }
        th[q][0] = a;
        th[q][1] = b;
        th[q][2] = c;
        sum[0] += a;
        sum[1] += b;
        sum[2] += c;
        if (pos < cap) {
          idx_out[pos] = i;
          rec_out[pos] = make_float4(a, b, c, static_cast<float>(dist[i]));
        }
        ++pos;
      }
    }
  }
  // tile mean (fixed-order reduction), then M2 about it
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = 0; d < 3; ++d) {
    double v = sum[d];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) red[d][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double v = 0.0;
    for (int w = 0; w < kTileThreads / 32; ++w) v += red[threadIdx.x][w];
    s_mean[threadIdx.x] = tot ? v / static_cast<double>(tot) : 0.0;
  }
  __syncthreads();
  double m2[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int q = 0; q < kPerThread; ++q) {
    if (flags & (1u << q)) {
      for (int d = 0; d < 3; ++d) {
        const double r = static_cast<double>(th[q][d]) - s_mean[d];
        m2[d] = fma(r, r, m2[d]);
      }
    }
  }
  for (int d = 0; d < 3; ++d) {
    double v = m2[d];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) red[d][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    MomentPart mp;
    mp.count = static_cast<double>(tot);
    for (int d = 0; d < 3; ++d) {
      double v = 0.0;
      for (int w = 0; w < kTileThreads / 32; ++w) v += red[d][w];
      mp.mean[d] = s_mean[d];
      mp.m2[d] = v;
    }
    mp.pad = 0.0;
    parts[blockIdx.x] = mp;
  }
}

// Chan, Golub & LeVeque pairwise combination of (count, mean, M2).
__device__ __forceinline__ void chan_merge(double& na, double* ma, double* qa, double nb,
                                           const double* mb, const double* qb) {
  if (nb == 0.0) return;
  if (na == 0.0) {
    na = nb;
    for (int d = 0; d < 3; ++d) {
      ma[d] = mb[d];
      qa[d] = qb[d];
    }
    return;
  }
  const double nab = na + nb;
  for (int d = 0; d < 3; ++d) {
    const double delta = mb[d] - ma[d];
    ma[d] = ma[d] + delta * (nb / nab);
    qa[d] = qa[d] + qb[d] + delta * delta * (na * nb / nab);
  }
  na = nab;
}

// Single CTA: merges the tile partials in a fixed order.
__global__ void __launch_bounds__(kTileThreads) select_moments(const MomentPart* __restrict__ parts,
                                                               uint32_t tiles, double* post_out) {
  __shared__ double s_n[kTileThreads], s_m[kTileThreads][3], s_q[kTileThreads][3];
  const uint32_t per = (tiles + kTileThreads - 1) / kTileThreads;
  double na = 0.0, ma[3] = {0, 0, 0}, qa[3] = {0, 0, 0};
  for (uint32_t t = threadIdx.x * per; t < tiles && t < (threadIdx.x + 1) * per; ++t) {
    const MomentPart p = parts[t];
    chan_merge(na, ma, qa, p.count, p.mean, p.m2);
  }
  s_n[threadIdx.x] = na;
  for (int d = 0; d < 3; ++d) {
    s_m[threadIdx.x][d] = ma[d];
    s_q[threadIdx.x][d] = qa[d];
  }
  __syncthreads();
  for (int stride = 1; stride < kTileThreads; stride <<= 1) {
    if ((threadIdx.x % (2 * stride)) == 0 && threadIdx.x + stride < kTileThreads) {
      double n0 = s_n[threadIdx.x];
      double m0[3], q0[3], m1[3], q1[3];
      for (int d = 0; d < 3; ++d) {
        m0[d] = s_m[threadIdx.x][d];
        q0[d] = s_q[threadIdx.x][d];
        m1[d] = s_m[threadIdx.x + stride][d];
        q1[d] = s_q[threadIdx.x + stride][d];
      }
      chan_merge(n0, m0, q0, s_n[threadIdx.x + stride], m1, q1);
      s_n[threadIdx.x] = n0;
      for (int d = 0; d < 3; ++d) {
        s_m[threadIdx.x][d] = m0[d];
        s_q[threadIdx.x][d] = q0[d];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double nn = s_n[0];
    for (int d = 0; d < 3; ++d) {
      post_out[d] = nn > 0.0 ? s_m[0][d] : nan("");
      post_out[3 + d] = nn > 1.0 ? s_q[0][d] / (nn - 1.0) : nan("");
    }
  }
}

// ---------------------------------------------------------------------------
// Small inputs (n <= kSmallMax): the whole selection in one CTA.  Keys and
// indices are bitonic-sorted in shared memory (ties by index), the accepted
// samples are flagged by index, then compacted in index order; the moments
// are a fixed-order block reduction.  One launch instead of eleven matters
// for the many small jobs of a serving mix.
// ---------------------------------------------------------------------------
constexpr int kSmallThreads = 1024;
constexpr int kSmallMax = 4096;
constexpr int kSmallPer = kSmallMax / kSmallThreads;

template <typename T>
__device__ __forceinline__ T block_sum_fixed(T v, T* red /* >= 32 */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T t = 0;
  for (int w = 0; w < kSmallThreads / 32; ++w) t += red[w];
  return t;
}

template <bool kTheta>
__global__ void __launch_bounds__(kSmallThreads) select_small(
    const double* __restrict__ dist, uint32_t n, uint32_t P, unsigned long long k, bool threshold,
    unsigned long long cut_thr, double eps_thr, const __grid_constant__ OUConst prm, uint32_t base,
    const float* __restrict__ theta, uint32_t* __restrict__ idx_out, float4* __restrict__ rec_out,
    unsigned long long cap, unsigned long long* __restrict__ n_acc_out, double* __restrict__ eps_out,
    double* __restrict__ post_out) {
  extern __shared__ unsigned long long sm_keys[];  // P keys, then P indices, then n flags
  uint32_t* sm_idx = reinterpret_cast<uint32_t*>(sm_keys + P);
  unsigned char* sm_flag = reinterpret_cast<unsigned char*>(sm_idx + P);
  __shared__ unsigned int scan_smem[kSmallThreads / 32];
  __shared__ double red[kSmallThreads / 32];
  for (uint32_t i = threadIdx.x; i < P; i += kSmallThreads) {
    sm_keys[i] = i < n ? dist_key(dist[i]) : 0xFFFFFFFFFFFFFFFFull;
    sm_idx[i] = i < n ? i : 0xFFFFFFFFu;
    if (i < n) sm_flag[i] = 0;
  }
  __syncthreads();
  if (!threshold) {
    for (uint32_t size = 2; size <= P; size <<= 1) {
      for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
        for (uint32_t t = threadIdx.x; t < (P >> 1); t += kSmallThreads) {
          const uint32_t lo = 2 * t - (t & (stride - 1));
          const uint32_t hi = lo + stride;
          const bool up = (lo & size) == 0;
          const unsigned long long ka = sm_keys[lo], kb = sm_keys[hi];
          const uint32_t ia = sm_idx[lo], ib = sm_idx[hi];
          const bool greater = ka > kb || (ka == kb && ia > ib);
          if (greater == up) {
            sm_keys[lo] = kb;
            sm_keys[hi] = ka;
            sm_idx[lo] = ib;
            sm_idx[hi] = ia;
          }
        }
        __syncthreads();
      }
    }
    for (uint32_t t = threadIdx.x; t < k; t += kSmallThreads) sm_flag[sm_idx[t]] = 1;
  } else {
    for (uint32_t i = threadIdx.x; i < n; i += kSmallThreads) sm_flag[i] = sm_keys[i] <= cut_thr;
  }
  __syncthreads();
  // Compaction in index order: thread t owns indices 4t .. 4t+3.
  unsigned int flags = 0;
#pragma unroll
  for (int q = 0; q < kSmallPer; ++q) {
    const uint32_t i = threadIdx.x * kSmallPer + q;
    if (i < n && sm_flag[i]) flags |= 1u << q;
  }
  unsigned int total;
  const unsigned int pos0 = block_exclusive_scan<unsigned int>(__popc(flags), &total, scan_smem);
  float th[kSmallPer][3];
  double sum[3] = {0.0, 0.0, 0.0};
  unsigned long long pos = pos0;
#pragma unroll
  for (int q = 0; q < kSmallPer; ++q) {
    if (flags & (1u << q)) {
      const uint32_t i = threadIdx.x * kSmallPer + q;
      float a, b, c;
      if (kTheta) {
        a = theta[i];
        b = theta[static_cast<size_t>(n) + i];
        c = theta[2 * static_cast<size_t>(n) + i];
      } else {
        ou_prior(prm, base + i, a, b, c);
      }
      th[q][0] = a;
      th[q][1] = b;
      th[q][2] = c;
      sum[0] += a;
      sum[1] += b;
      sum[2] += c;
      if (pos < cap) {
        idx_out[pos] = i;
        rec_out[pos] = make_float4(a, b, c, static_cast<float>(dist[i]));
      }
      ++pos;
    }
  }
  double mean[3], var[3];
  for (int d = 0; d < 3; ++d) {
    const double tsum = block_sum_fixed<double>(sum[d], red);
    mean[d] = total ? tsum / static_cast<double>(total) : 0.0;
  }
  for (int d = 0; d < 3; ++d) {
    double m2 = 0.0;
#pragma unroll
    for (int q = 0; q < kSmallPer; ++q) {
      if (flags & (1u << q)) {
        const double r = static_cast<double>(th[q][d]) - mean[d];
        m2 = fma(r, r, m2);
      }
    }
    var[d] = block_sum_fixed<double>(m2, red);
  }
  if (threadIdx.x == 0) {
    *n_acc_out = total;
    if (eps_out) *eps_out = threshold ? eps_thr : key_to_double(sm_keys[k - 1]);
    if (post_out) {
      for (int d = 0; d < 3; ++d) {
        post_out[d] = total > 0 ? mean[d] : nan("");
        post_out[3 + d] = total > 1 ? var[d] / static_cast<double>(total - 1) : nan("");
      }
    }
  }
}

unsigned long long host_dist_key(double d) {
  if (d != d) return 0xFFFFFFFFFFFFFFFFull;
  unsigned long long b;
  memcpy(&b, &d, sizeof(b));
  if (b == 0x8000000000000000ull) b = 0ull;
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

}  // namespace

size_t select_workspace_bytes(uint64_t n) { return WsLayout(n).total; }

cudaError_t launch_select(const double* dist, uint32_t n, uint64_t k, double eps,
                          const OUConst& P_, uint64_t base, const float* theta, uint32_t* idx_out,
                          float* rec_out, uint64_t cap, uint64_t* n_acc_out, double* eps_out,
                          double* post_out, void* ws, cudaStream_t s) {
  const bool threshold = (k == 0);
  if (n > 0 && n <= static_cast<uint32_t>(kSmallMax)) {
    uint32_t P = 2;
    while (P < n) P <<= 1;
    const size_t smem = P * (sizeof(unsigned long long) + sizeof(uint32_t)) + ((n + 15) & ~15u);
    const unsigned long long cut = threshold ? host_dist_key(eps) : 0ull;
    cudaError_t e;
    if (theta) {
      e = cudaFuncSetAttribute(select_small<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(smem));
      if (e != cudaSuccess) return e;
      select_small<true><<<1, kSmallThreads, smem, s>>>(
          dist, n, P, k, threshold, cut, eps, P_, static_cast<uint32_t>(base), theta, idx_out,
          reinterpret_cast<float4*>(rec_out), cap, reinterpret_cast<unsigned long long*>(n_acc_out),
          eps_out, post_out);
    } else {
      e = cudaFuncSetAttribute(select_small<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(smem));
      if (e != cudaSuccess) return e;
      select_small<false><<<1, kSmallThreads, smem, s>>>(
          dist, n, P, k, threshold, cut, eps, P_, static_cast<uint32_t>(base), theta, idx_out,
          reinterpret_cast<float4*>(rec_out), cap, reinterpret_cast<unsigned long long*>(n_acc_out),
          eps_out, post_out);
    }
    return cudaGetLastError();
  }
  const WsLayout L(n);
  char* w = static_cast<char*>(ws);
  SelState* st = reinterpret_cast<SelState*>(w + L.state);
  unsigned int* hist = reinterpret_cast<unsigned int*>(w + L.hist);
  unsigned int* tile_less = reinterpret_cast<unsigned int*>(w + L.tile_less);
  unsigned int* tile_eq = reinterpret_cast<unsigned int*>(w + L.tile_eq);
  unsigned int* tile_off = reinterpret_cast<unsigned int*>(w + L.tile_off);
  MomentPart* parts = reinterpret_cast<MomentPart*>(w + L.parts);
  const uint32_t tiles = static_cast<uint32_t>((static_cast<uint64_t>(n) + kTile - 1) / kTile);
  const unsigned long long cut_thr = threshold ? host_dist_key(eps) : 0ull;

  select_init<<<1, kHistThreads, 0, s>>>(st, hist, k);
  if (!threshold) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t want = (n + kHistThreads * 8 - 1) / (kHistThreads * 8);
    const uint32_t cap_blocks = static_cast<uint32_t>(sms > 0 ? sms : 1) * 8u;
    const uint32_t blocks = want < 1 ? 1 : (want > cap_blocks ? cap_blocks : want);
    for (int pass = 0; pass < kNumPasses; ++pass)
      select_hist<<<blocks, kHistThreads, 0, s>>>(dist, n, pass, st, hist);
  }
  if (tiles > 0) {
    select_count<<<tiles, kTileThreads, 0, s>>>(dist, n, st, threshold, cut_thr, tile_less, tile_eq);
  }
  select_scan<<<1, kTileThreads, 0, s>>>(st, threshold, cut_thr, eps, tile_less, tile_eq, tile_off,
                                         tiles, reinterpret_cast<unsigned long long*>(n_acc_out),
                                         eps_out);
  if (tiles > 0) {
    if (theta)
      select_write<true><<<tiles, kTileThreads, 0, s>>>(
          dist, n, st, threshold, cut_thr, tile_eq, tile_off, P_, static_cast<uint32_t>(base), theta,
          idx_out, reinterpret_cast<float4*>(rec_out), cap, parts);
    else
      select_write<false><<<tiles, kTileThreads, 0, s>>>(
          dist, n, st, threshold, cut_thr, tile_eq, tile_off, P_, static_cast<uint32_t>(base), theta,
          idx_out, reinterpret_cast<float4*>(rec_out), cap, parts);
  }
  if (post_out) select_moments<<<1, kTileThreads, 0, s>>>(parts, tiles, post_out);
  return cudaGetLastError();
}

}  // namespace ppabc
