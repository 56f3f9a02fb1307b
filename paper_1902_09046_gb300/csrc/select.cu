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
// the cut.  Ties at the cut go to the smaller index in both modes.  Up to
// 24576 distances one CTA runs the same radix select and a round-by-round
// compaction: a single launch for the many small jobs of a serving mix.
#include <math.h>
#include <string.h>

#include "dfloat.cuh"
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
// the largest key.  Integer operations only (a binary64 NaN test would go to
// this GPU's narrow FP64 pipe, which a one-CTA selection feels).
__device__ __forceinline__ unsigned long long dist_key(double d) {
  unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(d));
  if ((b & 0x7FFFFFFFFFFFFFFFull) > 0x7FF0000000000000ull) return 0xFFFFFFFFFFFFFFFFull;  // NaN
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

// Posterior mean and variance from the per-thread double-float sums of
// (theta - c) and (theta - c)^2 about a shift c (the first accepted theta):
// a fixed-order warp shuffle tree, then the warps in order in thread 0;
// mean = c + S1 / k and M2 = S2 - S1^2 / k in binary64.  Everything before
// the last step runs on the binary32 pipes (a one-CTA binary64 reduction
// would queue on this GPU's narrow FP64 pipe).  s_S1, s_S2 hold one value
// per warp and dimension; the result is written by thread 0.
template <int kWarps>
__device__ __forceinline__ void finish_moments(DF (&S1)[3], DF (&S2)[3], const float (&c)[3],
                                               unsigned long long k, DF (*s_S1)[kWarps], DF (*s_S2)[kWarps],
                                               double* post_out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      S1[d] = df_add(S1[d], DF{__shfl_xor_sync(0xFFFFFFFFu, S1[d].hi, o), __shfl_xor_sync(0xFFFFFFFFu, S1[d].lo, o)});
      S2[d] = df_add(S2[d], DF{__shfl_xor_sync(0xFFFFFFFFu, S2[d].hi, o), __shfl_xor_sync(0xFFFFFFFFu, S2[d].lo, o)});
    }
    if (lane == 0) {
      s_S1[d][warp] = S1[d];
      s_S2[d][warp] = S2[d];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && post_out) {
    const double kk = static_cast<double>(k);
    for (int d = 0; d < 3; ++d) {
      DF a = DF{0.0f, 0.0f}, b = DF{0.0f, 0.0f};
      for (int w = 0; w < kWarps; ++w) {
        a = df_add(a, s_S1[d][w]);
        b = df_add(b, s_S2[d][w]);
      }
      const double s1 = df_to_double(a), s2 = df_to_double(b);
      post_out[d] = k > 0 ? static_cast<double>(c[d]) + s1 / kk : nan("");
      post_out[3 + d] = k > 1 ? (s2 - s1 * s1 / kk) / (kk - 1.0) : nan("");
    }
  }
}

// Adds (theta - c) and (theta - c)^2 to the double-float sums; each
// difference is exact as a two-sum.
__device__ __forceinline__ void add_moment(DF (&S1)[3], DF (&S2)[3], const float (&th)[3], const float (&c)[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const DF r = df_two_sum(th[d], -c[d]);
    S1[d] = df_add(S1[d], r);
    S2[d] = df_add(S2[d], df_sqr(r));
  }
}


// ---------------------------------------------------------------------------
// Up to kMidMax distances: the whole selection in one CTA, reading the
// distances from global memory (L2) on every pass.  The
// radix select of the large path (six 11-bit passes with warp-aggregated
// shared histograms) runs in the CTA; the compaction walks the indices in
// rounds of 16 per thread, carrying the equal-key rank and the output
// position from round to round; the moments are double-float sums about the
// first accepted theta (binary32 pipes: a one-CTA binary64 reduction would
// queue on this GPU's narrow FP64 pipe).  One launch instead of eleven.
// ---------------------------------------------------------------------------
constexpr int kMidThreads = 1024;
constexpr uint32_t kMidMax = 24576;  // above this the multi-CTA passes are faster
constexpr int kMidPer = 16;
constexpr uint32_t kMidRound = kMidThreads * kMidPer;

template <bool kTheta>
__global__ void __launch_bounds__(kMidThreads) select_mid(
    const double* __restrict__ dist, uint32_t n, unsigned long long k, bool threshold,
    unsigned long long cut_thr, double eps_thr, const __grid_constant__ OUConst prm, uint32_t base,
    const float* __restrict__ theta, uint32_t* __restrict__ idx_out, float4* __restrict__ rec_out,
    unsigned long long cap, unsigned long long* __restrict__ n_acc_out, double* __restrict__ eps_out,
    double* __restrict__ post_out) {
  __shared__ unsigned int h[kBins];
  __shared__ unsigned int scan_smem[kMidThreads / 32];
  __shared__ unsigned long long scan64[kMidThreads / 32];
  __shared__ unsigned long long s_prefix, s_mask, s_krem;
  __shared__ unsigned int acc_bits[kMidMax / 32];
  __shared__ float s_shift[3];
  __shared__ DF s_S1[3][kMidThreads / 32], s_S2[3][kMidThreads / 32];
  const int lane = threadIdx.x & 31;
  unsigned long long prefix = 0ull, mask = 0ull, krem = k;
  // 1. Radix select of the k-th smallest key (skipped in threshold mode).
  if (!threshold) {
    for (int pass = 0; pass < kNumPasses; ++pass) {
      const int shift = kPassShift[pass];
      const unsigned long long dmask = (1ull << kPassBits[pass]) - 1ull;
      for (int b = threadIdx.x; b < kBins; b += kMidThreads) h[b] = 0u;
      __syncthreads();
      for (uint32_t b0 = 0; b0 < n; b0 += kMidThreads) {  // uniform bound: every lane reaches the match
        const uint32_t i = b0 + threadIdx.x;
        unsigned int bin = 0xFFFFFFFFu;
        if (i < n) {
          const unsigned long long key = dist_key(__ldg(dist + i));
          if ((key & mask) == prefix) bin = static_cast<unsigned int>((key >> shift) & dmask);
        }
        const unsigned int peers = __match_any_sync(0xFFFFFFFFu, bin);
        if (bin != 0xFFFFFFFFu && lane == __ffs(peers) - 1) atomicAdd(&h[bin], __popc(peers));
      }
      __syncthreads();
      constexpr int kPer = kBins / kMidThreads;  // bins owned by one thread
      unsigned int c[kPer];
      unsigned int mine = 0;
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        c[q] = h[threadIdx.x * kPer + q];
        mine += c[q];
      }
      unsigned int total;
      const unsigned int before = block_exclusive_scan<unsigned int>(mine, &total, scan_smem);
      if (before < krem && krem <= static_cast<unsigned long long>(before) + mine) {
        unsigned long long run = before;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
          if (run < krem && krem <= run + c[q]) {
            s_prefix = prefix | (static_cast<unsigned long long>(threadIdx.x * kPer + q) << shift);
            s_mask = mask | (dmask << shift);
            s_krem = krem - run;
          }
          run += c[q];
        }
      }
      __syncthreads();
      prefix = s_prefix;
      mask = s_mask;
      krem = s_krem;
    }
  }
  const unsigned long long cut = threshold ? cut_thr : prefix;
  if (threshold) krem = 0xFFFFFFFFFFFFFFFFull;
  // 2. Compaction in index order, 16 consecutive indices per thread and round;
  // the accepted indices are also marked in a bit set for the moments.
  for (uint32_t w = threadIdx.x; w < kMidMax / 32; w += kMidThreads) acc_bits[w] = 0u;
  if (threadIdx.x < 3) s_shift[threadIdx.x] = 0.0f;
  __syncthreads();
  unsigned long long carry_eq = 0ull, carry_acc = 0ull;
  for (uint32_t rb = 0; rb < n; rb += kMidRound) {
    const uint32_t t0 = rb + threadIdx.x * kMidPer;
    unsigned int flags = 0, eqmask = 0, my_eq = 0;
#pragma unroll
    for (int q = 0; q < kMidPer; ++q) {
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
    unsigned long long tot_eq;
    const unsigned long long eq_rank0 =
        carry_eq + block_exclusive_scan<unsigned long long>(my_eq, &tot_eq, scan64);
    {
      unsigned long long r = eq_rank0;
#pragma unroll
      for (int q = 0; q < kMidPer; ++q) {
        if (eqmask & (1u << q)) {
          if (r < krem) flags |= 1u << q;
          ++r;
        }
      }
    }
    unsigned long long tot_acc;
    unsigned long long pos =
        carry_acc + block_exclusive_scan<unsigned long long>(__popc(flags), &tot_acc, scan64);
    // 16 indices starting at a multiple of 16: half of one bit-set word
    if (flags) atomicOr(&acc_bits[t0 >> 5], flags << (t0 & 16u));
#pragma unroll
    for (int q = 0; q < kMidPer; ++q) {
      if (flags & (1u << q)) {
        const uint32_t i = t0 + q;
        float th[3];
        if (kTheta) {
          th[0] = theta[i];
          th[1] = theta[static_cast<size_t>(n) + i];
          th[2] = theta[2 * static_cast<size_t>(n) + i];
        } else {
          ou_prior(prm, base + i, th[0], th[1], th[2]);
        }
        if (pos == 0) {
          s_shift[0] = th[0];
          s_shift[1] = th[1];
          s_shift[2] = th[2];
        }
        if (pos < cap) {
          idx_out[pos] = i;
          rec_out[pos] = make_float4(th[0], th[1], th[2], static_cast<float>(dist[i]));
        }
        ++pos;
      }
    }
    carry_eq += tot_eq;
    carry_acc += tot_acc;
  }
  __syncthreads();
  // 3. Moments about the first accepted theta c: the sums of (theta - c) and
  // (theta - c)^2 in double-float (each difference exact as a two-sum), per
  // thread in index order, then a fixed-order tree over the CTA;
  // mean = c + S1 / k and M2 = S2 - S1^2 / k in binary64.  The accepted theta
  // are formed again from their counters (or read again).
  const float cs[3] = {s_shift[0], s_shift[1], s_shift[2]};
  DF S1[3] = {DF{0.0f, 0.0f}, DF{0.0f, 0.0f}, DF{0.0f, 0.0f}};
  DF S2[3] = {DF{0.0f, 0.0f}, DF{0.0f, 0.0f}, DF{0.0f, 0.0f}};
  for (uint32_t rb = 0; rb < n; rb += kMidRound) {
    const uint32_t t0 = rb + threadIdx.x * kMidPer;
    const unsigned int flags = t0 < n ? (acc_bits[t0 >> 5] >> (t0 & 16u)) & 0xFFFFu : 0u;
#pragma unroll 1
    for (int q = 0; q < kMidPer; ++q) {
      if (flags & (1u << q)) {
        const uint32_t i = t0 + q;
        float th[3];
        if (kTheta) {
          th[0] = theta[i];
          th[1] = theta[static_cast<size_t>(n) + i];
          th[2] = theta[2 * static_cast<size_t>(n) + i];
        } else {
          ou_prior(prm, base + i, th[0], th[1], th[2]);
        }
        add_moment(S1, S2, th, cs);
      }
    }
  }
  finish_moments<kMidThreads / 32>(S1, S2, cs, carry_acc, s_S1, s_S2, post_out);
  if (threadIdx.x == 0) {
    *n_acc_out = carry_acc;
    if (eps_out) *eps_out = threshold ? eps_thr : key_to_double(cut);
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
  if (n > 0 && n <= kMidMax) {
    const unsigned long long cut = threshold ? host_dist_key(eps) : 0ull;
    if (theta)
      select_mid<true><<<1, kMidThreads, 0, s>>>(dist, n, k, threshold, cut, eps, P_, static_cast<uint32_t>(base),
                                                 theta, idx_out, reinterpret_cast<float4*>(rec_out), cap,
                                                 reinterpret_cast<unsigned long long*>(n_acc_out), eps_out,
                                                 post_out);
    else
      select_mid<false><<<1, kMidThreads, 0, s>>>(dist, n, k, threshold, cut, eps, P_, static_cast<uint32_t>(base),
                                                  theta, idx_out, reinterpret_cast<float4*>(rec_out), cap,
                                                  reinterpret_cast<unsigned long long*>(n_acc_out), eps_out,
                                                  post_out);
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
