// select.cu -- accepted set of ABC rejection and posterior moments.
//
// The paper fixes N and then picks epsilon a posteriori from the empirical
// distribution of the discrepancy (Sec. 3.1): accepting the k nearest means
// epsilon is the k-th smallest distance.  This file finds it with an exact
// MSD radix select over the order-preserving 64-bit image of each binary64
// distance (up to 6 histogram passes of 11/11/11/11/11/9 bits, ending once a
// single key is left under the fixed bits; the last CTA of a pass picks the
// digit, so no host round trip), then writes the accepted samples in index
// order with a two-level scan, and reduces the posterior mean and variance
// with Chan's pairwise update in a fixed order.
//
// Threshold mode (k = 0) skips the radix passes: the key of epsilon itself is
// the cut.  Ties at the cut go to the smaller index in both modes.  For the
// many small jobs of a serving mix, the whole selection runs in one launch
// from shared memory: up to 12288 distances in one CTA, up to 196608 in a
// thread-block cluster of eight CTAs that pool their shared memory.
#include <math.h>
#include <string.h>

#include <atomic>

#include <cooperative_groups.h>

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
constexpr int kHistChunk = 4;  // histogram loads in flight per thread
__constant__ int kPassShift[kNumPasses] = {53, 42, 31, 20, 9, 0};
__constant__ int kPassBits[kNumPasses] = {11, 11, 11, 11, 11, 9};

struct SelState {
  unsigned long long prefix;  // key bits fixed so far
  unsigned long long mask;    // which bits of prefix are fixed
  unsigned long long krem;    // rank still to reach among keys matching prefix
  unsigned int ticket;        // CTAs done in the current pass
  unsigned int done;          // one key matches prefix: the later passes return at once
  unsigned long long n_acc;
  unsigned long long cut;     // full key of the k-th smallest, found by select_count once done
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
__device__ __forceinline__ unsigned long long key_of_bits(unsigned long long b) {
  if ((b & 0x7FFFFFFFFFFFFFFFull) > 0x7FF0000000000000ull) return 0xFFFFFFFFFFFFFFFFull;  // NaN
  if (b == 0x8000000000000000ull) b = 0ull;
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ unsigned long long dist_key(double d) {
  return key_of_bits(static_cast<unsigned long long>(__double_as_longlong(d)));
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
    st->done = 0u;
    st->n_acc = 0ull;
    st->cut = 0ull;
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
// krem and narrows the prefix.  Once that digit's bin holds a single key, the
// k-th smallest is the one key matching the prefix, and the passes left
// return without reading the distances.
__global__ void __launch_bounds__(kHistThreads) select_hist(const double* __restrict__ dist,
                                                            uint32_t n, int pass, SelState* st,
                                                            unsigned int* hist) {
  __shared__ unsigned int h[kBins];
  __shared__ bool is_last;
  __shared__ unsigned int scan_smem[8];
  if (st->done) return;
  const int shift = kPassShift[pass];
  const unsigned long long dmask = (1ull << kPassBits[pass]) - 1ull;
  for (int b = threadIdx.x; b < kBins; b += kHistThreads) h[b] = 0u;
  const unsigned long long prefix = st->prefix;
  const unsigned long long mask = st->mask;
  __syncthreads();
  // The loop bound is uniform across the CTA so every lane reaches the match.
  const int lane = threadIdx.x & 31;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kHistThreads;
  for (uint64_t b0 = static_cast<uint64_t>(blockIdx.x) * kHistThreads; b0 < n; b0 += stride * kHistChunk) {
    // kHistChunk keys loaded and binned per thread before their histogram
    // adds, so that the loads are in flight together
    unsigned int bin[kHistChunk];
#pragma unroll
    for (int j = 0; j < kHistChunk; ++j) {
      const uint64_t i = b0 + j * stride + threadIdx.x;
      const unsigned long long key = i < n ? dist_key(__ldg(dist + i)) : 0ull;
      bin[j] = (i < n && (key & mask) == prefix) ? static_cast<unsigned int>((key >> shift) & dmask)
                                                 : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int j = 0; j < kHistChunk; ++j) {
      // Distances crowd into few bins on the early passes: one shared atomic
      // per distinct bin in the warp.  On the later passes few keys match the
      // prefix, and warps without one skip the match.
      if (__any_sync(0xFFFFFFFFu, bin[j] != 0xFFFFFFFFu)) {
        const unsigned int peers = __match_any_sync(0xFFFFFFFFu, bin[j]);
        if (bin[j] != 0xFFFFFFFFu && lane == __ffs(peers) - 1) atomicAdd(&h[bin[j]], __popc(peers));
      }
    }
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
        if (c[q] == 1u) st->done = 1u;
      }
      run += c[q];
    }
  }
  if (threadIdx.x == 0) st->ticket = 0u;
}

// Per-tile counts of keys below and at the cut.
__global__ void __launch_bounds__(kTileThreads) select_count(const double* __restrict__ dist,
                                                             uint32_t n, SelState* st,
                                                             bool threshold,
                                                             unsigned long long cut_thr,
                                                             unsigned int* tile_less,
                                                             unsigned int* tile_eq) {
  __shared__ unsigned int s_less[kTileThreads / 32], s_eq[kTileThreads / 32];
  // Keys compare with the cut on the bits the passes fixed (all of them
  // unless the passes stopped early, when one key matches there).
  const unsigned long long cut = threshold ? cut_thr : st->prefix;
  const unsigned long long cmask = threshold ? 0xFFFFFFFFFFFFFFFFull : st->mask;
  const uint32_t t0 = blockIdx.x * kTile;
  unsigned int less = 0, eq = 0;
#pragma unroll 4
  for (int q = 0; q < kPerThread; ++q) {
    const uint32_t i = t0 + q * kTileThreads + threadIdx.x;  // coalesced
    if (i < n) {
      const unsigned long long key = dist_key(__ldg(dist + i));
      less += (key & cmask) < cut;
      if ((key & cmask) == cut) {
        ++eq;
        if (cmask != 0xFFFFFFFFFFFFFFFFull) st->cut = key;  // the one matching key
      }
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
// 1024 threads: a pass over 4096 tiles takes four rounds of block scans
// instead of sixteen (8 us less per selection of 2^24 distances).
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) select_scan(
    SelState* st, bool threshold, unsigned long long cut_thr, double eps_thr,
    const unsigned int* tile_less, unsigned int* tile_eq /* in: equal count, out: equal base */,
    unsigned int* tile_off, uint32_t tiles, unsigned long long* n_acc_out, double* eps_out) {
  __shared__ unsigned long long smem[kScanThreads / 32];
  __shared__ unsigned long long carry_eq, carry_acc;
  const unsigned long long krem = threshold ? 0xFFFFFFFFFFFFFFFFull : st->krem;
  if (threadIdx.x == 0) {
    carry_eq = 0ull;
    carry_acc = 0ull;
  }
  __syncthreads();
  for (uint32_t base = 0; base < tiles; base += kScanThreads) {
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
    if (eps_out)
      *eps_out = threshold ? eps_thr : key_to_double(st->mask == 0xFFFFFFFFFFFFFFFFull ? st->prefix : st->cut);
  }
}

// Writes the accepted samples of one tile in index order and the tile's
// (count, mean, M2) of theta.
// Four CTAs per SM (64 registers, a few hundred bytes of spills): a tile is
// latency-bound, and the occupancy pays more than the spills cost (416 ->
// 381 us for the whole selection of 2^24 distances, against two CTAs per SM
// at 128-141 registers).
template <bool kTheta>
__global__ void __launch_bounds__(kTileThreads, 4) select_write(
    const double* __restrict__ dist, uint32_t n, const SelState* st, bool threshold,
    unsigned long long cut_thr, const unsigned int* __restrict__ tile_eq_base,
    const unsigned int* __restrict__ tile_off, const __grid_constant__ OUConst P, uint32_t base,
    const float* __restrict__ theta, uint32_t* __restrict__ idx_out, float4* __restrict__ rec_out,
    unsigned long long cap, MomentPart* __restrict__ parts) {
  __shared__ unsigned int scan_smem[8];
  __shared__ double red[3][kTileThreads / 32];
  __shared__ double s_mean[3];
  const unsigned long long cut = threshold ? cut_thr : st->prefix;
  const unsigned long long cmask = threshold ? 0xFFFFFFFFFFFFFFFFull : st->mask;
  const unsigned long long krem = threshold ? 0xFFFFFFFFFFFFFFFFull : st->krem;
  const uint32_t t0 = blockIdx.x * kTile + threadIdx.x * kPerThread;  // contiguous per thread
  // pass 1: flags and per-thread counts
  unsigned int flags = 0, eqmask = 0, my_eq = 0;
  unsigned long long key[kPerThread];  // all loads in flight before the compares
#pragma unroll
  for (int q = 0; q < kPerThread; ++q) key[q] = t0 + q < n ? dist_key(__ldg(dist + t0 + q)) : 0ull;
#pragma unroll
  for (int q = 0; q < kPerThread; ++q) {
    if (t0 + q < n) {
      if ((key[q] & cmask) < cut) flags |= 1u << q;
      if ((key[q] & cmask) == cut) {
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
  // tile mean (fixed-order reduction), then M2 about it; a warp without an
  // accepted sample contributes zeros without its binary64 shuffles (the
  // same sums: its shuffle tree would add zeros only).
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool warp_any = __any_sync(0xFFFFFFFFu, flags != 0u);
  for (int d = 0; d < 3; ++d) {
    double v = sum[d];
    if (warp_any) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    }
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
    if (warp_any) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    }
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
  const double wb = nb / nab, wab = na * wb;  // one division per merge (the FP64 pipe is narrow here)
  for (int d = 0; d < 3; ++d) {
    const double delta = mb[d] - ma[d];
    ma[d] = ma[d] + delta * wb;
    qa[d] = qa[d] + qb[d] + delta * delta * wab;
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

// a / b for a double-float a and a binary32 b != 0: the binary32 quotient of
// the leading parts, corrected once by the residual a - q b (relative error
// about 2^-46).
__device__ __forceinline__ DF df_div_f(DF a, float b) {
  const float q1 = __fdiv_rn(a.hi, b);
  const DF r = df_add(a, df_neg(df_two_prod(q1, b)));
  return df_fast_two_sum(q1, __fdiv_rn(r.hi, b));
}

// Posterior mean and variance from double-float sums of (theta - c_w) and
// (theta - c_w)^2 about a shift c_w per warp (its first accepted theta; nw
// accepted samples): a fixed-order shuffle tree in each warp with any, then
// warp 0 moves each warp's sums to the common shift c (the first accepted
// theta overall, s_c0) -- with d = c_w - c exact as a two-sum,
//   sum (theta - c) = S1 + nw d,   sum (theta - c)^2 = S2 + d (S1 + sum (theta - c)),
// -- and sums them over the warps with the same tree; lane d of warp 0
// finishes dimension d: mean = c + S1 / k and M2 = S2 - S1 (S1 / k), both in
// double-float.  Everything runs on the binary32 pipes (a one-CTA binary64
// reduction would queue on this GPU's narrow FP64 pipe, which a chain of
// binary64 divisions there did), and the trees are rolled loops: this one-CTA kernel runs each instruction
// once, so its time follows its code size.  s_S1, s_S2, s_cw hold one value
// per warp and dimension, s_nw one count per warp (kWarps <= 32).
// cta_moment_sums is the part up to the CTA's totals (returns true in warp 0,
// whose lanes then all hold them); store_moments the finish.
template <int kWarps>
__device__ __forceinline__ bool cta_moment_sums(DF (&S1)[3], DF (&S2)[3], const float (&cw)[3], unsigned int nw,
                                                DF (*s_S1)[kWarps], DF (*s_S2)[kWarps], float (*s_cw)[kWarps],
                                                const unsigned int* s_nw, const float* s_c0) {
  static_assert(kWarps <= 32, "one warp sums the warps' partial sums");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (nw != 0u) {  // warp-uniform: the sums of a warp without accepted samples are zero
#pragma unroll 1
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        S1[d] = df_add(S1[d], DF{__shfl_xor_sync(0xFFFFFFFFu, S1[d].hi, o), __shfl_xor_sync(0xFFFFFFFFu, S1[d].lo, o)});
        S2[d] = df_add(S2[d], DF{__shfl_xor_sync(0xFFFFFFFFu, S2[d].hi, o), __shfl_xor_sync(0xFFFFFFFFu, S2[d].lo, o)});
      }
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      s_S1[d][warp] = S1[d];
      s_S2[d][warp] = S2[d];
      s_cw[d][warp] = cw[d];
    }
  }
  __syncthreads();
  if (warp != 0) return false;
  const unsigned int n_w = lane < kWarps ? s_nw[lane] : 0u;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    S1[d] = DF{0.0f, 0.0f};
    S2[d] = DF{0.0f, 0.0f};
    if (n_w != 0u) {
      const DF a = s_S1[d][lane], b = s_S2[d][lane];
      const DF dlt = df_two_sum(s_cw[d][lane], -s_c0[d]);
      S1[d] = df_add(a, df_mul_f(dlt, static_cast<float>(n_w)));
      S2[d] = df_add(b, df_mul(dlt, df_add(a, S1[d])));
    }
  }
#pragma unroll 1
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      S1[d] = df_add(S1[d], DF{__shfl_xor_sync(0xFFFFFFFFu, S1[d].hi, o), __shfl_xor_sync(0xFFFFFFFFu, S1[d].lo, o)});
      S2[d] = df_add(S2[d], DF{__shfl_xor_sync(0xFFFFFFFFu, S2[d].hi, o), __shfl_xor_sync(0xFFFFFFFFu, S2[d].lo, o)});
    }
  }
  return true;
}

// mean = c + S1 / k and the unbiased variance (S2 - S1 (S1 / k)) / (k - 1)
// from the totals about the shift s_c0, written by lanes 0..2 (dimension =
// lane).
__device__ __forceinline__ void store_moments(const DF (&S1)[3], const DF (&S2)[3], unsigned long long k,
                                              const float* s_c0, double* post_out) {
  const int lane = threadIdx.x & 31;
  if (lane < 3 && post_out) {
    const DF a = lane == 0 ? S1[0] : (lane == 1 ? S1[1] : S1[2]);
    const DF b = lane == 0 ? S2[0] : (lane == 1 ? S2[1] : S2[2]);
    const float kf = static_cast<float>(k);  // exact: k <= 2^24
    const DF m = df_div_f(a, kf);           // S1 / k
    post_out[lane] = k > 0 ? df_to_double(df_add_f(m, s_c0[lane])) : nan("");
    post_out[3 + lane] = k > 1 ? df_to_double(df_div_f(df_add(b, df_neg(df_mul(a, m))), kf - 1.0f)) : nan("");
  }
}

template <int kWarps>
__device__ __forceinline__ void finish_moments(DF (&S1)[3], DF (&S2)[3], const float (&cw)[3], unsigned int nw,
                                               unsigned long long k, DF (*s_S1)[kWarps], DF (*s_S2)[kWarps],
                                               float (*s_cw)[kWarps], const unsigned int* s_nw,
                                               const float* s_c0, double* post_out) {
  if (cta_moment_sums<kWarps>(S1, S2, cw, nw, s_S1, s_S2, s_cw, s_nw, s_c0)) store_moments(S1, S2, k, s_c0, post_out);
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
// Up to kMidMax distances: the whole selection in one CTA and one launch.
// The distances' bit patterns are read once into shared memory (a one-CTA
// kernel is bound by how many L2 reads one SM keeps in flight, so a pass
// over shared memory is several times cheaper than one over L2).  The radix
// select of the large path (up to six 11-bit passes, ending once a single
// key is left under the prefix) runs over them; the compaction gives each
// warp a block of consecutive indices, 32 at a time, so ranks in index order
// come from ballots and one scan over the warps' counts; with few accepted,
// their indices are listed first and then taken one per lane; the moments
// are double-float sums about per-warp shifts (binary32 pipes: a one-CTA
// binary64 reduction would queue on this GPU's narrow FP64 pipe).
// ---------------------------------------------------------------------------
constexpr int kMidThreads = 1024;
constexpr int kMidWarps = kMidThreads / 32;
constexpr uint32_t kMidMax = 24576;  // bit patterns in shared memory: 192 KB
constexpr int kMidChunk = 8;         // loads in flight per thread
constexpr uint32_t kMidList = kBins;  // accepted indices listed in the histogram's shared memory
constexpr size_t kMidKeyBytes = static_cast<size_t>(kMidMax) * sizeof(unsigned long long);

// Exclusive prefix over the warps of one value per warp (v[w], kMidWarps =
// 32 of them), computed by every warp for itself; *all = the sum.
static_assert(kMidWarps == 32, "one lane per warp of the CTA");
__device__ __forceinline__ unsigned int warp_base_of(const unsigned int* v, int warp, unsigned int* all) {
  const int lane = threadIdx.x & 31;
  const unsigned int x0 = v[lane];
  unsigned int x = x0;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  *all = __shfl_sync(0xFFFFFFFFu, x, 31);
  return __shfl_sync(0xFFFFFFFFu, x - x0, warp);
}

template <bool kTheta>
__global__ void __launch_bounds__(kMidThreads, 1) select_mid(
    const double* __restrict__ dist, uint32_t n, unsigned long long k, bool threshold,
    unsigned long long cut_thr, double eps_thr, const __grid_constant__ OUConst prm, uint32_t base,
    const float* __restrict__ theta, uint32_t* __restrict__ idx_out, float4* __restrict__ rec_out,
    unsigned long long cap, unsigned long long* __restrict__ n_acc_out, double* __restrict__ eps_out,
    double* __restrict__ post_out) {
  extern __shared__ unsigned long long s_raw[];  // the n distances' bit patterns
  __shared__ unsigned int h[kBins];
  __shared__ unsigned int scan_smem[kMidWarps];
  __shared__ unsigned long long s_prefix, s_mask, s_krem, s_cut;
  __shared__ unsigned int s_bin_count;
  __shared__ unsigned int acc_bits[kMidMax / 32];  // bit (i & 31) of word i >> 5: index i accepted
  __shared__ unsigned int s_weq[kMidWarps], s_wacc[kMidWarps];
  __shared__ float s_shift[3];
  __shared__ DF s_S1[3][kMidWarps], s_S2[3][kMidWarps];
  __shared__ float s_cw[3][kMidWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned int lane_lt = (1u << lane) - 1u;
  // 0. The distances into shared memory, kMidChunk loads in flight per
  // thread; their keys are formed where they are read.
  const unsigned long long* __restrict__ dbits = reinterpret_cast<const unsigned long long*>(dist);
  for (uint32_t i0 = 0; i0 < n; i0 += kMidThreads * kMidChunk) {
    unsigned long long t[kMidChunk];
#pragma unroll
    for (int j = 0; j < kMidChunk; ++j) {
      const uint32_t i = i0 + j * kMidThreads + threadIdx.x;
      t[j] = i < n ? __ldg(dbits + i) : 0ull;
    }
#pragma unroll
    for (int j = 0; j < kMidChunk; ++j) {
      const uint32_t i = i0 + j * kMidThreads + threadIdx.x;
      if (i < n) s_raw[i] = t[j];
    }
  }
  __syncthreads();
  unsigned long long prefix = 0ull, mask = 0ull, krem = k;
  // 1. Radix select of the k-th smallest key (skipped in threshold mode).
  if (!threshold) {
    for (int pass = 0; pass < kNumPasses; ++pass) {
      const int shift = kPassShift[pass];
      const unsigned long long dmask = (1ull << kPassBits[pass]) - 1ull;
      for (int b = threadIdx.x; b < kBins; b += kMidThreads) h[b] = 0u;
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < n; i += kMidThreads) {
        const unsigned long long key = key_of_bits(s_raw[i]);
        if ((key & mask) == prefix) atomicAdd(&h[static_cast<unsigned int>((key >> shift) & dmask)], 1u);
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
            s_bin_count = c[q];
          }
          run += c[q];
        }
      }
      __syncthreads();
      prefix = s_prefix;
      mask = s_mask;
      krem = s_krem;
      // One key left under the prefix: it is the k-th smallest, and the bits
      // fixed so far order every other key against it.
      if (s_bin_count == 1u) break;
    }
  }
  // Keys compare with the cut on the bits the passes fixed (all of them when
  // the passes ran out, as with ties); every key equal to the cut there has
  // the cut's full value (one such key if the passes stopped early), which
  // gives epsilon.
  const unsigned long long cut = threshold ? cut_thr : prefix;
  const unsigned long long cmask = threshold ? 0xFFFFFFFFFFFFFFFFull : mask;
  if (threshold) krem = 0xFFFFFFFFFFFFFFFFull;
  // 2. Compaction in index order: warp w takes the block [g0, g1) of
  // consecutive indices, 32 at a time (lane = index - g).  Where the keys
  // equal to the cut are split by the rank (ties across the k-th), one scan
  // over the warps gives their ranks; a second gives the output positions.
  if (threadIdx.x < 3) s_shift[threadIdx.x] = 0.0f;
  const uint32_t span = (n + kMidThreads - 1) / kMidThreads * 32u;  // a multiple of 32
  const uint32_t g0 = min(n, warp * span), g1 = min(n, g0 + span);  // warp-uniform
  const bool rank_eq = !threshold && krem < s_bin_count;            // CTA-uniform
  unsigned long long eq_rank = 0ull;  // equal keys before this warp's block
  if (rank_eq) {
    unsigned int weq = 0;
    for (uint32_t g = g0; g < g1; g += 32u) {
      const uint32_t i = g + lane;
      weq += __popc(__ballot_sync(0xFFFFFFFFu, i < n && (key_of_bits(s_raw[i]) & cmask) == cut));
    }
    if (lane == 0) s_weq[warp] = weq;
    __syncthreads();
    unsigned int tot_eq;
    eq_rank = warp_base_of(s_weq, warp, &tot_eq);
  }
  unsigned int wacc = 0;
  for (uint32_t g = g0; g < g1; g += 32u) {
    const uint32_t i = g + lane;
    const unsigned long long full = i < n ? key_of_bits(s_raw[i]) : 0ull;
    const unsigned long long key = full & cmask;
    const bool less = i < n && key < cut;
    const bool eq = i < n && key == cut;
    if (eq) s_cut = full;
    const unsigned int eqb = __ballot_sync(0xFFFFFFFFu, eq);
    const bool take_eq = eq && (!rank_eq || eq_rank + __popc(eqb & lane_lt) < krem);
    const unsigned int accb = __ballot_sync(0xFFFFFFFFu, less || take_eq);
    if (lane == 0) acc_bits[g >> 5] = accb;
    eq_rank += __popc(eqb);
    wacc += __popc(accb);
  }
  if (lane == 0) s_wacc[warp] = wacc;
  __syncthreads();
  // 3. Output in index order, and the moments: each thread sums (theta - c_w)
  // and (theta - c_w)^2 in double-float (each difference exact as a
  // two-sum) about its warp's first accepted theta c_w; the warps' sums are
  // moved to the first accepted theta overall and added in a fixed order.
  unsigned int n_acc;
  unsigned long long pos = warp_base_of(s_wacc, warp, &n_acc);  // accepted before this warp's
  float cw[3] = {0.0f, 0.0f, 0.0f};
  bool have_cw = false;  // warp-uniform
  DF S1[3] = {DF{0.0f, 0.0f}, DF{0.0f, 0.0f}, DF{0.0f, 0.0f}};
  DF S2[3] = {DF{0.0f, 0.0f}, DF{0.0f, 0.0f}, DF{0.0f, 0.0f}};
  // theta of accepted index i at output position p, written out; the first
  // accepted theta overall is the moments' common shift.
  auto emit = [&](uint32_t i, unsigned long long p, float (&th)[3]) {
    if (kTheta) {
      th[0] = theta[i];
      th[1] = theta[static_cast<size_t>(n) + i];
      th[2] = theta[2 * static_cast<size_t>(n) + i];
    } else {
      ou_prior(prm, base + i, th[0], th[1], th[2]);
    }
    if (p == 0) {
      s_shift[0] = th[0];
      s_shift[1] = th[1];
      s_shift[2] = th[2];
    }
    if (p < cap) {
      idx_out[p] = i;
      rec_out[p] = make_float4(th[0], th[1], th[2], static_cast<float>(__longlong_as_double(s_raw[i])));
    }
  };
  // Lane q holds the bit-set word of the warp's q-th group (at most 32
  // groups) and the number accepted in the groups before it.
  static_assert(kMidMax / kMidThreads <= 32, "a warp's groups fit in one word per lane");
  const uint32_t n_groups = (g1 - g0 + 31u) / 32u;
  const unsigned int word = static_cast<uint32_t>(lane) < n_groups ? acc_bits[(g0 >> 5) + lane] : 0u;
  unsigned int before = __popc(word);
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int y = __shfl_up_sync(0xFFFFFFFFu, before, o);
    if (lane >= o) before += y;
  }
  before -= __popc(word);
  unsigned int busy = __ballot_sync(0xFFFFFFFFu, word != 0u);
  unsigned int nw;  // accepted samples this warp sums
  if (n_acc <= kMidList) {  // CTA-uniform
    // Few accepted: their indices go to a list in output order (in the
    // histogram's place), and then every lane takes one, so that the prior
    // draws and the sums run on full warps.
    unsigned int* list = h;
#pragma unroll 1
    while (busy != 0u) {  // warp-uniform
      const int q = __ffs(busy) - 1;
      busy &= busy - 1u;
      const unsigned int accb = __shfl_sync(0xFFFFFFFFu, word, q);
      const unsigned int bq = __shfl_sync(0xFFFFFFFFu, before, q);
      if ((accb >> lane) & 1u) list[pos + bq + __popc(accb & lane_lt)] = g0 + 32u * q + lane;
    }
    __syncthreads();
    unsigned int mine_count = 0;
#pragma unroll 1
    for (uint32_t p0 = warp * 32u; p0 < n_acc; p0 += kMidThreads) {  // warp-uniform
      const uint32_t p = p0 + lane;
      const bool mine = p < n_acc;
      float th[3] = {0.0f, 0.0f, 0.0f};
      if (mine) emit(list[p], p, th);
      if (!have_cw) {  // lane 0 holds the warp's first sample
#pragma unroll
        for (int d = 0; d < 3; ++d) cw[d] = __shfl_sync(0xFFFFFFFFu, th[d], 0);
        have_cw = true;
      }
      if (mine) {
        add_moment(S1, S2, th, cw);
        ++mine_count;
      }
    }
    nw = __reduce_add_sync(0xFFFFFFFFu, mine_count);
    if (lane == 0) s_wacc[warp] = nw;  // read again only by the moments
  } else {
    // Many accepted: the warp visits its groups that hold accepted samples.
#pragma unroll 1
    while (busy != 0u) {  // warp-uniform
      const int q = __ffs(busy) - 1;
      busy &= busy - 1u;
      const unsigned int accb = __shfl_sync(0xFFFFFFFFu, word, q);
      const unsigned long long pq = pos + __shfl_sync(0xFFFFFFFFu, before, q);
      const bool mine = (accb >> lane) & 1u;
      float th[3] = {0.0f, 0.0f, 0.0f};
      if (mine) emit(g0 + 32u * q + lane, pq + __popc(accb & lane_lt), th);
      if (!have_cw) {
        const int src = __ffs(accb) - 1;
#pragma unroll
        for (int d = 0; d < 3; ++d) cw[d] = __shfl_sync(0xFFFFFFFFu, th[d], src);
        have_cw = true;
      }
      if (mine) add_moment(S1, S2, th, cw);
    }
    nw = wacc;
  }
  finish_moments<kMidWarps>(S1, S2, cw, nw, n_acc, s_S1, s_S2, s_cw, s_wacc, s_shift, post_out);
  if (threadIdx.x == 0) {
    *n_acc_out = n_acc;
    if (eps_out) *eps_out = threshold ? eps_thr : key_to_double(s_cut);
  }
}

// ---------------------------------------------------------------------------
// kMidMax < n <= kClusterMax distances: the same selection in one launch of a
// thread-block cluster of kClusterCtas CTAs, which pools their shared memory.
// CTA r holds the bit patterns of the index slice [lo, hi) (equal slices, a
// multiple of 32 long, in index order).  A radix pass: every CTA builds the
// histogram of its slice; CTA r sums bins [r kBinsPerCta, (r+1) kBinsPerCta)
// over the cluster through distributed shared memory and posts their total
// in CTA 0; the CTA whose bins hold the k-th key posts the digit there, and
// every CTA reads it back.  The compaction runs per CTA as in select_mid,
// with the keys equal to the cut and the accepted ones before each slice
// counted from the CTAs' counts posted in CTA 0; the moments are summed per
// CTA about the first accepted theta overall, then over the CTAs in rank
// order.  Every thread takes part in every cluster barrier and none leaves
// before the last one, after which no CTA touches another's shared memory.
// ---------------------------------------------------------------------------
constexpr int kClusterCtas = 8;
constexpr uint32_t kClusterMax = kClusterCtas * kMidMax;
// Below about this many distances the one CTA is faster (no cluster
// barriers): 14.4 against 15.8 us at n = 10^4, 19.0 against 16.2 us at 16384.
constexpr uint32_t kOneCtaMax = 12288;
constexpr int kBinsPerCta = kBins / kClusterCtas;
static_assert(kBinsPerCta * kClusterCtas == kBins && kBinsPerCta <= kMidThreads, "bins split evenly over the CTAs");
static_assert(kClusterCtas <= 32, "one lane per CTA");

template <bool kTheta>
__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kMidThreads, 1) select_cluster(
    const double* __restrict__ dist, uint32_t n, unsigned long long k, bool threshold,
    unsigned long long cut_thr, double eps_thr, const __grid_constant__ OUConst prm, uint32_t base,
    const float* __restrict__ theta, uint32_t* __restrict__ idx_out, float4* __restrict__ rec_out,
    unsigned long long cap, unsigned long long* __restrict__ n_acc_out, double* __restrict__ eps_out,
    double* __restrict__ post_out) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const unsigned int rank = cluster.block_rank();
  extern __shared__ unsigned long long s_raw[];  // this CTA's slice of bit patterns
  __shared__ unsigned int h[kBins];
  __shared__ unsigned int scan_smem[kMidWarps];
  // CTA 0's copies of these are the cluster's: per-CTA counts, the digit
  // found (prefix, mask, rank left, its bin's count), the cut's full key and
  // the CTAs' moment sums.
  __shared__ unsigned int c_tot[kClusterCtas], c_eq[kClusterCtas], c_acc[kClusterCtas];
  __shared__ unsigned long long c_res[4];
  __shared__ unsigned long long s_cut;
  __shared__ DF c_S1[3 * kClusterCtas], c_S2[3 * kClusterCtas];
  __shared__ unsigned int s_cnt[kClusterCtas];  // a local copy of one of the count arrays
  __shared__ unsigned int acc_bits[kMidMax / 32];
  __shared__ unsigned int s_weq[kMidWarps], s_wacc[kMidWarps];
  __shared__ float s_shift[3];
  __shared__ DF s_S1[3][kMidWarps], s_S2[3][kMidWarps];
  __shared__ float s_cw[3][kMidWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned int lane_lt = (1u << lane) - 1u;
  const uint32_t L = ((n + kClusterCtas - 1) / kClusterCtas + 31u) & ~31u;
  const uint32_t lo = min(n, rank * L), hi = min(n, lo + L), m = hi - lo;
  unsigned int* const tot0 = cluster.map_shared_rank(c_tot, 0);
  unsigned int* const eq0 = cluster.map_shared_rank(c_eq, 0);
  unsigned int* const acc0 = cluster.map_shared_rank(c_acc, 0);
  unsigned long long* const res0 = cluster.map_shared_rank(c_res, 0);
  // set here, before the first cluster barrier: the CTA that emits output
  // position 0 writes every CTA's copy later
  if (threadIdx.x < 3) s_shift[threadIdx.x] = 0.0f;
  // 0. This CTA's slice into shared memory.
  const unsigned long long* __restrict__ dbits = reinterpret_cast<const unsigned long long*>(dist) + lo;
  for (uint32_t i0 = 0; i0 < m; i0 += kMidThreads * kMidChunk) {
    unsigned long long t[kMidChunk];
#pragma unroll
    for (int j = 0; j < kMidChunk; ++j) {
      const uint32_t i = i0 + j * kMidThreads + threadIdx.x;
      t[j] = i < m ? __ldg(dbits + i) : 0ull;
    }
#pragma unroll
    for (int j = 0; j < kMidChunk; ++j) {
      const uint32_t i = i0 + j * kMidThreads + threadIdx.x;
      if (i < m) s_raw[i] = t[j];
    }
  }
  __syncthreads();
  unsigned long long prefix = 0ull, mask = 0ull, krem = k, bin_count = 0ull;
  // 1. Radix select of the k-th smallest key over the cluster (skipped in
  // threshold mode).
  if (!threshold) {
    for (int pass = 0; pass < kNumPasses; ++pass) {
      const int shift = kPassShift[pass];
      const unsigned long long dmask = (1ull << kPassBits[pass]) - 1ull;
      for (int b = threadIdx.x; b < kBins; b += kMidThreads) h[b] = 0u;
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < m; i += kMidThreads) {
        const unsigned long long key = key_of_bits(s_raw[i]);
        if ((key & mask) == prefix) atomicAdd(&h[static_cast<unsigned int>((key >> shift) & dmask)], 1u);
      }
      cluster.sync();  // every CTA's histogram complete
      unsigned int mine = 0;
      if (threadIdx.x < kBinsPerCta) {
        const unsigned int bin = rank * kBinsPerCta + threadIdx.x;
#pragma unroll 1
        for (int r = 0; r < kClusterCtas; ++r) mine += cluster.map_shared_rank(h, r)[bin];
      }
      unsigned int total;
      const unsigned int before = block_exclusive_scan<unsigned int>(mine, &total, scan_smem);
      if (threadIdx.x == 0) tot0[rank] = total;
      cluster.sync();  // totals posted; no CTA reads another's histogram any more
      if (threadIdx.x < kClusterCtas) s_cnt[threadIdx.x] = tot0[threadIdx.x];
      __syncthreads();
      if (threadIdx.x < kBinsPerCta) {
        unsigned long long b0 = before;  // keys under the prefix in lower bins
        for (unsigned int r = 0; r < rank; ++r) b0 += s_cnt[r];
        if (b0 < krem && krem <= b0 + mine) {  // one thread in the cluster
          res0[0] = prefix | (static_cast<unsigned long long>(rank * kBinsPerCta + threadIdx.x) << shift);
          res0[1] = mask | (dmask << shift);
          res0[2] = krem - b0;
          res0[3] = mine;
        }
      }
      cluster.sync();  // the digit posted
      prefix = res0[0];
      mask = res0[1];
      krem = res0[2];
      bin_count = res0[3];
      if (bin_count == 1ull) break;  // cluster-uniform, as in select_mid
    }
  }
  const unsigned long long cut = threshold ? cut_thr : prefix;
  const unsigned long long cmask = threshold ? 0xFFFFFFFFFFFFFFFFull : mask;
  if (threshold) krem = 0xFFFFFFFFFFFFFFFFull;
  // 2. Compaction in index order within the slice (local index i = global
  // index - lo), warp w over the block [g0, g1) as in select_mid.
  const uint32_t span = (m + kMidThreads - 1) / kMidThreads * 32u;  // a multiple of 32
  const uint32_t g0 = min(m, warp * span), g1 = min(m, g0 + span);  // warp-uniform
  const bool rank_eq = !threshold && krem < bin_count;               // cluster-uniform
  unsigned long long eq_rank = 0ull;  // equal keys before this warp's block, over the cluster
  if (rank_eq) {
    unsigned int weq = 0;
    for (uint32_t g = g0; g < g1; g += 32u) {
      const uint32_t i = g + lane;
      weq += __popc(__ballot_sync(0xFFFFFFFFu, i < m && (key_of_bits(s_raw[i]) & cmask) == cut));
    }
    if (lane == 0) s_weq[warp] = weq;
    __syncthreads();
    unsigned int tot_eq;
    eq_rank = warp_base_of(s_weq, warp, &tot_eq);
    if (threadIdx.x == 0) eq0[rank] = tot_eq;
    cluster.sync();  // equal-key counts posted
    if (threadIdx.x < kClusterCtas) s_cnt[threadIdx.x] = eq0[threadIdx.x];
    __syncthreads();
    for (unsigned int r = 0; r < rank; ++r) eq_rank += s_cnt[r];
  }
  unsigned long long* const cut0 = cluster.map_shared_rank(&s_cut, 0);
  unsigned int wacc = 0;
  for (uint32_t g = g0; g < g1; g += 32u) {
    const uint32_t i = g + lane;
    const unsigned long long full = i < m ? key_of_bits(s_raw[i]) : 0ull;
    const unsigned long long key = full & cmask;
    const bool less = i < m && key < cut;
    const bool eq = i < m && key == cut;
    if (eq) *cut0 = full;  // every such key has the same full value
    const unsigned int eqb = __ballot_sync(0xFFFFFFFFu, eq);
    const bool take_eq = eq && (!rank_eq || eq_rank + __popc(eqb & lane_lt) < krem);
    const unsigned int accb = __ballot_sync(0xFFFFFFFFu, less || take_eq);
    if (lane == 0) acc_bits[g >> 5] = accb;
    eq_rank += __popc(eqb);
    wacc += __popc(accb);
  }
  if (lane == 0) s_wacc[warp] = wacc;
  __syncthreads();
  unsigned int n_cta;  // accepted in this slice
  const unsigned long long pos_local = warp_base_of(s_wacc, warp, &n_cta);
  if (threadIdx.x == 0) acc0[rank] = n_cta;
  cluster.sync();  // accepted counts (and the cut's key) posted
  if (threadIdx.x < kClusterCtas) s_cnt[threadIdx.x] = acc0[threadIdx.x];
  __syncthreads();
  unsigned long long cta_before = 0ull, n_acc = 0ull;
#pragma unroll 1
  for (int r = 0; r < kClusterCtas; ++r) {
    if (r < static_cast<int>(rank)) cta_before += s_cnt[r];
    n_acc += s_cnt[r];
  }
  // 3. Output in index order and this CTA's moment sums, as in select_mid
  // (output positions offset by the accepted samples of the lower slices).
  float cw[3] = {0.0f, 0.0f, 0.0f};
  bool have_cw = false;  // warp-uniform
  DF S1[3] = {DF{0.0f, 0.0f}, DF{0.0f, 0.0f}, DF{0.0f, 0.0f}};
  DF S2[3] = {DF{0.0f, 0.0f}, DF{0.0f, 0.0f}, DF{0.0f, 0.0f}};
  auto emit = [&](uint32_t il, unsigned long long p, float (&th)[3]) {
    const uint32_t i = lo + il;
    if (kTheta) {
      th[0] = theta[i];
      th[1] = theta[static_cast<size_t>(n) + i];
      th[2] = theta[2 * static_cast<size_t>(n) + i];
    } else {
      ou_prior(prm, base + i, th[0], th[1], th[2]);
    }
    if (p == 0) {  // the moments' common shift, into every CTA
#pragma unroll 1
      for (int r = 0; r < kClusterCtas; ++r) {
        float* const sh = cluster.map_shared_rank(s_shift, r);
        sh[0] = th[0];
        sh[1] = th[1];
        sh[2] = th[2];
      }
    }
    if (p < cap) {
      idx_out[p] = i;
      rec_out[p] = make_float4(th[0], th[1], th[2], static_cast<float>(__longlong_as_double(s_raw[il])));
    }
  };
  const uint32_t n_groups = (g1 - g0 + 31u) / 32u;
  const unsigned int word = static_cast<uint32_t>(lane) < n_groups ? acc_bits[(g0 >> 5) + lane] : 0u;
  unsigned int before_g = __popc(word);
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int y = __shfl_up_sync(0xFFFFFFFFu, before_g, o);
    if (lane >= o) before_g += y;
  }
  before_g -= __popc(word);
  unsigned int busy = __ballot_sync(0xFFFFFFFFu, word != 0u);
  unsigned int nw;  // accepted samples this warp sums
  if (n_cta <= kMidList) {  // CTA-uniform: the list in the histogram's place
    unsigned int* list = h;
#pragma unroll 1
    while (busy != 0u) {  // warp-uniform
      const int q = __ffs(busy) - 1;
      busy &= busy - 1u;
      const unsigned int accb = __shfl_sync(0xFFFFFFFFu, word, q);
      const unsigned int bq = __shfl_sync(0xFFFFFFFFu, before_g, q);
      if ((accb >> lane) & 1u) list[pos_local + bq + __popc(accb & lane_lt)] = g0 + 32u * q + lane;
    }
    __syncthreads();
    unsigned int mine_count = 0;
#pragma unroll 1
    for (uint32_t p0 = warp * 32u; p0 < n_cta; p0 += kMidThreads) {  // warp-uniform
      const uint32_t p = p0 + lane;
      const bool mine = p < n_cta;
      float th[3] = {0.0f, 0.0f, 0.0f};
      if (mine) emit(list[p], cta_before + p, th);
      if (!have_cw) {
#pragma unroll
        for (int d = 0; d < 3; ++d) cw[d] = __shfl_sync(0xFFFFFFFFu, th[d], 0);
        have_cw = true;
      }
      if (mine) {
        add_moment(S1, S2, th, cw);
        ++mine_count;
      }
    }
    nw = __reduce_add_sync(0xFFFFFFFFu, mine_count);
    if (lane == 0) s_wacc[warp] = nw;
  } else {
#pragma unroll 1
    while (busy != 0u) {  // warp-uniform
      const int q = __ffs(busy) - 1;
      busy &= busy - 1u;
      const unsigned int accb = __shfl_sync(0xFFFFFFFFu, word, q);
      const unsigned long long pq = cta_before + pos_local + __shfl_sync(0xFFFFFFFFu, before_g, q);
      const bool mine = (accb >> lane) & 1u;
      float th[3] = {0.0f, 0.0f, 0.0f};
      if (mine) emit(g0 + 32u * q + lane, pq + __popc(accb & lane_lt), th);
      if (!have_cw) {
        const int src = __ffs(accb) - 1;
#pragma unroll
        for (int d = 0; d < 3; ++d) cw[d] = __shfl_sync(0xFFFFFFFFu, th[d], src);
        have_cw = true;
      }
      if (mine) add_moment(S1, S2, th, cw);
    }
    nw = wacc;
  }
  cluster.sync();  // the common shift written into every CTA
  if (cta_moment_sums<kMidWarps>(S1, S2, cw, nw, s_S1, s_S2, s_cw, s_wacc, s_shift) && lane == 0) {
    DF* const S1_0 = cluster.map_shared_rank(c_S1, 0);
    DF* const S2_0 = cluster.map_shared_rank(c_S2, 0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      S1_0[d * kClusterCtas + rank] = S1[d];
      S2_0[d * kClusterCtas + rank] = S2[d];
    }
  }
  cluster.sync();  // the CTAs' sums posted; the last barrier
  if (rank == 0 && warp == 0) {
    // the CTAs' sums (all about the common shift) added with a fixed tree
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      S1[d] = lane < kClusterCtas ? c_S1[d * kClusterCtas + lane] : DF{0.0f, 0.0f};
      S2[d] = lane < kClusterCtas ? c_S2[d * kClusterCtas + lane] : DF{0.0f, 0.0f};
    }
#pragma unroll 1
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        S1[d] = df_add(S1[d], DF{__shfl_xor_sync(0xFFFFFFFFu, S1[d].hi, o), __shfl_xor_sync(0xFFFFFFFFu, S1[d].lo, o)});
        S2[d] = df_add(S2[d], DF{__shfl_xor_sync(0xFFFFFFFFu, S2[d].hi, o), __shfl_xor_sync(0xFFFFFFFFu, S2[d].lo, o)});
      }
    }
    store_moments(S1, S2, n_acc, s_shift, post_out);
    if (lane == 0) {
      *n_acc_out = n_acc;
      if (eps_out) *eps_out = threshold ? eps_thr : key_to_double(s_cut);
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

// The one-CTA and cluster selections keep up to kMidMax distances per CTA in
// shared memory, above the default 48 KB: the limit is raised once per
// device (a host call, made before any stream capture that launches the
// selection), and the device is asked once whether a cluster of
// kClusterCtas such CTAs fits at all (if not, those sizes take the
// multi-launch path).
std::atomic<unsigned long long> g_cluster_ok{0ull};

cudaError_t select_prepare() {
  static std::atomic<unsigned long long> ready{0ull};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (ready.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  const int smem = static_cast<int>(kMidKeyBytes);
  e = cudaFuncSetAttribute(select_mid<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(select_mid<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(select_cluster<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(select_cluster<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kClusterCtas);
    cfg.blockDim = dim3(kMidThreads);
    cfg.dynamicSmemBytes = kMidKeyBytes;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = kClusterCtas;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    const cudaError_t q = cudaOccupancyMaxActiveClusters(&clusters, select_cluster<false>, &cfg);
    if (q == cudaSuccess && clusters > 0 && bit)
      g_cluster_ok.fetch_or(bit, std::memory_order_acq_rel);
    else if (q != cudaSuccess)
      (void)cudaGetLastError();  // not sticky: the multi-launch path serves these sizes
  }
  if (e == cudaSuccess && bit) ready.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

bool cluster_select_ok() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return false;
  return (g_cluster_ok.load(std::memory_order_acquire) >> dev) & 1ull;
}

cudaError_t launch_select(const double* dist, uint32_t n, uint64_t k, double eps,
                          const OUConst& P_, uint64_t base, const float* theta, uint32_t* idx_out,
                          float* rec_out, uint64_t cap, uint64_t* n_acc_out, double* eps_out,
                          double* post_out, void* ws, cudaStream_t s) {
  const bool threshold = (k == 0);
  bool cluster_ok = false;
  if (n > 0 && n <= kClusterMax) {
    cudaError_t e = select_prepare();
    if (e != cudaSuccess) return e;
    cluster_ok = cluster_select_ok();
  }
  if (n > 0 && n <= kMidMax && (n <= kOneCtaMax || !cluster_ok)) {
    const unsigned long long cut = threshold ? host_dist_key(eps) : 0ull;
    const size_t smem = static_cast<size_t>(n) * sizeof(unsigned long long);
    if (theta)
      select_mid<true><<<1, kMidThreads, smem, s>>>(dist, n, k, threshold, cut, eps, P_, static_cast<uint32_t>(base),
                                                    theta, idx_out, reinterpret_cast<float4*>(rec_out), cap,
                                                    reinterpret_cast<unsigned long long*>(n_acc_out), eps_out,
                                                    post_out);
    else
      select_mid<false><<<1, kMidThreads, smem, s>>>(dist, n, k, threshold, cut, eps, P_, static_cast<uint32_t>(base),
                                                     theta, idx_out, reinterpret_cast<float4*>(rec_out), cap,
                                                     reinterpret_cast<unsigned long long*>(n_acc_out), eps_out,
                                                     post_out);
    return cudaGetLastError();
  }
  if (n > 0 && n <= kClusterMax && cluster_ok) {
    const unsigned long long cut = threshold ? host_dist_key(eps) : 0ull;
    const uint32_t slice = ((n + kClusterCtas - 1) / kClusterCtas + 31u) & ~31u;
    const size_t smem = static_cast<size_t>(slice) * sizeof(unsigned long long);
    if (theta)
      select_cluster<true><<<kClusterCtas, kMidThreads, smem, s>>>(
          dist, n, k, threshold, cut, eps, P_, static_cast<uint32_t>(base), theta, idx_out,
          reinterpret_cast<float4*>(rec_out), cap, reinterpret_cast<unsigned long long*>(n_acc_out), eps_out,
          post_out);
    else
      select_cluster<false><<<kClusterCtas, kMidThreads, smem, s>>>(
          dist, n, k, threshold, cut, eps, P_, static_cast<uint32_t>(base), theta, idx_out,
          reinterpret_cast<float4*>(rec_out), cap, reinterpret_cast<unsigned long long*>(n_acc_out), eps_out,
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
    // one key per thread up to 8 CTAs per SM: the passes are latency-bound
    // at the sizes where that leaves the GPU partly idle
    const uint32_t want = (n + kHistThreads - 1) / kHistThreads;
    const uint32_t cap_blocks = static_cast<uint32_t>(sms > 0 ? sms : 1) * 8u;
    const uint32_t blocks = want < 1 ? 1 : (want > cap_blocks ? cap_blocks : want);
    for (int pass = 0; pass < kNumPasses; ++pass)
      select_hist<<<blocks, kHistThreads, 0, s>>>(dist, n, pass, st, hist);
  }
  if (tiles > 0) {
    select_count<<<tiles, kTileThreads, 0, s>>>(dist, n, st, threshold, cut_thr, tile_less, tile_eq);
  }
  select_scan<<<1, kScanThreads, 0, s>>>(st, threshold, cut_thr, eps, tile_less, tile_eq, tile_off,
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
