// rejection.cu -- ABC rejection as Algorithm 1 states it: propose, simulate,
// accept when rho <= epsilon, until M samples are accepted.
//
// Proposals are consumed in sample-index order, so the result is the first M
// accepted samples of the counter-indexed sequence -- the same set whatever
// the chunking, and the same as the threshold form of abc_select applied to
// a long enough prefix.  The GPU works a chunk of proposals at a time
// (simulation, threshold selection, append of the chunk's acceptances at the
// running count); the host reads the count after every group of chunks and
// stops once it reaches M or the proposal budget is spent.
#include <algorithm>

#include "internal.h"

namespace ppabc {

namespace {

constexpr int kRejGroup = 4;  // chunks between host checks of the count

inline size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

struct RejLayout {
  size_t dist, idx, rec, nacc, state, select, total;
  explicit RejLayout(uint64_t chunk) {
    size_t o = 0;
    dist = o;
    o = align256(o + sizeof(double) * chunk);
    idx = o;
    o = align256(o + sizeof(uint32_t) * chunk);
    rec = o;
    o = align256(o + 16 * chunk);
    nacc = o;
    o = align256(o + sizeof(unsigned long long));
    state = o;  // [0] accepted so far, [1] proposals used up to the M-th acceptance
    o = align256(o + 2 * sizeof(unsigned long long));
    select = o;
    o = align256(o + select_workspace_bytes(chunk));
    total = o;
  }
};

// Copies this chunk's accepted records (already in index order) behind the
// running count, up to M.
__global__ void rejection_append(const uint32_t* __restrict__ idx_c, const float4* __restrict__ rec_c,
                                 const unsigned long long* __restrict__ nacc_c,
                                 const unsigned long long* __restrict__ state, uint32_t base,
                                 unsigned long long m_accept, uint32_t* __restrict__ idx_out,
                                 float4* __restrict__ rec_out) {
  const unsigned long long count = state[0];
  if (count >= m_accept) return;
  const unsigned long long take = min(*nacc_c, m_accept - count);
  for (unsigned long long t = blockIdx.x * blockDim.x + threadIdx.x; t < take;
       t += static_cast<unsigned long long>(gridDim.x) * blockDim.x) {
    idx_out[count + t] = base + idx_c[t];
    rec_out[count + t] = rec_c[t];
  }
}

// Advances the count; records how many proposals the M-th acceptance used.
__global__ void rejection_advance(const uint32_t* __restrict__ idx_c,
                                  const unsigned long long* __restrict__ nacc_c,
                                  unsigned long long* __restrict__ state, uint32_t base,
                                  unsigned long long m_accept) {
  const unsigned long long count = state[0];
  if (count >= m_accept) return;
  const unsigned long long n = *nacc_c;
  const unsigned long long take = min(n, m_accept - count);
  if (count + n >= m_accept) state[1] = static_cast<unsigned long long>(base) + idx_c[take - 1] + 1;
  state[0] = count + take;
}

}  // namespace

}  // namespace ppabc

using namespace ppabc;

extern "C" {

size_t abc_rejection_workspace_bytes(uint64_t chunk) { return RejLayout(chunk ? chunk : 1).total; }

int abc_rejection(const ppabc_ou_model* h_model, const double* h_y_obs, double eps, uint64_t m_accept,
                  uint64_t max_samples, uint64_t chunk, uint64_t seed, uint32_t substream,
                  uint32_t* idx_out, float* rec_out, uint64_t* h_counts, void* workspace,
                  size_t workspace_bytes, void* stream) {
  OUConst P;
  int rc = make_ou_const(h_model, h_y_obs, seed, substream, &P);
  if (rc) return rc;
  if (!h_y_obs || !h_counts) return set_error(PPABC_EINVAL, "h_y_obs and h_counts must be non-NULL");
  if (eps != eps) return set_error(PPABC_EINVAL, "eps is NaN");
  if (m_accept == 0 || !idx_out || !rec_out)
    return set_error(PPABC_EINVAL, "m_accept >= 1 and idx_out / rec_out are required");
  if (reinterpret_cast<uintptr_t>(rec_out) & 15u) return set_error(PPABC_EINVAL, "rec_out must be 16-byte aligned");
  if (max_samples == 0 || max_samples > 0x100000000ull)
    return set_error(PPABC_EINVAL, "max_samples must be in [1, 2^32]");
  if (chunk == 0 || chunk > 0xFFFFFFFFull) return set_error(PPABC_EINVAL, "chunk must be in [1, 2^32)");
  const RejLayout L(chunk);
  if (!workspace || workspace_bytes < L.total)
    return set_error(PPABC_ENOMEM, "workspace needs %zu bytes, got %zu", L.total, workspace_bytes);
  if (reinterpret_cast<uintptr_t>(workspace) & 255u) return set_error(PPABC_EINVAL, "workspace must be 256-byte aligned");
  rc = require_device();
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(workspace);
  double* dist = reinterpret_cast<double*>(w + L.dist);
  uint32_t* idx_c = reinterpret_cast<uint32_t*>(w + L.idx);
  float* rec_c = reinterpret_cast<float*>(w + L.rec);
  uint64_t* nacc_c = reinterpret_cast<uint64_t*>(w + L.nacc);
  unsigned long long* state = reinterpret_cast<unsigned long long*>(w + L.state);
  void* sel_ws = w + L.select;
  cudaError_t e = cudaMemsetAsync(state, 0, 2 * sizeof(unsigned long long), s);
  unsigned long long h_state[2] = {0, 0};
  uint64_t base = 0;
  while (e == cudaSuccess && base < max_samples) {
    for (int gi = 0; gi < kRejGroup && base < max_samples && e == cudaSuccess; ++gi) {
      const uint32_t n = static_cast<uint32_t>(std::min<uint64_t>(chunk, max_samples - base));
      e = launch_em_ou(P, base, n, nullptr, nullptr, dist, s);
      if (e == cudaSuccess)
        e = launch_select(dist, n, 0, eps, P, base, nullptr, idx_c, rec_c, n, nacc_c, nullptr, nullptr,
                          sel_ws, s);
      if (e == cudaSuccess) {
        rejection_append<<<64, 256, 0, s>>>(idx_c, reinterpret_cast<const float4*>(rec_c),
                                            reinterpret_cast<unsigned long long*>(nacc_c), state,
                                            static_cast<uint32_t>(base), m_accept, idx_out,
                                            reinterpret_cast<float4*>(rec_out));
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) {
        rejection_advance<<<1, 1, 0, s>>>(idx_c, reinterpret_cast<unsigned long long*>(nacc_c), state,
                                          static_cast<uint32_t>(base), m_accept);
        e = cudaGetLastError();
      }
      base += n;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_state, state, sizeof(h_state), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && h_state[0] >= m_accept) break;
  }
  if (e != cudaSuccess) return check_cuda(e, "abc_rejection");
  h_counts[0] = h_state[0];
  h_counts[1] = h_state[0] >= m_accept ? h_state[1] : base;
  return PPABC_OK;
}

}  // extern "C"
