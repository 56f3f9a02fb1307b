// merge.cu -- the exchange step of a sample-sharded ABC job.
//
// A job of N prior samples split into contiguous index ranges over P ranks
// (the static split of the paper's sampler, Sec. 3.4) selects its k nearest
// (Sec. 3.1: the fixed-N form, epsilon the k-th smallest distance) in two
// steps.  Each rank selects its own k nearest; the global k nearest by
// (distance, index) are among those P k candidates, because a sample beaten
// by k others of its own range is beaten by them globally too.  So:
//   abc_select_candidates: this rank's accepted samples as a candidate
//     record -- the exact binary64 distance, the global index, theta;
//   (the caller all-gathers the records in rank order, which is the order of
//   the global indices);
//   abc_merge_candidates: the k nearest of the gathered candidates with the
//     selection kernels of abc_select (ties to the earlier position, so to
//     the smaller global index), their global indices, epsilon and the
//     posterior moments over the merged set in index order.
// The result equals the unsharded abc_select on the whole range.
#include <string.h>

#include "internal.h"

namespace ppabc {

namespace {

__global__ void candidates_kernel(const double* __restrict__ dist, uint64_t sample_base,
                                  const uint32_t* __restrict__ idx, const float4* __restrict__ rec,
                                  uint32_t count, double* __restrict__ cand_dist,
                                  uint64_t* __restrict__ cand_index, float* __restrict__ cand_theta) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const uint32_t j = idx[i];
  const float4 r = rec[i];
  cand_dist[i] = dist[j];
  cand_index[i] = sample_base + j;
  cand_theta[i] = r.x;
  cand_theta[static_cast<size_t>(count) + i] = r.y;
  cand_theta[2 * static_cast<size_t>(count) + i] = r.z;
}

__global__ void map_indices_kernel(const uint32_t* __restrict__ pos, const uint64_t* __restrict__ cand_index,
                                   const unsigned long long* __restrict__ n_acc, uint64_t cap,
                                   uint64_t* __restrict__ idx_out) {
  const uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const uint64_t n = *n_acc < cap ? *n_acc : cap;
  if (i < n) idx_out[i] = cand_index[pos[i]];
}

inline size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

}  // namespace

}  // namespace ppabc

using namespace ppabc;

extern "C" {

int abc_select_candidates(const double* dist, uint64_t n, uint64_t sample_base, const uint32_t* idx,
                          const float* rec, uint64_t count, double* cand_dist, uint64_t* cand_index,
                          float* cand_theta, void* stream) {
  if (count == 0) return PPABC_OK;
  if (count > n) return set_error(PPABC_EINVAL, "count (%llu) > n (%llu)", (unsigned long long)count,
                                  (unsigned long long)n);
  if (n > 0xFFFFFFFFull) return set_error(PPABC_EINVAL, "n must be < 2^32");
  if (!dist || !idx || !rec || !cand_dist || !cand_index || !cand_theta)
    return set_error(PPABC_EINVAL, "dist, idx, rec and the candidate arrays must be non-NULL");
  if (reinterpret_cast<uintptr_t>(rec) & 15u) return set_error(PPABC_EINVAL, "rec must be 16-byte aligned");
  if (sample_base > 0x100000000ull || n > 0x100000000ull - sample_base)
    return set_error(PPABC_EINVAL, "sample_base + n must be <= 2^32");
  int rc = require_device();
  if (rc) return rc;
  const unsigned blocks = static_cast<unsigned>((count + 255) / 256);
  candidates_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      dist, sample_base, idx, reinterpret_cast<const float4*>(rec), static_cast<uint32_t>(count), cand_dist,
      cand_index, cand_theta);
  return check_cuda(cudaGetLastError(), "abc_select_candidates launch");
}

size_t abc_merge_workspace_bytes(uint64_t m, uint64_t k) {
  return align256(select_workspace_bytes(m)) + align256(sizeof(uint32_t) * (k > 0 ? k : 1));
}

int abc_merge_candidates(const double* cand_dist, const uint64_t* cand_index, const float* cand_theta, uint64_t m,
                         uint64_t k, uint64_t* idx_out, float* rec_out, uint64_t* n_acc_out, double* eps_out,
                         double* post_out, void* workspace, size_t workspace_bytes, void* stream) {
  if (m > 0xFFFFFFFFull) return set_error(PPABC_EINVAL, "m must be < 2^32");
  if (k == 0 || k > m)
    return set_error(PPABC_EINVAL, "k must be in [1, m] (k = %llu, m = %llu)", (unsigned long long)k,
                     (unsigned long long)m);
  if (!cand_dist || !cand_index || !cand_theta || !idx_out || !rec_out || !n_acc_out)
    return set_error(PPABC_EINVAL, "candidate arrays, idx_out, rec_out and n_acc_out must be non-NULL");
  if (reinterpret_cast<uintptr_t>(rec_out) & 15u) return set_error(PPABC_EINVAL, "rec_out must be 16-byte aligned");
  if (!workspace || workspace_bytes < abc_merge_workspace_bytes(m, k))
    return set_error(PPABC_ENOMEM, "workspace needs %zu bytes, got %zu", abc_merge_workspace_bytes(m, k),
                     workspace_bytes);
  if (reinterpret_cast<uintptr_t>(workspace) & 255u)
    return set_error(PPABC_EINVAL, "workspace must be 256-byte aligned");
  int rc = require_device();
  if (rc) return rc;
  char* w = static_cast<char*>(workspace);
  uint32_t* pos = reinterpret_cast<uint32_t*>(w + align256(select_workspace_bytes(m)));
  OUConst P;
  memset(&P, 0, sizeof(P));  // theta is given: nothing is redrawn
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_select(cand_dist, static_cast<uint32_t>(m), k, 0.0, P, 0, cand_theta, pos, rec_out, k,
                                n_acc_out, eps_out, post_out, w, s);
  if (e != cudaSuccess) return check_cuda(e, "abc_merge_candidates selection");
  map_indices_kernel<<<static_cast<unsigned>((k + 255) / 256), 256, 0, s>>>(
      pos, cand_index, reinterpret_cast<const unsigned long long*>(n_acc_out), k, idx_out);
  return check_cuda(cudaGetLastError(), "abc_merge_candidates index map");
}

}  // extern "C"
