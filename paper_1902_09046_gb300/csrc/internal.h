// internal.h -- host-side launchers shared between the translation units of
// libppabc.so (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/ppabc.h"
#include "ou_path.cuh"

namespace ppabc {

// Records msg as the calling thread's last error and returns code.
int set_error(int code, const char* fmt, ...);
// PPABC_OK, or the status of a failed launch / CUDA call (with message).
int check_cuda(cudaError_t e, const char* what);
// PPABC_OK if the current device is sm_103 (cached per device).
int require_device();
// Fills an OUConst from a validated model, observed summaries and seed.
int make_ou_const(const ppabc_ou_model* m, const double* h_y_obs, uint64_t seed,
                  uint32_t substream, OUConst* out);

// Kernel launchers (return cudaGetLastError() of the launch).
cudaError_t launch_philox_raw(uint64_t seed, const uint32_t* ctr, uint64_t n, uint32_t* out,
                              cudaStream_t s);
cudaError_t launch_normals(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t tag, uint64_t j0,
                           uint64_t n, uint32_t method, float* z, cudaStream_t s);
cudaError_t launch_box_muller(const uint32_t* w, uint64_t n, uint32_t method, float* z, cudaStream_t s);
// Raises the shared-memory limit of the path kernels and the table-driven
// RNG hooks on the current device (once; launch_em_ou calls it too).  Call
// before capturing launches.
cudaError_t em_prepare();
cudaError_t launch_em_ou(const OUConst& P, uint64_t base, uint32_t n, float* theta_out,
                         double* summ_out, double* dist_out, cudaStream_t s);

// Selection.
size_t select_workspace_bytes(uint64_t n);
// Raises the one-CTA selection's shared-memory limit on the current device
// (once; launch_select calls it too).  Call before capturing launches.
cudaError_t select_prepare();
cudaError_t launch_select(const double* dist, uint32_t n, uint64_t k, double eps,
                          const OUConst& P, uint64_t base, const float* theta, uint32_t* idx_out,
                          float* rec_out, uint64_t cap, uint64_t* n_acc_out, double* eps_out,
                          double* post_out, void* ws, cudaStream_t s);

// p-value sweep.
cudaError_t launch_pvalue(const double* lambda, uint32_t n_lambda, uint32_t n_obs,
                          uint32_t m_sets, uint32_t set_base, double ybar_obs, uint64_t seed,
                          uint64_t* counts,
                          double* p_out, double* ybar_out, cudaStream_t s);

// Toggle switch: launch constants (binary32 prior box, sizes, observed
// quantiles, Philox key).
struct ToggleConst {
  float lo[7];
  float span[7];
  uint32_t T;
  uint32_t C;
  uint32_t sub;
  PhiloxKeys keys;
  double q_obs[PPABC_TOGGLE_NQ];
};
cudaError_t launch_toggle(const ToggleConst& P, uint64_t base, uint32_t n, float* theta_out,
                          double* summ_out, float* y_out, double* dist_out, cudaStream_t s);

// Weak-informativity test.
size_t weakinf_workspace_bytes(uint64_t n_lambda, uint64_t n_sets);
cudaError_t launch_weakinf(const double* lambda, uint32_t n_lambda, double lambda0, uint32_t n_obs,
                           uint32_t n_sets, double alpha, uint64_t seed, double* gamma_out,
                           uint32_t* counts_out, void* workspace, cudaStream_t s);

}  // namespace ppabc
