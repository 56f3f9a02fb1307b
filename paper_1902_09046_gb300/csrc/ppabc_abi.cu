// ppabc_abi.cu -- the extern "C" entry points of libppabc.so: argument
// validation, device check, error reporting, and kernel launches.  The
// meaning of each call is documented in include/ppabc.h.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "internal.h"

namespace ppabc {

namespace {
thread_local char g_last_error[512] = "";
constexpr int kMaxDevices = 64;
std::mutex g_dev_mutex;
int g_dev_state[kMaxDevices] = {0};  // 0 unknown, 1 ok, -1 unsupported
}  // namespace

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return code;
}

int check_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PPABC_OK;
  return set_error(PPABC_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

int require_device() {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return check_cuda(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(PPABC_ENODEV, "device index %d out of range", dev);
  {
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    if (g_dev_state[dev] == 1) return PPABC_OK;
  }
  int major = 0, minor = 0;
  e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (e != cudaSuccess) return check_cuda(e, "cudaDeviceGetAttribute");
  std::lock_guard<std::mutex> lock(g_dev_mutex);
  if (major == 10 && minor == 3) {
    g_dev_state[dev] = 1;
    return PPABC_OK;
  }
  g_dev_state[dev] = -1;
  return set_error(PPABC_ENODEV, "device %d is sm_%d%d; this library is built for sm_103a only", dev,
                   major, minor);
}

int validate_model(const ppabc_ou_model* m) {
  if (!m) return set_error(PPABC_EINVAL, "model is NULL");
  for (int j = 0; j < 3; ++j) {
    if (!isfinite(m->lo[j]) || !isfinite(m->hi[j]) || m->lo[j] > m->hi[j])
      return set_error(PPABC_EINVAL, "prior bound %d must be finite with lo <= hi", j);
  }
  if (!(m->dt > 0.0) || !isfinite(m->dt)) return set_error(PPABC_EINVAL, "dt must be positive and finite");
  if (!isfinite(m->x0)) return set_error(PPABC_EINVAL, "x0 must be finite");
  if (m->n_obs < 1 || m->n_obs > PPABC_MAX_OBS)
    return set_error(PPABC_EINVAL, "n_obs must be in [1, %d]", PPABC_MAX_OBS);
  if (m->n_steps < m->n_obs) return set_error(PPABC_EINVAL, "n_steps must be >= n_obs");
  if (m->n_steps > 0x80000000u) return set_error(PPABC_EINVAL, "n_steps must be <= 2^31");
  return PPABC_OK;
}

int make_ou_const(const ppabc_ou_model* m, const double* h_y_obs, uint64_t seed,
                  uint32_t substream, OUConst* out) {
  int rc = validate_model(m);
  if (rc) return rc;
  OUConst P;
  memset(&P, 0, sizeof(P));
  for (int j = 0; j < 3; ++j) {
    P.lo[j] = static_cast<float>(m->lo[j]);
    P.span[j] = static_cast<float>(m->hi[j] - m->lo[j]);
  }
  P.dt = static_cast<float>(m->dt);
  P.sqrt_dt = static_cast<float>(sqrt(m->dt));
  P.x0 = static_cast<float>(m->x0);
  P.n_steps = m->n_steps;
  P.n_obs = m->n_obs;
  P.keys = philox_keys(seed);
  P.sub = substream;
  for (uint32_t j = 1; j <= m->n_obs; ++j)
    P.s_obs[j - 1] = static_cast<uint32_t>((static_cast<uint64_t>(j) * m->n_steps) / m->n_obs);
  if (h_y_obs) {
    for (uint32_t j = 0; j < m->n_obs; ++j) {
      if (!isfinite(h_y_obs[j])) return set_error(PPABC_EINVAL, "y_obs[%u] is not finite", j);
      P.y[j] = h_y_obs[j];
    }
  }
  *out = P;
  return PPABC_OK;
}

}  // namespace ppabc

using namespace ppabc;

extern "C" {

int ppabc_abi_version(void) { return PPABC_ABI_VERSION; }

const char* ppabc_last_error(void) { return g_last_error; }

int ppabc_device_check(void) { return require_device(); }

int ppabc_device_info(int* sm_count, int* max_sm_clock_khz) {
  if (!sm_count || !max_sm_clock_khz) return set_error(PPABC_EINVAL, "sm_count and max_sm_clock_khz must be non-NULL");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(max_sm_clock_khz, cudaDevAttrClockRate, dev);
  return check_cuda(e, "device attributes");
}

int ppabc_philox_raw(uint64_t seed, const uint32_t* ctr, uint64_t n, uint32_t* out, void* stream) {
  if (n == 0) return PPABC_OK;
  if (!ctr || !out) return set_error(PPABC_EINVAL, "ctr and out must be non-NULL");
  if ((reinterpret_cast<uintptr_t>(ctr) | reinterpret_cast<uintptr_t>(out)) & 15u)
    return set_error(PPABC_EINVAL, "ctr and out must be 16-byte aligned");
  int rc = require_device();
  if (rc) return rc;
  return check_cuda(launch_philox_raw(seed, ctr, n, out, static_cast<cudaStream_t>(stream)),
                    "philox_raw launch");
}

int ppabc_normals(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t tag, uint64_t j0, uint64_t n,
                  uint32_t method, float* z, void* stream) {
  if (method > PPABC_BM_TABLE) return set_error(PPABC_EINVAL, "method must be PPABC_BM_POLY or PPABC_BM_TABLE");
  if (n == 0) return PPABC_OK;
  if (!z) return set_error(PPABC_EINVAL, "z must be non-NULL");
  if (j0 + n < j0 || ((j0 + n - 1) >> 2) > 0xFFFFFFFFull)
    return set_error(PPABC_EINVAL, "normal index range exceeds 2^34");
  int rc = require_device();
  if (rc) return rc;
  return check_cuda(launch_normals(seed, c1, c2, tag, j0, n, method, z, static_cast<cudaStream_t>(stream)),
                    "normals launch");
}

int ppabc_box_muller(const uint32_t* w, uint64_t n, uint32_t method, float* z, void* stream) {
  if (method > PPABC_BM_TABLE) return set_error(PPABC_EINVAL, "method must be PPABC_BM_POLY or PPABC_BM_TABLE");
  if (n == 0) return PPABC_OK;
  if (!w || !z) return set_error(PPABC_EINVAL, "w and z must be non-NULL");
  if ((reinterpret_cast<uintptr_t>(w) | reinterpret_cast<uintptr_t>(z)) & 7u)
    return set_error(PPABC_EINVAL, "w and z must be 8-byte aligned");
  if (n > 0x7FFFFFFFull * 256ull) return set_error(PPABC_EINVAL, "n too large");
  int rc = require_device();
  if (rc) return rc;
  return check_cuda(launch_box_muller(w, n, method, z, static_cast<cudaStream_t>(stream)), "box_muller launch");
}

int abc_prior_predictive(const ppabc_ou_model* h_model, const double* h_y_obs, uint64_t n_samples,
                         uint64_t sample_base, uint64_t seed, uint32_t substream, float* theta_out,
                         double* summ_out, double* dist_out, void* stream) {
  OUConst P;
  int rc = make_ou_const(h_model, h_y_obs, seed, substream, &P);
  if (rc) return rc;
  if (!h_y_obs) return set_error(PPABC_EINVAL, "h_y_obs is NULL");
  if (sample_base > 0x100000000ull || n_samples > 0x100000000ull - sample_base)
    return set_error(PPABC_EINVAL, "sample_base + n_samples must be <= 2^32");
  if (n_samples == 0) return PPABC_OK;
  if (n_samples > 0xFFFFFFFFull) return set_error(PPABC_EINVAL, "n_samples must be < 2^32");
  if (!dist_out) return set_error(PPABC_EINVAL, "dist_out is NULL");
  rc = require_device();
  if (rc) return rc;
  return check_cuda(launch_em_ou(P, sample_base, static_cast<uint32_t>(n_samples), theta_out, summ_out,
                                 dist_out, static_cast<cudaStream_t>(stream)),
                    "prior-predictive launch");
}

size_t abc_select_workspace_bytes(uint64_t n) { return select_workspace_bytes(n); }

int abc_select(const double* dist, uint64_t n, uint64_t k, double eps, const ppabc_ou_model* h_model,
               uint64_t sample_base, uint64_t seed, uint32_t substream, const float* theta,
               uint32_t* idx_out, float* rec_out, uint64_t cap, uint64_t* n_acc_out, double* eps_out,
               double* post_out, void* workspace, size_t workspace_bytes, void* stream) {
  if (n > 0xFFFFFFFFull) return set_error(PPABC_EINVAL, "n must be < 2^32");
  if (k > n) return set_error(PPABC_EINVAL, "k (%llu) > n (%llu)", (unsigned long long)k,
                              (unsigned long long)n);
  if (k == 0 && isnan(eps)) return set_error(PPABC_EINVAL, "eps is NaN");
  if (!n_acc_out) return set_error(PPABC_EINVAL, "n_acc_out is NULL");
  if (n > 0 && !dist) return set_error(PPABC_EINVAL, "dist is NULL");
  if (cap > 0 && (!idx_out || !rec_out)) return set_error(PPABC_EINVAL, "idx_out/rec_out NULL with cap > 0");
  if (rec_out && (reinterpret_cast<uintptr_t>(rec_out) & 15u))
    return set_error(PPABC_EINVAL, "rec_out must be 16-byte aligned");
  if (!workspace || workspace_bytes < select_workspace_bytes(n))
    return set_error(PPABC_ENOMEM, "workspace needs %zu bytes, got %zu", select_workspace_bytes(n),
                     workspace_bytes);
  if (reinterpret_cast<uintptr_t>(workspace) & 255u)
    return set_error(PPABC_EINVAL, "workspace must be 256-byte aligned");
  OUConst P;
  memset(&P, 0, sizeof(P));
  if (!theta) {
    if (!h_model) return set_error(PPABC_EINVAL, "theta is NULL and h_model is NULL");
    int rc = make_ou_const(h_model, nullptr, seed, substream, &P);
    if (rc) return rc;
    if (sample_base > 0x100000000ull || n > 0x100000000ull - sample_base)
      return set_error(PPABC_EINVAL, "sample_base + n must be <= 2^32");
  }
  int rc = require_device();
  if (rc) return rc;
  return check_cuda(launch_select(dist, static_cast<uint32_t>(n), k, eps, P, sample_base, theta, idx_out,
                                  rec_out, cap, n_acc_out, eps_out, post_out, workspace,
                                  static_cast<cudaStream_t>(stream)),
                    "abc_select launch");
}

int pvalue_sweep(const double* lambda, uint32_t n_lambda, uint32_t n_obs, uint64_t m_sets,
                 uint64_t set_base, double ybar_obs, uint64_t seed, uint64_t* counts, double* p_out,
                 double* ybar_out, void* stream) {
  if (n_lambda == 0) return PPABC_OK;
  if (n_lambda > 65535u) return set_error(PPABC_EINVAL, "n_lambda must be <= 65535");
  if (!lambda || !counts) return set_error(PPABC_EINVAL, "lambda and counts must be non-NULL");
  if (n_obs < 1) return set_error(PPABC_EINVAL, "n_obs must be >= 1");
  if (m_sets < 1 || m_sets > 0xFFFFFFFFull) return set_error(PPABC_EINVAL, "m_sets must be in [1, 2^32)");
  if (set_base > 0x100000000ull - m_sets)
    return set_error(PPABC_EINVAL, "set_base + m_sets must be <= 2^32");
  if (((static_cast<uint64_t>(n_obs) + 1 + 3) >> 2) > 0xFFFFFFFFull)
    return set_error(PPABC_EINVAL, "n_obs too large");
  if (!isfinite(ybar_obs)) return set_error(PPABC_EINVAL, "ybar_obs must be finite");
  int rc = require_device();
  if (rc) return rc;
  return check_cuda(launch_pvalue(lambda, n_lambda, n_obs, static_cast<uint32_t>(m_sets),
                                  static_cast<uint32_t>(set_base), ybar_obs, seed, counts, p_out,
                                  ybar_out, static_cast<cudaStream_t>(stream)),
                    "pvalue_sweep launch");
}

size_t weakinf_test_workspace_bytes(uint64_t n_lambda, uint64_t n_sets) {
  return weakinf_workspace_bytes(n_lambda, n_sets);
}

int weakinf_test(const double* lambda, uint32_t n_lambda, double lambda0, uint32_t n_obs,
                 uint64_t n_sets, double alpha, uint64_t seed, double* gamma_out, uint32_t* counts_out,
                 void* workspace, size_t workspace_bytes, void* stream) {
  if (n_lambda == 0) return PPABC_OK;
  if (n_lambda > 0x7FFFFFFFu) return set_error(PPABC_EINVAL, "n_lambda too large");
  if (!lambda || !gamma_out) return set_error(PPABC_EINVAL, "lambda and gamma_out must be non-NULL");
  if (n_obs < 1) return set_error(PPABC_EINVAL, "n_obs must be >= 1");
  if (n_sets < 1 || n_sets > PPABC_WEAKINF_MAX_SETS)
    return set_error(PPABC_EINVAL, "n_sets must be in [1, %d]", PPABC_WEAKINF_MAX_SETS);
  if (!(alpha > 0.0 && alpha <= 1.0)) return set_error(PPABC_EINVAL, "alpha must be in (0, 1]");
  if (!isfinite(lambda0) || lambda0 < 0.0) return set_error(PPABC_EINVAL, "lambda0 must be >= 0");
  const size_t need = weakinf_workspace_bytes(n_lambda, n_sets);
  if (!workspace || workspace_bytes < need)
    return set_error(PPABC_ENOMEM, "workspace needs %zu bytes, got %zu", need, workspace_bytes);
  if (reinterpret_cast<uintptr_t>(workspace) & 255u) return set_error(PPABC_EINVAL, "workspace must be 256-byte aligned");
  int rc = require_device();
  if (rc) return rc;
  return check_cuda(launch_weakinf(lambda, n_lambda, lambda0, n_obs, static_cast<uint32_t>(n_sets), alpha,
                                   seed, gamma_out, counts_out, workspace, static_cast<cudaStream_t>(stream)),
                    "weakinf launch");
}

int toggle_prior_predictive(const ppabc_toggle_model* h_model, const double* h_q_obs, uint64_t n,
                            uint64_t sample_base, uint64_t seed, uint32_t substream, float* theta_out,
                            double* summ_out, float* y_out, double* dist_out, void* stream) {
  if (!h_model || !h_q_obs) return set_error(PPABC_EINVAL, "h_model and h_q_obs must be non-NULL");
  if (h_model->T < 2) return set_error(PPABC_EINVAL, "T must be >= 2");
  if (h_model->C < 1 || h_model->C > PPABC_TOGGLE_MAX_CELLS)
    return set_error(PPABC_EINVAL, "C must be in [1, %d]", PPABC_TOGGLE_MAX_CELLS);
  for (int j = 0; j < 7; ++j)
    if (!isfinite(h_model->lo[j]) || !isfinite(h_model->hi[j]) || h_model->lo[j] > h_model->hi[j])
      return set_error(PPABC_EINVAL, "prior bound %d must be finite with lo <= hi", j);
  if (h_model->lo[0] < 0.0 || h_model->lo[1] < 0.0 || h_model->lo[2] < 0.0 || h_model->lo[5] < 0.0 ||
      h_model->lo[6] < 0.0)
    return set_error(PPABC_EINVAL, "mu, sigma, gamma and beta must have non-negative priors");
  if (substream >= (1u << 24)) return set_error(PPABC_EINVAL, "substream must be < 2^24");
  if (sample_base > 0x100000000ull || n > 0x100000000ull - sample_base)
    return set_error(PPABC_EINVAL, "sample_base + n must be <= 2^32");
  if (n == 0) return PPABC_OK;
  if (n > 0x7FFFFFFFull) return set_error(PPABC_EINVAL, "n must be < 2^31");
  if (!dist_out) return set_error(PPABC_EINVAL, "dist_out is NULL");
  ToggleConst P;
  memset(&P, 0, sizeof(P));
  for (int j = 0; j < 7; ++j) {
    P.lo[j] = static_cast<float>(h_model->lo[j]);
    P.span[j] = static_cast<float>(h_model->hi[j] - h_model->lo[j]);
  }
  P.T = h_model->T;
  P.C = h_model->C;
  P.sub = substream;
  P.keys = philox_keys(seed);
  for (int k = 0; k < PPABC_TOGGLE_NQ; ++k) {
    if (!isfinite(h_q_obs[k])) return set_error(PPABC_EINVAL, "q_obs[%d] is not finite", k);
    P.q_obs[k] = h_q_obs[k];
  }
  int rc = require_device();
  if (rc) return rc;
  return check_cuda(launch_toggle(P, sample_base, static_cast<uint32_t>(n), theta_out, summ_out, y_out,
                                  dist_out, static_cast<cudaStream_t>(stream)),
                    "toggle launch");
}

}  // extern "C"
