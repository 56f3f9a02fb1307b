// select_static.cu -- abc_select without caller-supplied scratch memory.
//
// Some callers cannot hand the library device memory: code that runs after an
// application has frozen its memory budget (no cudaMalloc allowed once serving
// starts, because an allocation can block on the whole device), or a plug-in
// living inside another framework whose allocator it cannot reach.  For them
// abc_select_static runs the same kernels as abc_select with its scratch in
// this file's static device array, so the call itself allocates nothing.
#include <mutex>

#include "internal.h"

namespace ppabc {

namespace {

// Scratch for up to PPABC_STATIC_SELECT_MAX_N distances (about 330 KB).  Every
// GPU that loads the library holds one copy until the process exits.
constexpr size_t kStaticScratchBytes = 340u * 1024u;
static __device__ __align__(256) unsigned char g_select_scratch[kStaticScratchBytes];

constexpr int kMaxDev = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDev] = {nullptr};

// Device address of g_select_scratch on the current device; resolved once per
// device (the host-side symbol is only a stand-in, not a device address) and
// kept for the life of the process, so a device reset, which may reload the
// module elsewhere, leaves it stale (documented in ppabc.h).
int scratch_for_current_device(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return check_cuda(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDev) return set_error(PPABC_ENODEV, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_select_scratch);
    if (e != cudaSuccess) return check_cuda(e, "cudaGetSymbolAddress(select scratch)");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return PPABC_OK;
}

}  // namespace

}  // namespace ppabc

using namespace ppabc;

extern "C" int abc_select_static(const double* dist, uint64_t n, uint64_t k, double eps,
                                 const ppabc_ou_model* h_model, uint64_t sample_base, uint64_t seed,
                                 uint32_t substream, const float* theta, uint32_t* idx_out,
                                 float* rec_out, uint64_t cap, uint64_t* n_acc_out, double* eps_out,
                                 double* post_out, void* stream) {
  if (n > PPABC_STATIC_SELECT_MAX_N)
    return set_error(PPABC_EINVAL,
                     "abc_select_static handles at most %llu distances (got %llu); use abc_select "
                     "with a workspace",
                     (unsigned long long)PPABC_STATIC_SELECT_MAX_N, (unsigned long long)n);
  if (select_workspace_bytes(PPABC_STATIC_SELECT_MAX_N) > kStaticScratchBytes)
    return set_error(PPABC_ENOMEM, "static select scratch is smaller than its stated maximum");
  int rc = require_device();
  if (rc) return rc;
  void* ws = nullptr;
  rc = scratch_for_current_device(&ws);
  if (rc) return rc;
  return abc_select(dist, n, k, eps, h_model, sample_base, seed, substream, theta, idx_out, rec_out,
                    cap, n_acc_out, eps_out, post_out, ws, kStaticScratchBytes, stream);
}
