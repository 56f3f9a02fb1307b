// batch.cu -- many uneven OU-ABC jobs in one persistent launch.
//
// The paper splits a fixed N evenly over OpenMP threads (Sec. 3.4); with
// jobs whose sizes and step counts differ by 10^5x an even split leaves most
// of the GPU idle.  Here every job is cut into tiles of (threads x spt)
// samples, where spt (samples per thread) is chosen so that one tile carries
// at least `min_tile_steps` Euler-Maruyama steps per thread.  A persistent
// grid -- one wave of CTAs -- pulls tiles from per-job queues (an atomic
// cursor per job) visited in order of decreasing step count, so long tiles
// start first and short ones fill the tail.  No CTA ever waits for another:
// a CTA only claims tiles with atomics and leaves when every queue is empty.
//
// After the simulation the accepted sets are selected per job with the same
// kernels as abc_select.  Prepare (upload of the job table) and launch are
// separate calls, so the launch can be captured into a CUDA graph and
// replayed.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "internal.h"

namespace ppabc {

namespace {

struct BatchJobDev {
  OUConst P;
  double* dist;
  uint32_t n;      // samples
  uint32_t tiles;  // tiles of threads * spt samples
  uint32_t spt;    // samples per thread in one tile
  uint32_t pad;
};

inline size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// The Box-Muller tables sit in shared memory: 512-thread CTAs hold the
// lane-replicated log table (80 KB, two CTAs per SM), 256-thread CTAs the
// compact one (50 KB, four per SM); the values, and so the results, are the
// same.
template <int kThreads>
constexpr bool batch_rep_log() { return kThreads >= 512; }

template <int kThreads>
constexpr size_t batch_smem() { return bm_smem_bytes<batch_rep_log<kThreads>()>(); }

template <int kThreads>
__global__ void __launch_bounds__(kThreads, 1024 / kThreads) em_ou_batch(const BatchJobDev* __restrict__ jobs,
                                                        const uint32_t* __restrict__ order,
                                                        uint32_t n_jobs, unsigned int* head,
                                                        unsigned int* cursors) {
  constexpr bool kRep = batch_rep_log<kThreads>();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_job;
  __shared__ uint32_t s_tile;
  bm_load<kRep>(smem);
  __syncthreads();
  const BmTab T = bm_tab<kRep>(smem);
  for (;;) {
    if (threadIdx.x == 0) {
      int jj = -1;
      uint32_t t = 0;
      uint32_t h = *reinterpret_cast<volatile unsigned int*>(head);
      while (h < n_jobs) {  // at most n_jobs iterations: h grows every round
        const uint32_t j = order[h];
        t = atomicAdd(&cursors[j], 1u);
        if (t < jobs[j].tiles) {
          jj = static_cast<int>(j);
          break;
        }
        atomicMax(head, h + 1);
        const uint32_t h2 = *reinterpret_cast<volatile unsigned int*>(head);
        h = h2 > h + 1 ? h2 : h + 1;
      }
      s_job = jj;
      s_tile = t;
    }
    __syncthreads();
    const int j = s_job;
    const uint32_t tile = s_tile;
    __syncthreads();
    if (j < 0) return;
    const BatchJobDev& J = jobs[j];
    const uint32_t n = J.n, spt = J.spt;
    const uint32_t base = tile * (kThreads * spt);
    // Samples q and q + 1 of the tile's column run together (ou_path2, the
    // two-path form of the plain kernel); an odd last one runs alone.
    uint32_t q = 0;
    for (; q + 1 < spt; q += 2) {
      const uint32_t i0 = base + q * kThreads + threadIdx.x;
      const uint32_t i1 = i0 + kThreads;
      if (i0 < n) {
        const uint32_t gi[2] = {i0, i1 < n ? i1 : i0};
        float th1[2], th2[2], th3[2];
        ou_prior(J.P, gi[0], th1[0], th2[0], th3[0]);
        ou_prior(J.P, gi[1], th1[1], th2[1], th3[1]);
        double d[2];
        ou_path2<false, kRep>(J.P, T, gi, th1, th2, th3, nullptr, nullptr, 0, d);
        J.dist[i0] = d[0];
        if (i1 < n) J.dist[i1] = d[1];
      }
    }
    if (q < spt) {
      const uint32_t i = base + q * kThreads + threadIdx.x;
      if (i < n) {
        float th1, th2, th3;
        ou_prior(J.P, i, th1, th2, th3);
        J.dist[i] = ou_path<false, kRep>(J.P, T, i, th1, th2, th3, nullptr, 0);
      }
    }
  }
}

struct SelectArgs {
  const double* dist;
  uint32_t n;
  uint64_t k;
  double eps;
  uint32_t* idx_out;
  float* rec_out;
  uint64_t cap;
  uint64_t* n_acc_out;
  double* eps_out;
  double* post_out;
};

}  // namespace

}  // namespace ppabc

using namespace ppabc;

// Host-side plan of a prepared batch (opaque to callers).
struct ppabc_batch_plan {
  uint32_t n_jobs = 0;
  uint32_t threads = 512;
  int grid = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  BatchJobDev* d_jobs = nullptr;
  uint32_t* d_order = nullptr;
  unsigned int* d_sched = nullptr;  // head, then one cursor per job
  void* d_select_ws = nullptr;
  std::vector<OUConst> consts;
  std::vector<SelectArgs> sel;
  cudaGraphExec_t graph = nullptr;
  cudaStream_t graph_stream = nullptr;
};

namespace {

struct Layout {
  size_t jobs, order, sched, dist, select, total;
};

int validate_jobs(const ppabc_abc_job* h_jobs, uint32_t n_jobs) {
  if (!h_jobs && n_jobs) return set_error(PPABC_EINVAL, "h_jobs is NULL");
  for (uint32_t j = 0; j < n_jobs; ++j) {
    const ppabc_abc_job& J = h_jobs[j];
    OUConst P;
    int rc = make_ou_const(&J.model, J.y_obs, J.seed, J.substream, &P);
    if (rc) {
      char msg[400];
      snprintf(msg, sizeof(msg), "%s", ppabc_last_error());
      return set_error(rc, "job %u: %s", j, msg);
    }
    if (J.n_samples == 0 || J.n_samples > 0xFFFFFFFFull)
      return set_error(PPABC_EINVAL, "job %u: n_samples must be in [1, 2^32)", j);
    if (J.k > J.n_samples) return set_error(PPABC_EINVAL, "job %u: k > n_samples", j);
    if (J.k == 0 && J.eps != J.eps) return set_error(PPABC_EINVAL, "job %u: eps is NaN", j);
    if (!J.n_acc_out) return set_error(PPABC_EINVAL, "job %u: n_acc_out is NULL", j);
    if (J.cap > 0 && (!J.idx_out || !J.rec_out))
      return set_error(PPABC_EINVAL, "job %u: idx_out/rec_out NULL with cap > 0", j);
    if (J.rec_out && (reinterpret_cast<uintptr_t>(J.rec_out) & 15u))
      return set_error(PPABC_EINVAL, "job %u: rec_out must be 16-byte aligned", j);
    if (J.dist && (reinterpret_cast<uintptr_t>(J.dist) & 7u))
      return set_error(PPABC_EINVAL, "job %u: dist must be 8-byte aligned", j);
  }
  return PPABC_OK;
}

Layout layout_of(const ppabc_abc_job* h_jobs, uint32_t n_jobs) {
  Layout L;
  size_t o = 0;
  uint64_t max_n = 1;
  L.jobs = o;
  o = align256(o + sizeof(BatchJobDev) * n_jobs);
  L.order = o;
  o = align256(o + sizeof(uint32_t) * n_jobs);
  L.sched = o;
  o = align256(o + sizeof(unsigned int) * (n_jobs + 1));
  L.dist = o;
  for (uint32_t j = 0; j < n_jobs; ++j) {
    if (!h_jobs[j].dist) o = align256(o + sizeof(double) * h_jobs[j].n_samples);
    max_n = std::max<uint64_t>(max_n, h_jobs[j].n_samples);
  }
  L.select = o;
  o = align256(o + select_workspace_bytes(max_n));
  L.total = o;
  return L;
}

}  // namespace

extern "C" {

size_t ppabc_batch_workspace_bytes(const ppabc_abc_job* h_jobs, uint32_t n_jobs) {
  if (!h_jobs || n_jobs == 0) return 256;
  return layout_of(h_jobs, n_jobs).total;
}

int ppabc_batch_prepare(const ppabc_abc_job* h_jobs, uint32_t n_jobs,
                        const ppabc_tile_config* h_cfg, void* workspace, size_t workspace_bytes,
                        void* stream, ppabc_batch_plan** plan_out) {
  if (!plan_out) return set_error(PPABC_EINVAL, "plan_out is NULL");
  *plan_out = nullptr;
  int rc = validate_jobs(h_jobs, n_jobs);
  if (rc) return rc;
  const uint32_t threads = h_cfg ? h_cfg->threads : 512u;
  const uint32_t min_steps = h_cfg ? h_cfg->min_tile_steps : 4096u;
  if (threads != 256u && threads != 512u)
    return set_error(PPABC_EINVAL, "tile threads must be 256 or 512");
  if (min_steps == 0) return set_error(PPABC_EINVAL, "min_tile_steps must be >= 1");
  const Layout L = layout_of(h_jobs, n_jobs);
  if (!workspace || workspace_bytes < L.total)
    return set_error(PPABC_ENOMEM, "batch workspace needs %zu bytes, got %zu", L.total, workspace_bytes);
  if (reinterpret_cast<uintptr_t>(workspace) & 255u)
    return set_error(PPABC_EINVAL, "workspace must be 256-byte aligned");
  rc = require_device();
  if (rc) return rc;

  ppabc_batch_plan* plan = new (std::nothrow) ppabc_batch_plan();
  if (!plan) return set_error(PPABC_ENOMEM, "host allocation of the batch plan failed");
  char* w = static_cast<char*>(workspace);
  plan->n_jobs = n_jobs;
  plan->threads = threads;
  plan->ws = workspace;
  plan->ws_bytes = workspace_bytes;
  plan->d_jobs = reinterpret_cast<BatchJobDev*>(w + L.jobs);
  plan->d_order = reinterpret_cast<uint32_t*>(w + L.order);
  plan->d_sched = reinterpret_cast<unsigned int*>(w + L.sched);
  plan->d_select_ws = w + L.select;

  std::vector<BatchJobDev> hj(n_jobs);
  std::vector<uint32_t> order(n_jobs);
  plan->consts.resize(n_jobs);
  plan->sel.resize(n_jobs);
  size_t dist_off = L.dist;
  for (uint32_t j = 0; j < n_jobs; ++j) {
    const ppabc_abc_job& J = h_jobs[j];
    BatchJobDev& D = hj[j];
    memset(&D, 0, sizeof(D));
    make_ou_const(&J.model, J.y_obs, J.seed, J.substream, &D.P);
    plan->consts[j] = D.P;
    if (J.dist) {
      D.dist = J.dist;
    } else {
      D.dist = reinterpret_cast<double*>(w + dist_off);
      dist_off = align256(dist_off + sizeof(double) * J.n_samples);
    }
    D.n = static_cast<uint32_t>(J.n_samples);
    uint32_t spt = (min_steps + J.model.n_steps - 1) / J.model.n_steps;
    spt = std::max(1u, std::min(spt, 64u));
    D.spt = spt;
    D.tiles = static_cast<uint32_t>((J.n_samples + static_cast<uint64_t>(threads) * spt - 1) /
                                    (static_cast<uint64_t>(threads) * spt));
    order[j] = j;
    plan->sel[j] = SelectArgs{D.dist, D.n, J.k, J.eps, J.idx_out, J.rec_out, J.cap, J.n_acc_out,
                              J.eps_out, J.post_out};
  }
  std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
    return h_jobs[a].model.n_steps > h_jobs[b].model.n_steps;
  });
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(plan->d_jobs, hj.data(), sizeof(BatchJobDev) * n_jobs,
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(plan->d_order, order.data(), sizeof(uint32_t) * n_jobs, cudaMemcpyHostToDevice, s);
  // The host vectors die when this function returns: wait for the copies.
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    delete plan;
    return check_cuda(e, "batch job-table upload");
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaFuncSetAttribute(em_ou_batch<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(batch_smem<256>()));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(em_ou_batch<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(batch_smem<512>()));
  if (e == cudaSuccess) {
    if (threads == 256)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, em_ou_batch<256>, 256, batch_smem<256>());
    else
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, em_ou_batch<512>, 512, batch_smem<512>());
  }
  if (e != cudaSuccess) {
    delete plan;
    return check_cuda(e, "occupancy query");
  }
  e = select_prepare();  // before a graph capture of the launches
  if (e != cudaSuccess) {
    delete plan;
    return check_cuda(e, "selection setup");
  }
  plan->grid = std::max(1, sms) * std::max(1, per_sm);
  *plan_out = plan;
  return PPABC_OK;
}

int ppabc_batch_launch(ppabc_batch_plan* plan, void* stream) {
  if (!plan) return set_error(PPABC_EINVAL, "plan is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint32_t n_jobs = plan->n_jobs;
  if (n_jobs == 0) return PPABC_OK;
  cudaError_t e = cudaMemsetAsync(plan->d_sched, 0, sizeof(unsigned int) * (n_jobs + 1), s);
  if (e != cudaSuccess) return check_cuda(e, "batch scheduler reset");
  unsigned int* head = plan->d_sched;
  unsigned int* cursors = plan->d_sched + 1;
  if (plan->threads == 256)
    em_ou_batch<256><<<plan->grid, 256, batch_smem<256>(), s>>>(plan->d_jobs, plan->d_order, n_jobs, head,
                                                                cursors);
  else
    em_ou_batch<512><<<plan->grid, 512, batch_smem<512>(), s>>>(plan->d_jobs, plan->d_order, n_jobs, head,
                                                                cursors);
  e = cudaGetLastError();
  if (e != cudaSuccess) return check_cuda(e, "em_ou_batch launch");
  for (uint32_t j = 0; j < n_jobs; ++j) {
    const SelectArgs& a = plan->sel[j];
    e = launch_select(a.dist, a.n, a.k, a.eps, plan->consts[j], 0, nullptr, a.idx_out, a.rec_out,
                      a.cap, a.n_acc_out, a.eps_out, a.post_out, plan->d_select_ws, s);
    if (e != cudaSuccess) return check_cuda(e, "batch select launch");
  }
  return PPABC_OK;
}

int ppabc_batch_launch_graph(ppabc_batch_plan* plan, void* stream) {
  if (!plan) return set_error(PPABC_EINVAL, "plan is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!s) return set_error(PPABC_EINVAL, "graph launch needs a non-default stream");
  if (!plan->graph) {
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return check_cuda(e, "cudaStreamBeginCapture");
    int rc = ppabc_batch_launch(plan, stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return check_cuda(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&plan->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      plan->graph = nullptr;
      return check_cuda(e, "cudaGraphInstantiate");
    }
  }
  return check_cuda(cudaGraphLaunch(plan->graph, s), "cudaGraphLaunch");
}

int ppabc_batch_plan_destroy(ppabc_batch_plan* plan) {
  if (!plan) return PPABC_OK;
  if (plan->graph) cudaGraphExecDestroy(plan->graph);
  delete plan;
  return PPABC_OK;
}

int ppabc_batch_run(const ppabc_abc_job* h_jobs, uint32_t n_jobs, const ppabc_tile_config* h_cfg,
                    void* workspace, size_t workspace_bytes, void* stream) {
  ppabc_batch_plan* plan = nullptr;
  int rc = ppabc_batch_prepare(h_jobs, n_jobs, h_cfg, workspace, workspace_bytes, stream, &plan);
  if (rc) return rc;
  rc = ppabc_batch_launch(plan, stream);
  ppabc_batch_plan_destroy(plan);
  return rc;
}

}  // extern "C"
