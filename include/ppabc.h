/*
 * ppabc.h -- C ABI of the GB300 (sm_103a) prior-predictive Monte Carlo
 * library libppabc.so.
 *
 * The library implements the data-parallel hot path of prior-predictive
 * sampling as used by ABC rejection sampling and by prior-predictive p-values
 * (Warne, Sisson & Drovandi, "Vector operations for accelerating expensive
 * Bayesian computations -- a tutorial guide", arXiv:1902.09046):
 *   abc_prior_predictive -- draw theta from the prior, simulate the model,
 *                           reduce to summaries and a discrepancy (Sec. 3.1,
 *                           Eq. 2 and Algorithm 1; Euler-Maruyama, Eq. 5);
 *   abc_select           -- choose the accepted set: the k nearest samples
 *                           (epsilon chosen a posteriori, Sec. 3.1) or all
 *                           samples with distance <= epsilon (Algorithm 1),
 *                           and the posterior mean / variance of theta;
 *   pvalue_sweep         -- prior-predictive p-values p_lambda over a grid of
 *                           hyperparameters (Sec. 4.1, Eq. 6 and Eq. 8) by
 *                           exact tail counts.
 *
 * General rules for every entry point:
 *   - Pointers are DEVICE pointers (memory of the current CUDA device) unless
 *     the parameter name starts with h_, in which case it is host memory read
 *     before the call returns.  The caller owns all memory; the library never
 *     allocates device memory.  Scratch memory is supplied by the caller and
 *     sized by the matching *_workspace_bytes function.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL is the legacy default
 *     stream) and is asynchronous: outputs are valid once the stream has been
 *     synchronised.  Calls are stream-ordered and do not synchronise the host.
 *   - Every call returns a status (PPABC_OK or a negative PPABC_E* code).  On
 *     error nothing has been enqueued, except for PPABC_ECUDA raised by a
 *     failed launch; ppabc_last_error() returns a message for the calling
 *     thread's last failure.
 *   - Only sm_103 devices are supported; any other device gives PPABC_ENODEV.
 *     There is no CPU fallback.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = (seed low 32
 * bits, seed high 32 bits).  Block b of the stream (index, substream, tag)
 * is counter (c0, c1, c2, c3) = (tag, b, substream, index), with tag 0 for
 * prior draws (block 0) and 1 for path / data normals; the index is the
 * global sample or data-set index.  A 32-bit word w encodes the uniform ((w >> 9) + 1/2) 2^-23 and
 * normals come from Box-Muller on consecutive word pairs.  Results therefore
 * depend only on (seed, substream, global sample index), never on launch
 * shape, batching or sharding.
 */
#ifndef PPABC_H
#define PPABC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PPABC_ABI_VERSION 1

#define PPABC_OK 0
#define PPABC_EINVAL (-1)     /* invalid argument */
#define PPABC_ENOMEM (-2)     /* workspace too small / admission refused */
#define PPABC_ECUDA (-3)      /* a CUDA runtime call or launch failed */
#define PPABC_ETIMEOUT (-4)   /* a bounded wait expired (ppabc_server_wait) */
#define PPABC_ENODEV (-5)     /* no sm_103 device current */
#define PPABC_ECANCELLED (-6) /* job cancelled by the host */
#define PPABC_PENDING 1       /* server job not finished yet (not an error) */

/* Most observations a model may have. */
#define PPABC_MAX_OBS 32

/* Counter tags. */
#define PPABC_TAG_PRIOR 0u
#define PPABC_TAG_PATH 1u
#define PPABC_TAG_BASE 2u /* base-prior data sets of the weak-informativity test */

/*
 * Ornstein-Uhlenbeck model of the ABC workloads:
 *   dX = th1 (th2 - X) dt + th3 dW,  X(0) = x0,
 * with independent uniform priors th_j ~ U(lo[j], hi[j]) (lo[j] <= hi[j];
 * equal bounds fix th_j).  The path takes n_steps Euler-Maruyama steps of
 * size dt (Eq. 5 applied to this SDE) and is observed after steps
 * s_j = floor(j n_steps / n_obs), j = 1..n_obs; 1 <= n_obs <= PPABC_MAX_OBS
 * and n_steps >= n_obs.
 */
typedef struct ppabc_ou_model {
  double lo[3];
  double hi[3];
  double x0;
  double dt;
  uint32_t n_steps;
  uint32_t n_obs;
} ppabc_ou_model;

/* ABI version (PPABC_ABI_VERSION of the built library). */
int ppabc_abi_version(void);

/* Message for the calling thread's last failed call ("" if none). */
const char *ppabc_last_error(void);

/* PPABC_OK if the current CUDA device is sm_103, else PPABC_ENODEV or
 * PPABC_ECUDA. */
int ppabc_device_check(void);

/* The current device's SM count and maximum SM clock (kHz), as the CUDA
 * runtime reports them; the roofline figures are built from these.  Both
 * pointers must be non-NULL (EINVAL).  No device work is enqueued. */
int ppabc_device_info(int *sm_count, int *max_sm_clock_khz);

/*
 * Raw Philox4x32-10 blocks: out[i][0..3] = philox(ctr[i][0..3], key(seed)),
 * i < n.  ctr and out are [n][4] uint32, 16-byte aligned.  Exposes the
 * generator that replaces the paper's MKL MT2203 streams (Sec. 2.5, option
 * (ii): one generator split into independent sub-streams).
 */
int ppabc_philox_raw(uint64_t seed, const uint32_t *ctr, uint64_t n,
                     uint32_t *out, void *stream);

/* The two binary32 evaluations of Box-Muller (Sec. 3.4, the transform of the
 * paper's MKL calls) in the library: polynomial -2 ln u and sin/cos (the
 * p-value, Algorithm 2 and toggle-switch kernels), and table-driven ones
 * (Tang's log tables and a two-level sin/cos table in shared memory: the OU
 * path kernels).  Both are within about 1 ulp of the binary64 transform. */
#define PPABC_BM_POLY 0u
#define PPABC_BM_TABLE 1u

/*
 * Standard normals j0 .. j0+n-1 of stream (seed, index c1, substream c2,
 * tag), in binary32: normal j is lane j%4 of counter (tag, j/4, c2, c1)
 * after the Box-Muller evaluation `method` (PPABC_BM_POLY or
 * PPABC_BM_TABLE; EINVAL otherwise).  z is [n] float.
 */
int ppabc_normals(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t tag,
                  uint64_t j0, uint64_t n, uint32_t method, float *z, void *stream);

/*
 * Box-Muller transform of given word pairs, in binary32: w is [n][2] uint32
 * (even, odd), z is [n][2] float with z_even = r cos 2 pi u(w_odd),
 * z_odd = r sin 2 pi u(w_odd), r = sqrt(-2 ln u(w_even)), by the evaluation
 * `method` (PPABC_BM_POLY or PPABC_BM_TABLE).  Exposes the transforms every
 * normal of the library goes through, so each can be checked on all 2^23
 * uniforms.  w and z 8-byte aligned.
 */
int ppabc_box_muller(const uint32_t *w, uint64_t n, uint32_t method, float *z, void *stream);

/*
 * Prior-predictive sampling for ABC (Sec. 3.1, Eq. 2; Algorithm 1 with N
 * fixed), one sample per global index g = sample_base + i, i < n_samples:
 *   theta ~ prior        (counter (PRIOR, 0, substream, g), words 0..2),
 *   X_s = X_{s-1} + th1 (th2 - X_{s-1}) dt + th3 sqrt(dt) xi_{s-1},
 *                        (xi_j: normal j of stream (seed, g, substream, PATH)),
 *   S(D*) = (X_{s_1}, .., X_{s_nobs}),  rho = || S(D*) - y_obs ||_2.
 * The path is integrated in binary32 with a compensated (Kahan) state; the
 * summaries and the discrepancy are accumulated in binary64.
 *   h_model     model and prior (host).
 *   h_y_obs     observed summaries, n_obs doubles (host).
 *   theta_out   nullable; [3][n_samples] float (structure of arrays).
 *   summ_out    nullable; [n_obs][n_samples] double, the simulated summaries.
 *   dist_out    [n_samples] double, the discrepancy rho.
 * Requires sample_base + n_samples <= 2^32.  n_samples == 0 is a no-op.
 */
int abc_prior_predictive(const ppabc_ou_model *h_model, const double *h_y_obs,
                         uint64_t n_samples, uint64_t sample_base,
                         uint64_t seed, uint32_t substream, float *theta_out,
                         double *summ_out, double *dist_out, void *stream);

/* Bytes of scratch abc_select needs for n distances (256-byte aligned). */
size_t abc_select_workspace_bytes(uint64_t n);

/*
 * Accepted set and posterior summaries.
 *   k > 0: accept the k samples with the smallest (dist, index); epsilon is
 *          then the k-th smallest distance (the a-posteriori choice of
 *          Sec. 3.1).  Requires k <= n.
 *   k = 0: accept every sample with dist <= eps (Algorithm 1's test);
 *          eps = +inf accepts every sample with a non-NaN distance.
 * Distances are ordered as binary64 values with -0 == +0 and every NaN after
 * +inf; ties go to the smaller index.
 * Outputs, in ascending index order:
 *   idx_out    [cap] uint32: local indices i (0 <= i < n) of accepted samples;
 *   rec_out    [cap][4] float (16-byte aligned): (th1, th2, th3, (float)dist);
 *              theta is read from `theta` ([3][n] float, as written by
 *              abc_prior_predictive) or, when theta is NULL, redrawn from the
 *              prior counter of sample sample_base + i using h_model, seed and
 *              substream (bit-identical to what abc_prior_predictive draws);
 *   n_acc_out  [1] uint64: number accepted (may exceed cap; only the first
 *              cap are written);
 *   eps_out    [1] double (nullable): the epsilon used;
 *   post_out   [6] double (nullable): posterior mean of (th1, th2, th3) then
 *              the unbiased (n_acc - 1) variances, over ALL accepted samples,
 *              reduced in a fixed order (deterministic); NaN when undefined.
 * workspace must hold abc_select_workspace_bytes(n) bytes.
 */
int abc_select(const double *dist, uint64_t n, uint64_t k, double eps,
               const ppabc_ou_model *h_model, uint64_t sample_base,
               uint64_t seed, uint32_t substream, const float *theta,
               uint32_t *idx_out, float *rec_out, uint64_t cap,
               uint64_t *n_acc_out, double *eps_out, double *post_out,
               void *workspace, size_t workspace_bytes, void *stream);

/*
 * The exchange step of a job whose samples are split over ranks in
 * contiguous index ranges (the static split of the paper's sampler,
 * Sec. 3.4), for the fixed-N selection of Sec. 3.1.  Each rank selects its
 * own k nearest with abc_select; the global k nearest by (distance, index)
 * are among those candidates, so the ranks gather them and select again.
 *
 * abc_select_candidates: this rank's accepted samples as a candidate record.
 *   dist          device [n] binary64, the distances abc_select ran on.
 *   sample_base   global index of dist[0]; sample_base + n <= 2^32.
 *   idx, rec      device, abc_select's idx_out and rec_out (rec 16-byte
 *                 aligned); count = how many of them to take (<= n).
 *   cand_dist     device [count] binary64: dist[idx[i]].
 *   cand_index    device [count] uint64: sample_base + idx[i].
 *   cand_theta    device [3][count] binary32: the accepted theta (SoA).
 * EINVAL on bad arguments (nothing enqueued).
 */
int abc_select_candidates(const double *dist, uint64_t n, uint64_t sample_base,
                          const uint32_t *idx, const float *rec, uint64_t count,
                          double *cand_dist, uint64_t *cand_index, float *cand_theta,
                          void *stream);

/* Bytes of scratch abc_merge_candidates needs for m candidates and k accepted. */
size_t abc_merge_workspace_bytes(uint64_t m, uint64_t k);

/*
 * The k nearest of m gathered candidates (abc_select_candidates records of
 * all ranks concatenated in rank order, i.e. in ascending global index), by
 * (distance, position): the same set, epsilon and posterior moments as
 * abc_select on the unsharded range.
 *   cand_*        device, as written by abc_select_candidates ([m], [m], [3][m]).
 *   k             1 <= k <= m < 2^32.
 *   idx_out       device [k] uint64: global indices, ascending.
 *   rec_out       device [k] float4 (theta1, theta2, theta3, rho), 16-byte aligned.
 *   n_acc_out     device uint64 (= k); eps_out, post_out nullable device
 *                 ([1] epsilon, [6] posterior mean and unbiased variance).
 *   workspace     device, abc_merge_workspace_bytes(m, k), 256-byte aligned.
 * EINVAL / ENOMEM on bad arguments or a short workspace (nothing enqueued).
 */
int abc_merge_candidates(const double *cand_dist, const uint64_t *cand_index,
                         const float *cand_theta, uint64_t m, uint64_t k,
                         uint64_t *idx_out, float *rec_out, uint64_t *n_acc_out,
                         double *eps_out, double *post_out, void *workspace,
                         size_t workspace_bytes, void *stream);

/* Bytes of scratch abc_rejection needs for a chunk size (256-byte aligned). */
size_t abc_rejection_workspace_bytes(uint64_t chunk);

/*
 * ABC rejection as Algorithm 1 states it: proposals g = 0, 1, 2, ... are
 * simulated as in abc_prior_predictive and accepted when rho <= eps, until
 * m_accept samples are accepted or max_samples proposals are spent.
 * Proposals are taken in index order, so the accepted set is the first
 * m_accept samples of the sequence with rho <= eps, independent of `chunk`
 * (the proposals simulated per launch).
 *   idx_out   [m_accept] uint32 global sample indices, ascending;
 *   rec_out   [m_accept][4] float (th1, th2, th3, (float)rho), 16-byte aligned;
 *   h_counts  host [2]: accepted (<= m_accept), proposals used -- the index
 *             of the m_accept-th acceptance + 1, or every proposal simulated
 *             if fewer were accepted (m_accept / h_counts[1] estimates the
 *             acceptance probability).
 * The host checks the count every 4 chunks, so this call synchronises
 * `stream`; up to 3 chunks past the last acceptance may be simulated (their
 * results are not used).  workspace: abc_rejection_workspace_bytes(chunk).
 */
int abc_rejection(const ppabc_ou_model *h_model, const double *h_y_obs, double eps,
                  uint64_t m_accept, uint64_t max_samples, uint64_t chunk, uint64_t seed,
                  uint32_t substream, uint32_t *idx_out, float *rec_out, uint64_t *h_counts,
                  void *workspace, size_t workspace_bytes, void *stream);

/* Most accepted samples abc_recalibrate takes. */
#define PPABC_RECAL_MAX_Q 32768

/* Bytes of scratch abc_recalibrate needs for n stored pairs and k neighbours. */
size_t abc_recalibrate_workspace_bytes(uint64_t n, uint64_t k);

/*
 * ABC recalibration of an accepted sample (Sec. 5, Discussion: every
 * accepted theta* is recalibrated with a further ABC posterior built from
 * all stored (theta*, D*) pairs, taking its own D* as the observation,
 * through the univariate marginal distribution functions).  For accepted
 * i < q with a = acc_idx[i]:
 *   N_i  = the k pairs j nearest to summ[:, a] (Euclidean over the n_obs
 *          summaries, binary64 with one fma per coordinate in order; ties to
 *          the smaller index; a itself is one of them),
 *   u_out[d][i] = c / k with c = #{j in N_i : theta[d][j] <= theta[d][a]},
 *   theta_rc_out[d][i] = the ceil(c q / k)-th smallest (at least the first) of
 *          theta[d][acc_idx[0..q-1]] -- the u-quantile of the accepted
 *          marginal, i.e. of the posterior given the real observation.
 *   summ     [n_obs][n] double (as abc_prior_predictive's summ_out);
 *   theta    [3][n] float;  acc_idx [q] uint32 (indices >= n give NaN);
 *   u_out    [3][q] double; theta_rc_out [3][q] float.
 * Cost O(q n n_obs); q <= PPABC_RECAL_MAX_Q, 1 <= k <= n.
 */
int abc_recalibrate(const double *summ, const float *theta, uint64_t n, uint32_t n_obs,
                    const uint32_t *acc_idx, uint64_t q, uint64_t k, double *u_out,
                    float *theta_rc_out, void *workspace, size_t workspace_bytes, void *stream);

/* Largest n that abc_select_static accepts. */
#define PPABC_STATIC_SELECT_MAX_N (1ull << 24)

/*
 * abc_select without a workspace argument: identical arguments, outputs and
 * results, but the scratch memory is a fixed static device array inside the
 * library (about 330 KB, held on every GPU that loads the library until the
 * process exits), so the call allocates no memory of any kind.  The paper
 * has no counterpart; this entry point exists for callers that cannot
 * provide device memory -- for example a service that forbids allocation
 * once it is running (an allocation can stall the whole device), or a
 * plug-in hosted by a framework whose allocator it cannot reach.
 *   - n must be <= PPABC_STATIC_SELECT_MAX_N; larger n gives PPABC_EINVAL.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current); make that first call before
 *     any stream capture.  The address stays cached for the life of the
 *     process: cudaDeviceReset, or anything else that destroys and re-creates
 *     the device's primary context, can move the array, and the cached
 *     address then no longer points at it.  Do not call abc_select_static on
 *     a device after resetting it.
 *   - Every call uses the same array and clears what must start at zero, so
 *     calls whose work overlaps on the GPU (different streams, or different
 *     host threads without ordering) race with each other; order them on one
 *     stream.
 */
int abc_select_static(const double *dist, uint64_t n, uint64_t k, double eps,
                      const ppabc_ou_model *h_model, uint64_t sample_base,
                      uint64_t seed, uint32_t substream, const float *theta,
                      uint32_t *idx_out, float *rec_out, uint64_t cap,
                      uint64_t *n_acc_out, double *eps_out, double *post_out,
                      void *stream);

/*
 * ---------------------------------------------------------------------------
 * Batched execution: many uneven OU-ABC jobs in one persistent launch.
 * ---------------------------------------------------------------------------
 * One job is abc_prior_predictive over samples 0..n_samples-1 followed by
 * abc_select with theta redrawn from the prior counter; results are
 * bit-identical to running the job alone with those two calls.
 */
typedef struct ppabc_abc_job {
  ppabc_ou_model model;
  double y_obs[PPABC_MAX_OBS]; /* observed summaries (first model.n_obs used) */
  uint64_t n_samples;          /* 1 .. 2^32-1 */
  uint64_t seed;
  uint32_t substream;
  uint32_t reserved;
  uint64_t k;                  /* > 0: k nearest; 0: dist <= eps */
  double eps;
  double *dist;                /* nullable device [n_samples]: NULL keeps the
                                  distances in the batch workspace */
  uint32_t *idx_out;           /* device [cap] */
  float *rec_out;              /* device [cap][4], 16-byte aligned */
  uint64_t cap;
  uint64_t *n_acc_out;         /* device [1] */
  double *eps_out;             /* nullable device [1] */
  double *post_out;            /* nullable device [6] */
} ppabc_abc_job;

/*
 * Tile shape of the persistent kernel: `threads` per CTA (256 or 512) and the
 * least number of Euler-Maruyama steps one thread runs per tile (a job with S
 * steps gets ceil(min_tile_steps / S) samples per thread, capped at 64).
 * NULL selects (512, 4096).  The Python binding's autotuner picks it.
 */
typedef struct ppabc_tile_config {
  uint32_t threads;
  uint32_t min_tile_steps;
} ppabc_tile_config;

/* Opaque host-side plan of a prepared batch. */
typedef struct ppabc_batch_plan ppabc_batch_plan;

/* Workspace bytes for a batch (job table, schedule, distances of jobs with
 * dist == NULL, selection scratch). */
size_t ppabc_batch_workspace_bytes(const ppabc_abc_job *h_jobs, uint32_t n_jobs);

/*
 * Validates the jobs, uploads the job table into `workspace` and synchronises
 * `stream` once (the upload is the only host-device transfer of a batch).
 * The plan refers to the workspace and to the jobs' output pointers, which
 * must stay valid while the plan is used.
 */
int ppabc_batch_prepare(const ppabc_abc_job *h_jobs, uint32_t n_jobs,
                        const ppabc_tile_config *h_cfg, void *workspace,
                        size_t workspace_bytes, void *stream,
                        ppabc_batch_plan **plan_out);

/* Enqueues the batch (persistent simulation kernel, then one selection per
 * job) on `stream`; no host synchronisation. */
int ppabc_batch_launch(ppabc_batch_plan *plan, void *stream);

/* As ppabc_batch_launch, but the first call captures the launch into a CUDA
 * graph kept in the plan and every call replays it.  `stream` must not be the
 * legacy default stream. */
int ppabc_batch_launch_graph(ppabc_batch_plan *plan, void *stream);

/* Releases the plan (and its graph).  NULL is allowed. */
int ppabc_batch_plan_destroy(ppabc_batch_plan *plan);

/* prepare + launch + destroy. */
int ppabc_batch_run(const ppabc_abc_job *h_jobs, uint32_t n_jobs,
                    const ppabc_tile_config *h_cfg, void *workspace,
                    size_t workspace_bytes, void *stream);

/*
 * ---------------------------------------------------------------------------
 * Request server: continuous batching of ABC and p-value jobs.
 * ---------------------------------------------------------------------------
 * Jobs may be submitted from any host thread at any time.  A scheduler thread
 * admits them in arrival order as soon as one of `n_slots` CUDA streams is
 * free and the job's device footprint fits in the caller's arena (the HBM
 * admission cap), then enqueues the job's whole pipeline on that stream;
 * jobs on different streams overlap on the GPU.  n_slots = 1 gives the plain
 * one-job-at-a-time form.  The server allocates no device memory: every job
 * buffer is carved from the arena.  Accepted samples of an ABC job stay in
 * the arena until ppabc_server_release.  Timestamps are seconds on the
 * server's monotonic clock (ppabc_server_now).
 *
 * An ABC job is abc_prior_predictive over samples 0..n_samples-1 (seed,
 * substream) followed by abc_select of the k nearest with theta redrawn; a
 * p-value job is pvalue_sweep with one lambda.  Results are bit-identical to
 * the same job run alone through those calls.
 */
#define PPABC_JOB_ABC 0
#define PPABC_JOB_PVALUE 1

typedef struct ppabc_request {
  int32_t kind;                /* PPABC_JOB_ABC or PPABC_JOB_PVALUE */
  uint32_t substream;          /* ABC only */
  uint64_t seed;
  ppabc_ou_model model;        /* ABC */
  double y_obs[PPABC_MAX_OBS]; /* ABC */
  uint64_t n_samples;          /* ABC: 1 .. 2^32-1 */
  uint64_t k;                  /* ABC: accept the k nearest, 1 .. n_samples */
  double lambda;               /* p-value: prior sd of mu */
  uint32_t n_obs;              /* p-value: n */
  uint32_t reserved;
  uint64_t m_sets;             /* p-value: data sets M */
  double ybar_obs;             /* p-value */
} ppabc_request;

typedef struct ppabc_result {
  int32_t status;              /* PPABC_OK, PPABC_ECANCELLED or PPABC_ECUDA */
  int32_t kind;
  uint64_t job_id;
  double t_submit, t_admit, t_done;
  uint64_t n_acc;              /* ABC */
  double eps;                  /* ABC */
  double post[6];              /* ABC: posterior means then variances */
  uint64_t count;              /* p-value: tail count */
  double p;                    /* p-value */
} ppabc_result;

typedef struct ppabc_server_stats {
  uint64_t submitted, admitted, completed, failed, cancelled, queued, running;
  uint64_t arena_used_bytes, peak_arena_bytes;
} ppabc_server_stats;

typedef struct ppabc_server ppabc_server;

/* d_arena: device memory the server may use, 256-byte aligned, >= 4096 bytes. */
int ppabc_server_create(void *d_arena, size_t arena_bytes, uint32_t n_slots,
                        ppabc_server **out);
/* PPABC_ENOMEM if the job could never fit in the arena. */
int ppabc_server_submit(ppabc_server *s, const ppabc_request *req, uint64_t *job_id);
/* PPABC_OK and *out filled when finished, PPABC_PENDING otherwise. */
int ppabc_server_poll(ppabc_server *s, uint64_t job_id, ppabc_result *out);
/* Waits up to timeout_s seconds; PPABC_ETIMEOUT if still running. */
int ppabc_server_wait(ppabc_server *s, uint64_t job_id, double timeout_s,
                      ppabc_result *out);
/* Copies up to cap accepted (index, record) pairs of a finished ABC job to
 * host memory (h_idx [cap] uint32, h_rec [cap][4] float; either nullable). */
int ppabc_server_fetch(ppabc_server *s, uint64_t job_id, uint32_t *h_idx,
                       float *h_rec, uint64_t cap, uint64_t *n_out);
/* Frees a finished job's device results and forgets the job. */
int ppabc_server_release(ppabc_server *s, uint64_t job_id);
/* A queued job never runs; a running job's result is discarded. */
int ppabc_server_cancel(ppabc_server *s, uint64_t job_id);
int ppabc_server_get_stats(ppabc_server *s, ppabc_server_stats *out);
double ppabc_server_now(ppabc_server *s);
/* Stops the scheduler after the running jobs finish; NULL is allowed. */
int ppabc_server_destroy(ppabc_server *s);

/*
 * Prior-predictive p-value sweep (Sec. 4.1, Eq. 6 and Eq. 8) for the
 * conjugate model y_i ~ N(mu, 1), i = 1..n_obs, mu ~ N(0, lambda_k^2).  For
 * lambda index k < n_lambda and data set m = set_base .. set_base+m_sets-1,
 * with z_t the normals of stream (seed, index m, substream k, PATH):
 *   ybar = lambda_k z_0 + (1/n_obs) sum_{t=1..n_obs} z_t,
 *   counts[k] = #{m : |ybar| >= |ybar_obs|}  (exact, uint64),
 *   p_out[k]  = counts[k] / m_sets.
 * set_base lets ranks of a sharded sweep take disjoint data-set ranges; the
 * counts of all ranks then add up to the unsharded counts.
 * The statistic ybar is sufficient and its prior predictive law is
 * N(0, lambda^2 + 1/n_obs), whose density falls with |ybar|, so the count is
 * the indicator estimate of P(pi(D) <= pi(D_obs)) (Algorithm 2's estimator).
 * Normals are binary32; each sum is Kahan-compensated binary32 and ybar and
 * the comparison are binary64.
 *   lambda    [n_lambda] double (device).
 *   counts    [n_lambda] uint64; overwritten (zeroed by the call).
 *   p_out     [n_lambda] double (nullable).
 *   ybar_out  [n_lambda][m_sets] double (nullable).
 * Requires 1 <= m_sets, set_base + m_sets <= 2^32, n_obs >= 1.
 */
int pvalue_sweep(const double *lambda, uint32_t n_lambda, uint32_t n_obs,
                 uint64_t m_sets, uint64_t set_base, double ybar_obs, uint64_t seed,
                 uint64_t *counts, double *p_out, double *ybar_out,
                 void *stream);

/* Genetic toggle switch (the paper's example model). */
#define PPABC_TOGGLE_NQ 19        /* summaries: quantiles at 0.05, 0.10, .., 0.95 */
#define PPABC_TOGGLE_MAX_CELLS 16384
#define PPABC_TAG_TOGGLE_PRIOR 4u
#define PPABC_TAG_TOGGLE_PATH 5u

/*
 * Toggle-switch model (Sec. 3.2, Eq. 3-4): theta = (mu, sigma, gamma,
 * alpha_u, alpha_v, beta_u, beta_v) with independent uniform priors
 * U(lo[j], hi[j]) (the paper's box is U(250,400) x U(0.05,0.5) x
 * U(0.05,0.35) x U(0,50)^2 x U(0,7)^2); C cells, T time points (T-1
 * Euler-Maruyama steps of size 1, Eq. 5).
 */
typedef struct ppabc_toggle_model {
  double lo[7];
  double hi[7];
  uint32_t T;  /* >= 2 */
  uint32_t C;  /* 1 .. PPABC_TOGGLE_MAX_CELLS */
} ppabc_toggle_model;

/*
 * Toggle-switch prior predictive for ABC, one sample per global index
 * g = sample_base + i: theta from counters (TOGGLE_PRIOR, 0|1, substream, g);
 * cell c evolves from u = v = 10 with, at step j = 1..T-1,
 *   u = max(0.97 u + alpha_u / (1 + v^beta_u) - 1 + 0.5 zeta_u, 1),
 *   v = max(0.97 v + alpha_v / (1 + u^beta_v) - 1 + 0.5 zeta_v, 1)
 * (both from the previous u, v; zeta_u, zeta_v are normals 2(j-1), 2(j-1)+1
 * of stream (index c, substream g, tag (substream << 8) | TOGGLE_PATH)),
 * and is observed as
 * y = max(u + mu + mu sigma eta / u^gamma, 1), eta = normal 2(T-1).
 * S(D*) = the quantiles at levels k/20, k = 1..19 (linear interpolation
 * between order statistics: h = (C-1) k / 20), rho = ||S - q_obs||_2.
 * The path is binary32; quantiles and rho are binary64.
 *   h_q_obs     19 observed quantiles (host).
 *   theta_out   nullable [7][n] float;  summ_out nullable [19][n] double;
 *   y_out       nullable [n][C] float (every cell's observation);
 *   dist_out    [n] double.
 * Requires substream < 2^24 and sample_base + n <= 2^32.
 */
int toggle_prior_predictive(const ppabc_toggle_model *h_model, const double *h_q_obs,
                            uint64_t n, uint64_t sample_base, uint64_t seed,
                            uint32_t substream, float *theta_out, double *summ_out,
                            float *y_out, double *dist_out, void *stream);

/* Most data sets per hyperparameter in weakinf_test. */
#define PPABC_WEAKINF_MAX_SETS 16384

/*
 * Weak-informativity test (Sec. 4.1, Eq. 9 and Algorithm 2) for the
 * conjugate model y_i ~ N(mu, 1), i = 1..n_obs, mu ~ N(0, lambda^2), base
 * hyperparameter lambda0.  For each k < n_lambda:
 *   base sets   i < N: ybar_0^i of stream (seed, index i, substream k, BASE), lambda0,
 *   lambda sets j < N: ybar_k^j of stream (seed, index j, substream k, PATH), lambda[k],
 *   count_k^i = #{j : |ybar_k^j| >= |ybar_0^i|}      (p_k^i = count_k^i / N),
 *   gamma_out[k] = the ceil(alpha N)-th smallest p_k^i (the alpha quantile).
 * Priors with gamma_k > gamma_0 for lambda_0 = lambda0 are weakly informative
 * relative to the base prior (Eq. 9).  ybar as in pvalue_sweep; the
 * comparisons are binary64.
 *   lambda      [n_lambda] double (device).
 *   gamma_out   [n_lambda] double (device).
 *   counts_out  nullable [n_lambda][N] uint32 (device).
 *   workspace   weakinf_test_workspace_bytes(n_lambda, N) bytes (the |ybar| of
 *               every data set), 256-byte aligned.
 * Requires 1 <= N <= PPABC_WEAKINF_MAX_SETS, 0 < alpha <= 1, n_obs >= 1.
 */
size_t weakinf_test_workspace_bytes(uint64_t n_lambda, uint64_t n_sets);
int weakinf_test(const double *lambda, uint32_t n_lambda, double lambda0, uint32_t n_obs,
                 uint64_t n_sets, double alpha, uint64_t seed, double *gamma_out,
                 uint32_t *counts_out, void *workspace, size_t workspace_bytes, void *stream);

/* BEGE likelihood limits and constants. */
#define PPABC_BEGE_NPAR 11
#define PPABC_BEGE_NW 100
#define PPABC_BEGE_MAX_PARTICLES (1 << 20)
#define PPABC_BEGE_MAX_T (1 << 16)

/*
 * BEGE log-likelihood (Sec. 4.2: the BEGE model of monthly return
 * innovations, its shape recursion, Eq. BEGE_LL, the distribution function
 * Eq. CDF_BEGE discretised as Eq. BEGE_LL_approx, P(a, x) of Eq. incompGamma)
 * for n_particles parameter vectors on one return series r_1..r_T.
 * Particle i has theta = (p0, sigma_p, rho_p, phi_p+, phi_p-, n0, sigma_n,
 * rho_n, phi_n+, phi_n-, mu), row k of theta holding parameter k of every
 * particle.  With u_t = r_t - mu:
 *   ll_i = sum_{t=1..T} log f(u_t; sigma_p, sigma_n, p_{t-1}, n_{t-1}),
 *   p_t = p0 + rho_p p_{t-1} + phi_p^{+|-} u_t^2 / (2 sigma_p^2)   (+ if u_t >= 0),
 *   n_t likewise with sigma_n, rho_n, phi_n^{+|-};  (p_0, n_0) = (p0, n0),
 *   f(u) = (F(u + h) - F(u - h)) / (2 h),
 *   F(u) = sum_{j=1..100} [1 - P(n, (w_{j-1} - u + n sigma_n) / sigma_n)]
 *                          [P(p, (w_j + p sigma_p) / sigma_p) - P(p, (w_{j-1} + p sigma_p) / sigma_p)],
 *   w_j = w_0 + j dw,  w_0 = 1e-4 - p sigma_p,  dw = (10 sigma_p sqrt(p) - w_0) / 99,
 * P(a, x) the regularised lower incomplete gamma (0 for x <= 0): its power
 * series for x < a + 1 and Legendre's continued fraction for the complement
 * otherwise.  A scale <= 0, a shape that is not a positive finite number, or
 * a density that is not a positive finite number, gives ll_i = -inf.  The
 * inputs, shapes and sums over t are binary64; the per-node work (P(a, x),
 * its prefactor exp(a ln x - x - lgamma(a)), and F(u + h) - F(u - h) taken
 * node by node, away from the support's edge from the Taylor expansion of
 * P(n, .) to fifth order in h / sigma_n) runs in double-float (two binary32
 * numbers, about 48 bits).
 *   theta      [11][n_particles] double (device).
 *   r          [T] double (device): the returns r_1..r_T.
 *   h          finite-difference step, 0 < h < 1.
 *   ll_out     [n_particles] double (device).
 *   logf_out   nullable [n_particles][T] double (device): log f per step
 *              (NaN after the step that ended a particle).
 *   workspace  bege_loglik_workspace_bytes(n_particles, T) bytes, 256-byte aligned.
 * Requires 1 <= n_particles <= PPABC_BEGE_MAX_PARTICLES, 1 <= T <= PPABC_BEGE_MAX_T.
 */
size_t bege_loglik_workspace_bytes(uint64_t n_particles, uint32_t T);
int bege_loglik(const double *theta, uint64_t n_particles, const double *r, uint32_t T, double h,
                double *ll_out, double *logf_out, void *workspace, size_t workspace_bytes,
                void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PPABC_H */
