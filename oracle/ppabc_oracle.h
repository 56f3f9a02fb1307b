/*
 * ppabc_oracle.h -- plain FP64 CPU oracle for prior-predictive Monte Carlo
 * (Warne, Sisson & Drovandi, "Vector operations for accelerating expensive
 * Bayesian computations -- a tutorial guide", arXiv:1902.09046).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously correct
 * reference that the CUDA path is checked against.  It shares no source with
 * the CUDA path and must only be loaded by the test-suite, by the smoke check
 * and by the CPU-baseline leg of the benchmark.  Nothing in the product path
 * may call it.
 *
 * Conventions shared *by definition* (not by code) with the CUDA path:
 *   - Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) keyed by the 64-bit
 *     seed split as key = (seed & 0xffffffff, seed >> 32);
 *   - counter = (c0 block, c1 sample or data-set index, c2 substream, c3 tag);
 *   - uniform  u(w) = ((w >> 9) + 1/2) * 2^-23, an exact value in (0,1);
 *   - Box-Muller: (w_even, w_odd) -> r = sqrt(-2 ln u(w_even)),
 *     z_even = r cos(2 pi u(w_odd)), z_odd = r sin(2 pi u(w_odd)).
 * All arithmetic below is IEEE binary64.
 */
#ifndef PPABC_ORACLE_H
#define PPABC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_TAG_PRIOR 0u
#define ORC_TAG_PATH 1u

/* OU model for ABC: dX = th1 (th2 - X) dt + th3 dW, X(0) = x0, with
 * independent uniform priors th_j ~ U(lo[j], hi[j]). */
typedef struct orc_ou_model {
  double lo[3];
  double hi[3];
  double x0;
  double dt;
  uint32_t n_steps;
  uint32_t n_obs;
} orc_ou_model;

/* One Philox4x32-10 block: out = philox(ctr, key). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]);

/* n blocks: ctr is [n][4], out is [n][4]; key from the 64-bit seed. */
void orc_philox_batch(uint64_t seed, const uint32_t *ctr, uint64_t n,
                      uint32_t *out);

/* The uniform that a 32-bit word encodes (see header comment). */
double orc_u01(uint32_t w);

/* Normals j0 .. j0+n-1 of stream (seed, c1, c2, tag): normal j comes from
 * counter block j/4, lane j%4. */
void orc_stream_normals(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t tag,
                        uint64_t j0, uint64_t n, double *z);

/* Prior-predictive OU samples i = base .. base+n-1 (sample index enters the
 * counter as c1).  Outputs (each may be NULL except dist):
 *   theta [n][3], summ [n][n_obs] (X at the observation steps), dist [n].
 * Returns 0, or -1 on invalid arguments. */
int orc_ou_prior_predictive(const orc_ou_model *m, const double *y_obs,
                            uint64_t base, uint64_t n, uint64_t seed,
                            uint32_t sub, double *theta, double *summ,
                            double *dist, int n_threads);

/* The k samples with the smallest (dist, index), written as indices in
 * ascending index order.  Returns 0, -1 if k > n. */
int orc_select_topk(const double *dist, uint64_t n, uint64_t k,
                    uint64_t *idx_out);

/* All i with dist[i] <= eps, in ascending index order; returns the count. */
uint64_t orc_select_eps(const double *dist, uint64_t n, double eps,
                        uint64_t *idx_out);

/* Mean and unbiased (k-1) variance of theta[idx[j]][0..2]; theta is [.][3].
 * mean is NaN for k = 0, var is NaN for k < 2. */
void orc_moments(const double *theta, const uint64_t *idx, uint64_t k,
                 double mean[3], double var[3]);

/* Prior-predictive p-value sweep for y_i ~ N(mu,1), i=1..n, mu ~ N(0,lam^2):
 * for each lambda_k and data set m = base..base+M-1 the normals of stream
 * (seed, c1 = m, c2 = k, PATH) give mu = lam_k z_0 and
 * ybar = mu + (1/n) sum_{i=1..n} z_i; counts[k] = #{m : |ybar| >= |ybar_obs|},
 * p[k] = counts[k] / M.  ybar (nullable) is [n_lambda][M]. */
int orc_pvalue_sweep(const double *lambda, uint32_t n_lambda, uint32_t n_obs,
                     uint64_t m_sets, uint64_t base, double ybar_obs, uint64_t seed,
                     uint64_t *counts, double *p, double *ybar, int n_threads);

#ifdef __cplusplus
}
#endif

#endif /* PPABC_ORACLE_H */
