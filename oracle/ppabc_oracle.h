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
 *   - counter = (c0 tag, c1 block, c2 substream, c3 sample or data-set index):
 *     normal j of the stream (index, substream, tag) is lane j%4 of the
 *     block j/4, and a prior draw is block 0 of its tag;
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
#define ORC_TAG_BASE 2u
#define ORC_TAG_TOGGLE_PRIOR 4u
#define ORC_TAG_TOGGLE_PATH 5u
#define ORC_TOGGLE_NQ 19

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

/* Box-Muller on given word pairs: w is [n][2] (even, odd), z is [n][2]. */
void orc_box_muller_words(const uint32_t *w, uint64_t n, double *z);

/* Normals j0 .. j0+n-1 of stream (seed, index c1, substream c2, tag): normal
 * j comes from counter (tag, j/4, c2, c1), lane j%4. */
void orc_stream_normals(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t tag,
                        uint64_t j0, uint64_t n, double *z);

/* Prior-predictive OU samples i = base .. base+n-1 (the sample index is the
 * stream index, counter word c3).  Outputs (each may be NULL except dist):
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
 * (seed, index m, substream k, PATH) give mu = lam_k z_0 and
 * ybar = mu + (1/n) sum_{i=1..n} z_i; counts[k] = #{m : |ybar| >= |ybar_obs|},
 * p[k] = counts[k] / M.  ybar (nullable) is [n_lambda][M]. */
int orc_pvalue_sweep(const double *lambda, uint32_t n_lambda, uint32_t n_obs,
                     uint64_t m_sets, uint64_t base, double ybar_obs, uint64_t seed,
                     uint64_t *counts, double *p, double *ybar, int n_threads);

/* Weak-informativity test (Algorithm 2) for the conjugate normal model, with
 * the sufficient statistic ybar.  For each k < n_lambda:
 *   base sets   i < N: ybar0 from stream (seed, index i, substream k, BASE), lambda_0,
 *   lambda sets j < N: ybar  from stream (seed, index j, substream k, PATH), lambda_k,
 *   p_k^i = #{j : |ybar_k^j| >= |ybar0_k^i|} / N           (indicator estimate)
 *   gamma_k = the ceil(alpha N)-th smallest of p_k^1..p_k^N (alpha quantile).
 * counts (nullable) is [n_lambda][N] (the numerators of p_k^i). */
int orc_weakinf(const double *lambda, uint32_t n_lambda, double lambda0, uint32_t n_obs,
                uint64_t n_sets, double alpha, uint64_t seed, double *gamma,
                uint64_t *counts, int n_threads);

/* Genetic toggle switch (Sec. 3.2-3.4): theta = (mu, sigma, gamma, alpha_u,
 * alpha_v, beta_u, beta_v) with independent uniform priors on [lo, hi];
 * C cells, each evolved over T-1 Euler-Maruyama steps (Delta t = 1) from
 * u = v = 10, then observed with noise; summaries are the 19 quantiles at
 * levels 0.05 .. 0.95 (linear interpolation between order statistics).
 * Random numbers, for sample g:
 *   prior:  counters (TOGGLE_PRIOR, 0, sub, g) words 0..3 -> theta_0..3 and
 *           (TOGGLE_PRIOR, 1, sub, g) words 0..2 -> theta_4..6;
 *   cell c: stream (index c, substream g, tag (sub << 8) | TOGGLE_PATH):
 *           normal 2(j-1) and 2(j-1)+1 drive u and v at step j = 1..T-1,
 *           normal 2(T-1) is eta. */
typedef struct orc_toggle_model {
  double lo[7];
  double hi[7];
  uint32_t T;
  uint32_t C;
} orc_toggle_model;

/* uv (nullable) receives the final (u, v) of every cell, [n][C][2]. */
int orc_toggle_prior_predictive(const orc_toggle_model *m, const double *q_obs, uint64_t base,
                                uint64_t n, uint64_t seed, uint32_t sub, double *theta,
                                double *summ, double *y, double *uv, double *dist, int n_threads);

/* ABC recalibration.  summ is [n_obs][n] (column j = the summaries of pair j),
 * theta [3][n], acc [q] indices of the accepted pairs.  For accepted i with
 * a = acc[i]: the k pairs nearest to summ[:, a] (Euclidean, ties to the
 * smaller index, a itself included), u[d][i] = #{neighbours j : theta[d][j]
 * <= theta[d][a]} / k = c / k, and theta_rc[d][i] = the ceil(c q / k)-th
 * smallest (at least the first) of theta[d][acc[0..q-1]], the rank formed in
 * integers.  Distances use fma for every
 * squared difference, in summary order. */
int orc_recalibrate(const double *summ, const float *theta, uint64_t n, uint32_t n_obs,
                    const uint32_t *acc, uint64_t q, uint64_t k, double *u, float *theta_rc,
                    int n_threads);

/* BEGE log-likelihood (Sec. 4.2).  theta is [ORC_BEGE_NPAR][np] (row k =
 * parameter k of every particle) in the order (p0, sigma_p, rho_p, phi_p+,
 * phi_p-, n0, sigma_n, rho_n, phi_n+, phi_n-, mu); r holds r_1..r_T; the
 * density is the central difference of the discretised distribution function
 * with step h.  ll[np] gets each log-likelihood (-inf where a scale is not
 * positive, or a shape or a density is not a positive finite number);
 * dens[np][T], if non-NULL, the densities (NaN after the step that ended a
 * particle). */
#define ORC_BEGE_NPAR 11
#define ORC_BEGE_NW 100
double orc_gammainc_p(double a, double x);
double orc_bege_cdf(double u, double sp, double sn, double p, double n);
double orc_bege_density(double u, double sp, double sn, double p, double n, double h);
int orc_bege_loglik(const double *theta, uint64_t np, const double *r, uint32_t T, double h,
                    double *ll, double *dens, int n_threads);

#ifdef __cplusplus
}
#endif

#endif /* PPABC_ORACLE_H */
