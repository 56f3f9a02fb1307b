/*
 * ppabc_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * The slow, obviously correct reference for the prior-predictive Monte Carlo
 * path of Warne, Sisson & Drovandi (arXiv:1902.09046).  Every function follows
 * one passage of the paper (cited at the function) or one published
 * definition, in the paper's order, with no blocking, fusion or reordering.
 * Loaded only by tests, the smoke check and the benchmark's CPU-baseline leg;
 * it shares no code with the CUDA path.
 *
 * Threads (where a function takes n_threads) split the sample range into
 * equal contiguous pieces, which is the static schedule the paper uses for its
 * OpenMP prior-predictive sampler (Sec. 3.4).  Each sample depends only on its
 * own counter, so the split changes no result.
 */
#include "ppabc_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------------
 * Philox4x32-10 (Salmon et al., SC'11, "Parallel random numbers: as easy as
 * 1, 2, 3").  The paper needs independent streams per worker (Sec. 2.5); of
 * its three options this is (ii), a generator that splits into sub-streams,
 * here by the counter.  One round maps (c0,c1,c2,c3) with key (k0,k1) to
 *   (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
 * and the key is bumped by the Weyl constants between rounds.
 * ------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

static void seed_to_key(uint64_t seed, uint32_t key[2]) {
  key[0] = (uint32_t)(seed & 0xffffffffu);
  key[1] = (uint32_t)(seed >> 32);
}

void orc_philox_batch(uint64_t seed, const uint32_t *ctr, uint64_t n,
                      uint32_t *out) {
  uint32_t key[2];
  seed_to_key(seed, key);
  for (uint64_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* u(w) = ((w >> 9) + 1/2) 2^-23: the midpoint of one of 2^23 equal cells of
 * (0,1), never 0 or 1. */
double orc_u01(uint32_t w) { return ((double)(w >> 9) + 0.5) * 0x1p-23; }

/* Box-Muller transform (the paper draws its normals with MKL's Box-Muller
 * method, Sec. 3.4): two uniforms give two independent standard normals. */
static void box_muller(uint32_t w_even, uint32_t w_odd, double *z_even,
                       double *z_odd) {
  const double two_pi = 6.283185307179586476925286766559;
  double u1 = orc_u01(w_even);
  double u2 = orc_u01(w_odd);
  double r = sqrt(-2.0 * log(u1));
  *z_even = r * cos(two_pi * u2);
  *z_odd = r * sin(two_pi * u2);
}

void orc_box_muller_words(const uint32_t *w, uint64_t n, double *z) {
  for (uint64_t i = 0; i < n; ++i) box_muller(w[2 * i], w[2 * i + 1], &z[2 * i], &z[2 * i + 1]);
}

/* The four normals of block b of the stream (index c1, substream c2, tag):
 * counter (tag, b, c2, c1). */
static void block_normals(const uint32_t key[2], uint32_t b, uint32_t c1,
                          uint32_t c2, uint32_t tag, double z[4]) {
  uint32_t ctr[4] = {tag, b, c2, c1};
  uint32_t w[4];
  orc_philox4x32_10(ctr, key, w);
  box_muller(w[0], w[1], &z[0], &z[1]);
  box_muller(w[2], w[3], &z[2], &z[3]);
}

void orc_stream_normals(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t tag,
                        uint64_t j0, uint64_t n, double *z) {
  uint32_t key[2];
  seed_to_key(seed, key);
  for (uint64_t t = 0; t < n; ++t) {
    uint64_t j = j0 + t;
    double zb[4];
    block_normals(key, (uint32_t)(j / 4), c1, c2, tag, zb);
    z[t] = zb[j % 4];
  }
}

/* ---------------------------------------------------------------------------
 * Prior-predictive sampling for ABC (Sec. 3.1, Eq. 2 and Algorithm 1, in the
 * fixed-N form the paper describes after Algorithm 1), with the model
 * simulated by the Euler-Maruyama scheme (Sec. 3.3, Eq. 5) applied to the
 * Ornstein-Uhlenbeck SDE dX = th1 (th2 - X) dt + th3 dW.
 *
 * For sample i:
 *   1. theta* ~ pi(theta): th_j = lo_j + (hi_j - lo_j) u(w_j), w = Philox
 *      counter (PRIOR, 0, sub, i) (uniform priors, as in the paper's sampler).
 *   2. D* ~ s(D; theta*): X_0 = x0 and for s = 1..S
 *        X_s = X_{s-1} + th1 (th2 - X_{s-1}) dt + th3 sqrt(dt) xi_{s-1},
 *      xi_j = normal j of stream (seed, i, sub, PATH).
 *   3. S(D*): X at the observation steps s_j = floor(j S / n_obs),
 *      j = 1..n_obs.
 *   4. rho = Euclidean distance between S(D*) and the observed summaries.
 * ------------------------------------------------------------------------- */
static void ou_one_sample(const orc_ou_model *m, const double *y_obs,
                          const uint32_t key[2], uint64_t i, uint32_t sub,
                          double *theta, double *summ, double *dist) {
  uint32_t prior_ctr[4] = {ORC_TAG_PRIOR, 0u, sub, (uint32_t)i};
  uint32_t w[4];
  orc_philox4x32_10(prior_ctr, key, w);
  double th[3];
  for (int j = 0; j < 3; ++j) th[j] = m->lo[j] + (m->hi[j] - m->lo[j]) * orc_u01(w[j]);
  if (theta) {
    theta[0] = th[0];
    theta[1] = th[1];
    theta[2] = th[2];
  }

  const double dt = m->dt;
  const double sqrt_dt = sqrt(dt);
  const uint32_t S = m->n_steps, n_obs = m->n_obs;
  double X = m->x0;
  double acc = 0.0;
  uint32_t j = 1;
  uint64_t s_next = ((uint64_t)j * S) / n_obs;
  double z[4];
  for (uint32_t s = 1; s <= S; ++s) {
    uint32_t jz = s - 1; /* index of the normal this step consumes */
    if (jz % 4 == 0) block_normals(key, jz / 4, (uint32_t)i, sub, ORC_TAG_PATH, z);
    double xi = z[jz % 4];
    X = X + th[0] * (th[1] - X) * dt + th[2] * sqrt_dt * xi;
    if (s == s_next) {
      double r = X - y_obs[j - 1];
      if (summ) summ[j - 1] = X;
      acc += r * r;
      ++j;
      s_next = (j <= n_obs) ? ((uint64_t)j * S) / n_obs : 0;
    }
  }
  *dist = sqrt(acc);
}

typedef struct ou_job {
  const orc_ou_model *m;
  const double *y_obs;
  uint32_t key[2];
  uint64_t base, lo, hi;
  uint32_t sub;
  double *theta, *summ, *dist;
} ou_job;

static void *ou_worker(void *arg) {
  ou_job *J = (ou_job *)arg;
  for (uint64_t t = J->lo; t < J->hi; ++t) {
    ou_one_sample(J->m, J->y_obs, J->key, J->base + t, J->sub,
                  J->theta ? J->theta + 3 * t : NULL,
                  J->summ ? J->summ + (uint64_t)J->m->n_obs * t : NULL,
                  J->dist + t);
  }
  return NULL;
}

int orc_ou_prior_predictive(const orc_ou_model *m, const double *y_obs,
                            uint64_t base, uint64_t n, uint64_t seed,
                            uint32_t sub, double *theta, double *summ,
                            double *dist, int n_threads) {
  if (!m || !y_obs || !dist) return -1;
  if (m->n_obs == 0 || m->n_steps < m->n_obs || !(m->dt > 0.0)) return -1;
  if (base + n > 0x100000000ull) return -1;
  if (n_threads < 1) n_threads = 1;
  if ((uint64_t)n_threads > n) n_threads = (int)(n > 0 ? n : 1);
  ou_job *jobs = (ou_job *)calloc((size_t)n_threads, sizeof(ou_job));
  pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  if (!jobs || !th) {
    free(jobs);
    free(th);
    return -1;
  }
  for (int t = 0; t < n_threads; ++t) {
    ou_job *J = &jobs[t];
    J->m = m;
    J->y_obs = y_obs;
    seed_to_key(seed, J->key);
    J->base = base;
    J->lo = n * (uint64_t)t / (uint64_t)n_threads;
    J->hi = n * (uint64_t)(t + 1) / (uint64_t)n_threads;
    J->sub = sub;
    J->theta = theta;
    J->summ = summ;
    J->dist = dist;
  }
  for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, ou_worker, &jobs[t]);
  ou_worker(&jobs[0]);
  for (int t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
  free(jobs);
  free(th);
  return 0;
}

/* ---------------------------------------------------------------------------
 * Selection.  The paper fixes N and then picks epsilon a posteriori from the
 * empirical distribution of the discrepancy (Sec. 3.1, after Algorithm 1):
 * accepting the k nearest is choosing epsilon as the k-th smallest distance.
 * Ties in distance are broken by the smaller sample index, so the accepted
 * set always has exactly k members.  NaN distances sort after everything.
 * ------------------------------------------------------------------------- */
typedef struct dist_idx {
  double d;
  uint64_t i;
} dist_idx;

static int cmp_dist_idx(const void *a, const void *b) {
  const dist_idx *x = (const dist_idx *)a, *y = (const dist_idx *)b;
  int xn = isnan(x->d), yn = isnan(y->d);
  if (xn != yn) return xn - yn;
  if (!xn) {
    if (x->d < y->d) return -1;
    if (x->d > y->d) return 1;
  }
  return (x->i > y->i) - (x->i < y->i);
}

static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return (x > y) - (x < y);
}

int orc_select_topk(const double *dist, uint64_t n, uint64_t k,
                    uint64_t *idx_out) {
  if (k > n) return -1;
  if (k == 0) return 0;
  dist_idx *a = (dist_idx *)malloc((size_t)n * sizeof(dist_idx));
  if (!a) return -1;
  for (uint64_t i = 0; i < n; ++i) {
    a[i].d = dist[i];
    a[i].i = i;
  }
  qsort(a, (size_t)n, sizeof(dist_idx), cmp_dist_idx);
  for (uint64_t j = 0; j < k; ++j) idx_out[j] = a[j].i;
  free(a);
  qsort(idx_out, (size_t)k, sizeof(uint64_t), cmp_u64);
  return 0;
}

/* Algorithm 1's acceptance test rho <= epsilon, applied to every sample. */
uint64_t orc_select_eps(const double *dist, uint64_t n, double eps,
                        uint64_t *idx_out) {
  uint64_t c = 0;
  for (uint64_t i = 0; i < n; ++i)
    if (dist[i] <= eps) idx_out[c++] = i;
  return c;
}

/* Posterior summaries of the accepted sample: mean, then the unbiased
 * variance about that mean (two passes). */
void orc_moments(const double *theta, const uint64_t *idx, uint64_t k,
                 double mean[3], double var[3]) {
  for (int j = 0; j < 3; ++j) {
    if (k == 0) {
      mean[j] = NAN;
      var[j] = NAN;
      continue;
    }
    double s = 0.0;
    for (uint64_t t = 0; t < k; ++t) s += theta[3 * idx[t] + j];
    mean[j] = s / (double)k;
    if (k < 2) {
      var[j] = NAN;
      continue;
    }
    double q = 0.0;
    for (uint64_t t = 0; t < k; ++t) {
      double r = theta[3 * idx[t] + j] - mean[j];
      q += r * r;
    }
    var[j] = q / (double)(k - 1);
  }
}

/* ---------------------------------------------------------------------------
 * Prior-predictive p-value (Sec. 4.1, Eq. 6 and Eq. 8) for the conjugate
 * normal model y_i ~ N(mu, 1), mu ~ N(0, lambda^2).  The sufficient statistic
 * ybar has prior predictive density N(0, lambda^2 + 1/n), which decreases in
 * |ybar|, so the event pi(D) <= pi(D_obs) is |ybar| >= |ybar_obs|.  The
 * probability is estimated by the indicator count of Algorithm 2's inner
 * loop over M prior-predictive data sets.
 * ------------------------------------------------------------------------- */
/* ybar of one prior-predictive data set: normals z_0..z_n of stream
 * (seed, c1, c2, tag), mu = lam z_0, ybar = mu + (1/n) sum_{t=1..n} z_t. */
static double ybar_of(const uint32_t key[2], double lam, uint32_t n_obs, uint32_t c1, uint32_t c2,
                      uint32_t tag) {
  double z[4];
  double mu = 0.0, s = 0.0;
  for (uint32_t t = 0; t <= n_obs; ++t) {
    if (t % 4 == 0) block_normals(key, t / 4, c1, c2, tag, z);
    if (t == 0)
      mu = lam * z[0];
    else
      s += z[t % 4];
  }
  return mu + s / (double)n_obs;
}

typedef struct pv_job {
  const double *lambda;
  uint32_t n_lambda, n_obs;
  uint64_t m_sets, base, lo, hi; /* flat range over (k, m) */
  double ybar_obs;
  uint32_t key[2];
  uint64_t *counts; /* [n_lambda], private to the worker */
  double *ybar;
} pv_job;

static void *pv_worker(void *arg) {
  pv_job *J = (pv_job *)arg;
  for (uint64_t f = J->lo; f < J->hi; ++f) {
    uint32_t k = (uint32_t)(f / J->m_sets);
    uint64_t m = J->base + f % J->m_sets;
    double ybar = ybar_of(J->key, J->lambda[k], J->n_obs, (uint32_t)m, k, ORC_TAG_PATH);
    if (J->ybar) J->ybar[f] = ybar;
    if (fabs(ybar) >= fabs(J->ybar_obs)) J->counts[k] += 1;
  }
  return NULL;
}

int orc_pvalue_sweep(const double *lambda, uint32_t n_lambda, uint32_t n_obs,
                     uint64_t m_sets, uint64_t base, double ybar_obs, uint64_t seed,
                     uint64_t *counts, double *p, double *ybar, int n_threads) {
  if (!lambda || !counts || n_lambda == 0 || n_obs == 0 || m_sets == 0) return -1;
  if (m_sets > 0x100000000ull || base > 0x100000000ull - m_sets) return -1;
  uint64_t total = (uint64_t)n_lambda * m_sets;
  if (n_threads < 1) n_threads = 1;
  if ((uint64_t)n_threads > total) n_threads = (int)total;
  pv_job *jobs = (pv_job *)calloc((size_t)n_threads, sizeof(pv_job));
  pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  uint64_t *priv = (uint64_t *)calloc((size_t)n_threads * n_lambda, sizeof(uint64_t));
  if (!jobs || !th || !priv) {
    free(jobs);
    free(th);
    free(priv);
    return -1;
  }
  for (int t = 0; t < n_threads; ++t) {
    pv_job *J = &jobs[t];
    J->lambda = lambda;
    J->n_lambda = n_lambda;
    J->n_obs = n_obs;
    J->m_sets = m_sets;
    J->base = base;
    J->lo = total * (uint64_t)t / (uint64_t)n_threads;
    J->hi = total * (uint64_t)(t + 1) / (uint64_t)n_threads;
    J->ybar_obs = ybar_obs;
    seed_to_key(seed, J->key);
    J->counts = priv + (size_t)t * n_lambda;
    J->ybar = ybar;
  }
  for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, pv_worker, &jobs[t]);
  pv_worker(&jobs[0]);
  for (int t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
  for (uint32_t k = 0; k < n_lambda; ++k) {
    uint64_t c = 0;
    for (int t = 0; t < n_threads; ++t) c += priv[(size_t)t * n_lambda + k];
    counts[k] = c;
    if (p) p[k] = (double)c / (double)m_sets;
  }
  free(jobs);
  free(th);
  free(priv);
  return 0;
}

/* ---------------------------------------------------------------------------
 * Weak-informativity test (Sec. 4.1, Eq. 9 and Algorithm 2) for the conjugate
 * normal model.  Algorithm 2 draws, for every hyperparameter lambda_k, N data
 * sets from the base prior predictive and N from the lambda_k prior
 * predictive, estimates the p-value of every base data set under lambda_k by
 * the indicator average over the lambda_k data sets, and returns the alpha
 * quantile of those p-values.  With the sufficient statistic ybar, whose
 * prior predictive density under lambda falls with |ybar|, the event
 * pi(D_k^j | lambda_k) <= pi(D_0^i | lambda_k) is |ybar_k^j| >= |ybar_0^i|.
 * The comparisons are done by brute force over all (i, j) pairs.
 * ------------------------------------------------------------------------- */
static int cmp_u64_asc(const void *a, const void *b) { return cmp_u64(a, b); }

typedef struct wi_job {
  const double *lambda;
  double lambda0;
  uint32_t n_obs, k_lo, k_hi;
  uint64_t n_sets;
  double alpha;
  uint32_t key[2];
  double *gamma;
  uint64_t *counts;
  int rc;
} wi_job;

static void *wi_worker(void *arg) {
  wi_job *J = (wi_job *)arg;
  const uint64_t N = J->n_sets;
  double *y0 = (double *)malloc(N * sizeof(double));
  double *yk = (double *)malloc(N * sizeof(double));
  uint64_t *cnt = (uint64_t *)malloc(N * sizeof(uint64_t));
  if (!y0 || !yk || !cnt) {
    J->rc = -1;
    free(y0);
    free(yk);
    free(cnt);
    return NULL;
  }
  for (uint32_t k = J->k_lo; k < J->k_hi; ++k) {
    for (uint64_t i = 0; i < N; ++i) {
      y0[i] = ybar_of(J->key, J->lambda0, J->n_obs, (uint32_t)i, k, ORC_TAG_BASE);
      yk[i] = ybar_of(J->key, J->lambda[k], J->n_obs, (uint32_t)i, k, ORC_TAG_PATH);
    }
    for (uint64_t i = 0; i < N; ++i) {
      uint64_t c = 0;
      for (uint64_t j = 0; j < N; ++j)
        if (fabs(yk[j]) >= fabs(y0[i])) ++c;
      cnt[i] = c;
      if (J->counts) J->counts[(uint64_t)k * N + i] = c;
    }
    qsort(cnt, (size_t)N, sizeof(uint64_t), cmp_u64_asc);
    uint64_t r = (uint64_t)ceil(J->alpha * (double)N);
    if (r < 1) r = 1;
    if (r > N) r = N;
    J->gamma[k] = (double)cnt[r - 1] / (double)N;
  }
  free(y0);
  free(yk);
  free(cnt);
  return NULL;
}

int orc_weakinf(const double *lambda, uint32_t n_lambda, double lambda0, uint32_t n_obs,
                uint64_t n_sets, double alpha, uint64_t seed, double *gamma,
                uint64_t *counts, int n_threads) {
  if (!lambda || !gamma || n_lambda == 0 || n_obs == 0 || n_sets == 0) return -1;
  if (n_sets > 0x100000000ull || !(alpha > 0.0 && alpha <= 1.0)) return -1;
  if (n_threads < 1) n_threads = 1;
  if ((uint32_t)n_threads > n_lambda) n_threads = (int)n_lambda;
  wi_job *jobs = (wi_job *)calloc((size_t)n_threads, sizeof(wi_job));
  pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  if (!jobs || !th) {
    free(jobs);
    free(th);
    return -1;
  }
  for (int t = 0; t < n_threads; ++t) {
    wi_job *J = &jobs[t];
    J->lambda = lambda;
    J->lambda0 = lambda0;
    J->n_obs = n_obs;
    J->k_lo = (uint32_t)((uint64_t)n_lambda * t / n_threads);
    J->k_hi = (uint32_t)((uint64_t)n_lambda * (t + 1) / n_threads);
    J->n_sets = n_sets;
    J->alpha = alpha;
    seed_to_key(seed, J->key);
    J->gamma = gamma;
    J->counts = counts;
  }
  for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, wi_worker, &jobs[t]);
  wi_worker(&jobs[0]);
  int rc = jobs[0].rc;
  for (int t = 1; t < n_threads; ++t) {
    pthread_join(th[t], NULL);
    if (jobs[t].rc) rc = jobs[t].rc;
  }
  free(jobs);
  free(th);
  return rc;
}

/* ---------------------------------------------------------------------------
 * Genetic toggle switch prior predictive (Sec. 3.2, Eq. 3-4; Euler-Maruyama
 * with Delta t = 1 as in Sec. 3.3, Eq. 5; the per-cell update and the noisy
 * observation as the paper's C implementation orders them, Sec. 3.4).
 * For each cell: u = v = 10; for j = 1..T-1
 *     p_u = v^beta_u, p_v = u^beta_v            (previous values)
 *     u = 0.97 u + alpha_u / (1 + p_u) - 1 + 0.5 zeta_u
 *     v = 0.97 v + alpha_v / (1 + p_v) - 1 + 0.5 zeta_v
 *     u = max(u, 1), v = max(v, 1)
 * then y = max(u + mu + mu sigma eta / u^gamma, 1).  The summaries are the
 * 19 equally spaced quantiles of the C values (Vo et al.'s choice, cited in
 * Sec. 3.2); rho is the Euclidean distance to the observed quantiles.
 * ------------------------------------------------------------------------- */
static int cmp_double_asc(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x > y) - (x < y);
}

/* Quantile at level k/20 of sorted x[0..C-1]: h = (C-1) k / 20, linear
 * interpolation between x[floor(h)] and the next order statistic. */
static double quantile_k20(const double *x, uint32_t C, uint32_t k) {
  uint64_t num = (uint64_t)(C - 1) * k;
  uint64_t lo = num / 20;
  double frac = (double)(num % 20) / 20.0;
  if (lo + 1 >= C) return x[C - 1];
  return x[lo] + frac * (x[lo + 1] - x[lo]);
}

static void toggle_one_sample(const orc_toggle_model *m, const double *q_obs,
                              const uint32_t key[2], uint64_t g, uint32_t sub, double *theta,
                              double *summ, double *ycell, double *uv, double *dist, double *ybuf) {
  uint32_t w0[4], w1[4];
  uint32_t c0[4] = {ORC_TAG_TOGGLE_PRIOR, 0u, sub, (uint32_t)g};
  uint32_t c1[4] = {ORC_TAG_TOGGLE_PRIOR, 1u, sub, (uint32_t)g};
  orc_philox4x32_10(c0, key, w0);
  orc_philox4x32_10(c1, key, w1);
  const uint32_t words[7] = {w0[0], w0[1], w0[2], w0[3], w1[0], w1[1], w1[2]};
  double th[7];
  for (int j = 0; j < 7; ++j) th[j] = m->lo[j] + (m->hi[j] - m->lo[j]) * orc_u01(words[j]);
  if (theta)
    for (int j = 0; j < 7; ++j) theta[j] = th[j];
  const double mu = th[0], sigma = th[1], gam = th[2];
  const double alpha_u = th[3], alpha_v = th[4], beta_u = th[5], beta_v = th[6];
  const uint32_t T = m->T, C = m->C;
  const uint32_t tag = (sub << 8) | ORC_TAG_TOGGLE_PATH;
  for (uint32_t c = 0; c < C; ++c) {
    double u = 10.0, v = 10.0;
    double z[4];
    uint32_t zi = 0; /* index of the next normal of this cell's stream */
    for (uint32_t j = 1; j < T; ++j) {
      double p_u = pow(v, beta_u);
      double p_v = pow(u, beta_v);
      double zu, zv;
      if (zi % 4 == 0) block_normals(key, zi / 4, c, (uint32_t)g, tag, z);
      zu = z[zi % 4];
      ++zi;
      if (zi % 4 == 0) block_normals(key, zi / 4, c, (uint32_t)g, tag, z);
      zv = z[zi % 4];
      ++zi;
      u = 0.97 * u + alpha_u / (1.0 + p_u) - 1.0 + 0.5 * zu;
      v = 0.97 * v + alpha_v / (1.0 + p_v) - 1.0 + 0.5 * zv;
      if (u < 1.0) u = 1.0;
      if (v < 1.0) v = 1.0;
    }
    if (uv) {
      uv[2 * c] = u;
      uv[2 * c + 1] = v;
    }
    if (zi % 4 == 0) block_normals(key, zi / 4, c, (uint32_t)g, tag, z);
    double eta = z[zi % 4];
    double yv = u + mu + mu * sigma * eta / pow(u, gam);
    if (yv < 1.0) yv = 1.0;
    ybuf[c] = yv;
    if (ycell) ycell[c] = yv;
  }
  qsort(ybuf, C, sizeof(double), cmp_double_asc);
  double acc = 0.0;
  for (uint32_t k = 1; k <= ORC_TOGGLE_NQ; ++k) {
    double q = quantile_k20(ybuf, C, k);
    if (summ) summ[k - 1] = q;
    double r = q - q_obs[k - 1];
    acc += r * r;
  }
  *dist = sqrt(acc);
}

typedef struct tg_job {
  const orc_toggle_model *m;
  const double *q_obs;
  uint32_t key[2];
  uint64_t base, lo, hi;
  uint32_t sub;
  double *theta, *summ, *y, *uv, *dist;
  int rc;
} tg_job;

static void *tg_worker(void *arg) {
  tg_job *J = (tg_job *)arg;
  double *ybuf = (double *)malloc((size_t)J->m->C * sizeof(double));
  if (!ybuf) {
    J->rc = -1;
    return NULL;
  }
  for (uint64_t t = J->lo; t < J->hi; ++t)
    toggle_one_sample(J->m, J->q_obs, J->key, J->base + t, J->sub,
                      J->theta ? J->theta + 7 * t : NULL,
                      J->summ ? J->summ + ORC_TOGGLE_NQ * t : NULL,
                      J->y ? J->y + (uint64_t)J->m->C * t : NULL,
                      J->uv ? J->uv + 2 * (uint64_t)J->m->C * t : NULL, J->dist + t, ybuf);
  free(ybuf);
  return NULL;
}

int orc_toggle_prior_predictive(const orc_toggle_model *m, const double *q_obs, uint64_t base,
                                uint64_t n, uint64_t seed, uint32_t sub, double *theta,
                                double *summ, double *y, double *uv, double *dist, int n_threads) {
  if (!m || !q_obs || !dist || m->T < 2 || m->C < 1) return -1;
  if (sub > 0xFFFFFFu || base + n > 0x100000000ull) return -1;
  if (n_threads < 1) n_threads = 1;
  if ((uint64_t)n_threads > n) n_threads = (int)(n > 0 ? n : 1);
  tg_job *jobs = (tg_job *)calloc((size_t)n_threads, sizeof(tg_job));
  pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  if (!jobs || !th) {
    free(jobs);
    free(th);
    return -1;
  }
  for (int t = 0; t < n_threads; ++t) {
    tg_job *J = &jobs[t];
    J->m = m;
    J->q_obs = q_obs;
    seed_to_key(seed, J->key);
    J->base = base;
    J->lo = n * (uint64_t)t / (uint64_t)n_threads;
    J->hi = n * (uint64_t)(t + 1) / (uint64_t)n_threads;
    J->sub = sub;
    J->theta = theta;
    J->summ = summ;
    J->y = y;
    J->uv = uv;
    J->dist = dist;
  }
  for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, tg_worker, &jobs[t]);
  tg_worker(&jobs[0]);
  int rc = jobs[0].rc;
  for (int t = 1; t < n_threads; ++t) {
    pthread_join(th[t], NULL);
    if (jobs[t].rc) rc = jobs[t].rc;
  }
  free(jobs);
  free(th);
  return rc;
}

/* ---------------------------------------------------------------------------
 * ABC recalibration (Discussion, Sec. 5): every accepted theta* is recalibrated
 * with a further ABC posterior built from all stored (theta, D) pairs, taking
 * its own simulated data D* as the observation, through the univariate
 * marginal posterior distribution functions: u = F(theta* | D*) from the k
 * nearest pairs, and the recalibrated value is the u-quantile of the
 * accepted sample's marginal (the posterior given the real observation).
 * ------------------------------------------------------------------------- */
static int cmp_float_asc(const void *a, const void *b) {
  float x = *(const float *)a, y = *(const float *)b;
  return (x > y) - (x < y);
}

typedef struct rc_job {
  const double *summ;
  const float *theta;
  uint64_t n, q, k, lo, hi;
  uint32_t n_obs;
  const uint32_t *acc;
  double *u;
  int rc;
} rc_job;

static void *rc_worker(void *arg) {
  rc_job *J = (rc_job *)arg;
  dist_idx *a = (dist_idx *)malloc((size_t)J->n * sizeof(dist_idx));
  if (!a) {
    J->rc = -1;
    return NULL;
  }
  for (uint64_t i = J->lo; i < J->hi; ++i) {
    uint64_t qa = J->acc[i];
    for (uint64_t j = 0; j < J->n; ++j) {
      double acc = 0.0;
      for (uint32_t m = 0; m < J->n_obs; ++m) {
        double r = J->summ[(uint64_t)m * J->n + j] - J->summ[(uint64_t)m * J->n + qa];
        acc = fma(r, r, acc);
      }
      a[j].d = sqrt(acc);
      a[j].i = j;
    }
    qsort(a, (size_t)J->n, sizeof(dist_idx), cmp_dist_idx);
    for (int d = 0; d < 3; ++d) {
      float t0 = J->theta[(uint64_t)d * J->n + qa];
      uint64_t c = 0;
      for (uint64_t t = 0; t < J->k; ++t)
        if (J->theta[(uint64_t)d * J->n + a[t].i] <= t0) ++c;
      J->u[(uint64_t)d * J->q + i] = (double)c / (double)J->k;
    }
  }
  free(a);
  return NULL;
}

int orc_recalibrate(const double *summ, const float *theta, uint64_t n, uint32_t n_obs,
                    const uint32_t *acc, uint64_t q, uint64_t k, double *u, float *theta_rc,
                    int n_threads) {
  if (!summ || !theta || !acc || !u || !theta_rc || n == 0 || q == 0 || k == 0 || k > n) return -1;
  for (uint64_t i = 0; i < q; ++i)
    if (acc[i] >= n) return -1;
  if (n_threads < 1) n_threads = 1;
  if ((uint64_t)n_threads > q) n_threads = (int)q;
  rc_job *jobs = (rc_job *)calloc((size_t)n_threads, sizeof(rc_job));
  pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  float *sorted = (float *)malloc((size_t)q * sizeof(float));
  if (!jobs || !th || !sorted) {
    free(jobs);
    free(th);
    free(sorted);
    return -1;
  }
  for (int t = 0; t < n_threads; ++t) {
    rc_job *J = &jobs[t];
    J->summ = summ;
    J->theta = theta;
    J->n = n;
    J->q = q;
    J->k = k;
    J->n_obs = n_obs;
    J->acc = acc;
    J->u = u;
    J->lo = q * (uint64_t)t / (uint64_t)n_threads;
    J->hi = q * (uint64_t)(t + 1) / (uint64_t)n_threads;
  }
  for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, rc_worker, &jobs[t]);
  rc_worker(&jobs[0]);
  int rc = jobs[0].rc;
  for (int t = 1; t < n_threads; ++t) {
    pthread_join(th[t], NULL);
    if (jobs[t].rc) rc = jobs[t].rc;
  }
  for (int d = 0; d < 3 && rc == 0; ++d) {
    for (uint64_t i = 0; i < q; ++i) sorted[i] = theta[(uint64_t)d * n + acc[i]];
    qsort(sorted, (size_t)q, sizeof(float), cmp_float_asc);
    for (uint64_t i = 0; i < q; ++i) {
      /* u = c / k; the rank ceil(u q) = ceil(c q / k) is formed from the count
       * in integers (the binary64 product u q can round above an integer). */
      const uint64_t c = (uint64_t)llround(u[(uint64_t)d * q + i] * (double)k);
      uint64_t r = (c * q + k - 1) / k;
      if (r < 1) r = 1;
      if (r > q) r = q;
      theta_rc[(uint64_t)d * q + i] = sorted[r - 1];
    }
  }
  free(jobs);
  free(th);
  free(sorted);
  return rc;
}

/* ---------------------------------------------------------------------------
 * BEGE log-likelihood (Sec. 4.2: the BEGE model, its shape recursion, the
 * log-likelihood Eq. BEGE_LL, the distribution function Eq. CDF_BEGE
 * discretised as Eq. BEGE_LL_approx, and P(a, x) of Eq. incompGamma).
 * ------------------------------------------------------------------------- */

/* Regularised lower incomplete gamma P(a, x) = gamma(a, x) / Gamma(a), a > 0.
 * x < a + 1: the power series the paper names (Press et al. 1992),
 *   P = exp(-x + a ln x - lnGamma(a)) sum_{j>=0} x^j / (a (a+1) ... (a+j)),
 * summed term by term until a term is below ORC_GAMMA_EPS of the sum.
 * x >= a + 1: the same reference's continued fraction for Q = 1 - P,
 *   Q = exp(-x + a ln x - lnGamma(a)) / (x+1-a- 1(1-a)/(x+3-a- 2(2-a)/(x+5-a- ...))),
 * evaluated from the top by the modified Lentz method; there the series would
 * need O(x) terms and its partial sums overflow binary64 beyond x ~ 700.
 * Both loops stop after ORC_GAMMA_MAX_ITER terms. */
#define ORC_GAMMA_EPS 1e-17
#define ORC_GAMMA_TINY 1e-300
#define ORC_GAMMA_MAX_ITER 1000000

double orc_gammainc_p(double a, double x) {
  if (!(a > 0.0) || x != x) return NAN;
  if (x <= 0.0) return 0.0;
  const double lead = -x + a * log(x) - lgamma(a);
  if (x < a + 1.0) {
    double ap = a, term = 1.0 / a, sum = term;
    for (int k = 1; k < ORC_GAMMA_MAX_ITER; ++k) {
      ap += 1.0;
      term *= x / ap;
      sum += term;
      if (fabs(term) < fabs(sum) * ORC_GAMMA_EPS || term == 0.0) break;
    }
    return sum * exp(lead);
  }
  double b = x + 1.0 - a;
  double c = 1.0 / ORC_GAMMA_TINY;
  double d = 1.0 / b;
  double h = d;
  for (int i = 1; i < ORC_GAMMA_MAX_ITER; ++i) {
    const double an = -i * (i - a);
    b += 2.0;
    d = an * d + b;
    if (fabs(d) < ORC_GAMMA_TINY) d = ORC_GAMMA_TINY;
    c = b + an / c;
    if (fabs(c) < ORC_GAMMA_TINY) c = ORC_GAMMA_TINY;
    d = 1.0 / d;
    const double del = d * c;
    h *= del;
    if (fabs(del - 1.0) < ORC_GAMMA_EPS) break;
  }
  return 1.0 - exp(lead) * h;
}

/* The BEGE distribution function at u, Eq. BEGE_LL_approx: with shapes p, n
 * and scales sp, sn of the centred-gamma shocks, N_w = ORC_BEGE_NW intervals,
 *   w_j = w_0 + j dw, w_0 = 1e-4 - p sp, dw = (10 sp sqrt(p) - w_0) / (N_w - 1),
 *   F(u) ~ sum_{j=1..N_w} [1 - P(n, (w_{j-1} - u + n sn) / sn)]
 *                         [P(p, (w_j + p sp) / sp) - P(p, (w_{j-1} + p sp) / sp)],
 * with P(a, x) = 0 for x <= 0 (below the shock's support). */
double orc_bege_cdf(double u, double sp, double sn, double p, double n) {
  const int Nw = ORC_BEGE_NW;
  const double w0 = 1e-4 - p * sp;
  const double dw = (10.0 * sp * sqrt(p) - w0) / (double)(Nw - 1);
  double Fprev = orc_gammainc_p(p, (w0 + p * sp) / sp);
  double acc = 0.0;
  for (int j = 1; j <= Nw; ++j) {
    const double wj = w0 + (double)j * dw;
    const double wjm1 = w0 + (double)(j - 1) * dw;
    const double Fj = orc_gammainc_p(p, (wj + p * sp) / sp);
    const double xn = (wjm1 - u + n * sn) / sn;
    const double Gn = xn > 0.0 ? orc_gammainc_p(n, xn) : 0.0;
    acc += (1.0 - Gn) * (Fj - Fprev);
    Fprev = Fj;
  }
  return acc;
}

/* The BEGE density by central finite differences of the distribution
 * function (Sec. 4.2: density from the distribution function by finite
 * differences), step h. */
double orc_bege_density(double u, double sp, double sn, double p, double n, double h) {
  return (orc_bege_cdf(u + h, sp, sn, p, n) - orc_bege_cdf(u - h, sp, sn, p, n)) / (2.0 * h);
}

/* Log-likelihood of one parameter vector th = (p0, sp, rho_p, phi_p+, phi_p-,
 * n0, sn, rho_n, phi_n+, phi_n-, mu) on returns r_1..r_T (Eq. BEGE_LL):
 *   u_t = r_t - mu,  ll = sum_t log f(u_t; sp, sn, p_{t-1}, n_{t-1}),
 * shapes from (p_0, n_0) = (p0, n0) by the printed recursion
 *   p_t = p0 + rho_p p_{t-1} + phi_p^{+|-} / (2 sp^2) u_t^2   (+ if u_t >= 0),
 * and n_t likewise with sn and the n parameters.  A scale <= 0, a shape that
 * is not a positive finite number, or a density that is not a positive finite
 * number, gives -inf. */
static double bege_ll_one(const double th[ORC_BEGE_NPAR], const double *r, uint32_t T, double h,
                          double *dens) {
  const double p0 = th[0], sp = th[1], rp = th[2], fpp = th[3], fpm = th[4];
  const double n0 = th[5], sn = th[6], rn = th[7], fnp = th[8], fnm = th[9], mu = th[10];
  if (!(sp > 0.0) || !(sn > 0.0)) return -INFINITY;
  double p = p0, n = n0, ll = 0.0;
  for (uint32_t t = 0; t < T; ++t) {
    if (!(p > 0.0) || !(n > 0.0) || !isfinite(p) || !isfinite(n)) return -INFINITY;
    const double u = r[t] - mu;
    const double f = orc_bege_density(u, sp, sn, p, n, h);
    if (dens) dens[t] = f;
    if (!(f > 0.0) || !isfinite(f)) return -INFINITY;
    ll += log(f);
    const double cp = (u >= 0.0 ? fpp : fpm) / (2.0 * sp * sp);
    const double cn = (u >= 0.0 ? fnp : fnm) / (2.0 * sn * sn);
    p = p0 + rp * p + cp * u * u;
    n = n0 + rn * n + cn * u * u;
  }
  return ll;
}

typedef struct bege_job {
  const double *theta, *r;
  uint64_t np, lo, hi;
  uint32_t T;
  double h;
  double *ll, *dens;
} bege_job;

static void *bege_worker(void *arg) {
  bege_job *J = (bege_job *)arg;
  for (uint64_t i = J->lo; i < J->hi; ++i) {
    double th[ORC_BEGE_NPAR];
    for (int k = 0; k < ORC_BEGE_NPAR; ++k) th[k] = J->theta[(uint64_t)k * J->np + i];
    J->ll[i] = bege_ll_one(th, J->r, J->T, J->h, J->dens ? J->dens + i * (uint64_t)J->T : NULL);
  }
  return NULL;
}

int orc_bege_loglik(const double *theta, uint64_t np, const double *r, uint32_t T, double h,
                    double *ll, double *dens, int n_threads) {
  if (!theta || !r || !ll || np == 0 || T == 0 || !(h > 0.0)) return -1;
  if (dens)
    for (uint64_t i = 0; i < np * (uint64_t)T; ++i) dens[i] = NAN;
  if (n_threads < 1) n_threads = 1;
  if ((uint64_t)n_threads > np) n_threads = (int)np;
  bege_job *jobs = (bege_job *)calloc((size_t)n_threads, sizeof(bege_job));
  pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  if (!jobs || !th) {
    free(jobs);
    free(th);
    return -1;
  }
  for (int t = 0; t < n_threads; ++t) {
    bege_job *J = &jobs[t];
    J->theta = theta;
    J->r = r;
    J->np = np;
    J->T = T;
    J->h = h;
    J->ll = ll;
    J->dens = dens;
    J->lo = np * (uint64_t)t / (uint64_t)n_threads;
    J->hi = np * (uint64_t)(t + 1) / (uint64_t)n_threads;
  }
  for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, bege_worker, &jobs[t]);
  bege_worker(&jobs[0]);
  for (int t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
  free(jobs);
  free(th);
  return 0;
}
