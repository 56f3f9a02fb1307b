"""Seeded synthetic inputs for the prior-predictive workloads.

This module only draws *inputs*: model constants, observed data and job
mixes.  It holds none of the method's arithmetic (no Philox stream, no
Euler-Maruyama step, no distance, no selection), so the CUDA path and the CPU
oracle can both be fed from it without sharing any of the computation they
are compared on.  All randomness here comes from numpy's PCG64 generator with
a fixed seed.

Observed data are drawn from the *exact* Ornstein-Uhlenbeck transition
X(t+h) = th2 + (X(t) - th2) e^{-th1 h} + th3 sqrt((1 - e^{-2 th1 h}) / (2 th1)) Z,
i.e. from the process the Euler-Maruyama sampler approximates, not from the
sampler itself.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Uniform prior box of the OU workloads: th1 (mean reversion rate), th2 (long-run
# mean), th3 (diffusion scale).
OU_PRIOR_LO = (0.1, -2.0, 0.1)
OU_PRIOR_HI = (2.0, 2.0, 1.0)
OU_T_END = 10.0
OU_N_OBS = 10
OU_THETA_TRUE = (1.0, 0.5, 0.3)


def ou_model(n_steps: int, t_end: float = OU_T_END, n_obs: int = OU_N_OBS,
             x0: float = 0.0, lo=OU_PRIOR_LO, hi=OU_PRIOR_HI) -> dict:
    """OU model record: dt = t_end / n_steps, observed at n_obs equal spacings."""
    return {"lo": tuple(lo), "hi": tuple(hi), "x0": float(x0),
            "dt": float(t_end) / int(n_steps), "n_steps": int(n_steps), "n_obs": int(n_obs)}


def ou_observed(theta, seed: int, t_end: float = OU_T_END, n_obs: int = OU_N_OBS,
                x0: float = 0.0) -> np.ndarray:
    """Observed OU data at t_j = j t_end / n_obs, j = 1..n_obs, from the exact
    transition density (float64), drawn with numpy's PCG64(seed)."""
    th1, th2, th3 = (float(v) for v in theta)
    rng = np.random.default_rng(seed)
    h = t_end / n_obs
    decay = np.exp(-th1 * h)
    sd = th3 * np.sqrt((1.0 - np.exp(-2.0 * th1 * h)) / (2.0 * th1))
    x = float(x0)
    y = np.empty(n_obs, dtype=np.float64)
    for j in range(n_obs):
        x = th2 + (x - th2) * decay + sd * rng.standard_normal()
        y[j] = x
    return y


# --------------------------------------------------------------------------
# Workload configurations (sizes of the OU-ABC and p-value workloads).
# --------------------------------------------------------------------------

@dataclass
class ABCWorkload:
    name: str
    model: dict
    y_obs: np.ndarray
    n_samples: int
    k_accept: int
    seed: int
    substream: int = 0


def abc_small() -> ABCWorkload:
    """OU-ABC, N = 1e4 prior samples, 1000 EM steps (dt = 0.01), accept the 100
    nearest; observed data from theta* = (1, 0.5, 0.3), seed 1."""
    return ABCWorkload("ou_abc_n1e4_s1e3", ou_model(1000), ou_observed(OU_THETA_TRUE, 1),
                       10_000, 100, seed=1)


def abc_large(n_samples: int = 1 << 24) -> ABCWorkload:
    """OU-ABC precision study: N = 2^24, 10^4 EM steps (dt = 0.001), accept 0.1%."""
    return ABCWorkload("ou_abc_n2p24_s1e4", ou_model(10_000), ou_observed(OU_THETA_TRUE, 1),
                       n_samples, int(0.001 * n_samples), seed=1)


@dataclass
class PValueWorkload:
    name: str
    lambdas: np.ndarray
    n_obs: int
    m_sets: int
    ybar_obs: float
    seed: int


def pvalue_lambdas(n_lambda: int = 64, lo: float = 0.01, hi: float = 100.0) -> np.ndarray:
    return np.logspace(np.log10(lo), np.log10(hi), n_lambda)


def pvalue_observed_ybar(seed: int = 2, mu_true: float = 3.0, n_obs: int = 50) -> float:
    """ybar of n_obs draws y_i ~ N(mu_true, 1), PCG64(seed)."""
    rng = np.random.default_rng(seed)
    return float(mu_true + rng.standard_normal(n_obs).mean())


def pvalue_sweep_workload(m_sets: int = 1_000_000) -> PValueWorkload:
    """64 lambdas log-spaced in [0.01, 100], n = 50, M data sets per lambda."""
    return PValueWorkload("pvalue_k64_n50_m1e6", pvalue_lambdas(), 50, m_sets,
                          pvalue_observed_ybar(), seed=2)


# --------------------------------------------------------------------------
# Job mixes for batched and served execution.
# --------------------------------------------------------------------------

@dataclass
class Job:
    job_id: int
    kind: str                 # "abc" or "pvalue"
    seed: int
    n: int                    # ABC: prior samples; p-value: data sets M
    n_steps: int = 0          # ABC only
    k_accept: int = 0         # ABC only
    y_obs: np.ndarray | None = None
    theta_star: tuple | None = None
    lam: float = 0.0          # p-value only
    n_obs: int = 50           # p-value only
    ybar_obs: float = 0.0     # p-value only
    arrival_s: float = 0.0
    model: dict = field(default_factory=dict)

    @property
    def path_steps(self) -> int:
        """EM steps (ABC) or normals drawn (p-value: n_obs + 1 per data set)."""
        return self.n * (self.n_steps if self.kind == "abc" else self.n_obs + 1)


def _log_uniform_int(rng, lo: float, hi: float) -> int:
    return int(round(float(np.exp(rng.uniform(np.log(lo), np.log(hi))))))


def _abc_job(rng, job_id: int, n_lo: float, n_hi: float, s_lo: int, s_hi: int,
             accept_frac: float) -> Job:
    n = _log_uniform_int(rng, n_lo, n_hi)
    steps = int(rng.integers(s_lo, s_hi + 1))
    jr = np.random.default_rng(job_id)        # per-job observed data: seed = job id
    theta_star = tuple(float(jr.uniform(l, h)) for l, h in zip(OU_PRIOR_LO, OU_PRIOR_HI))
    y = ou_observed(theta_star, seed=job_id + 1_000_003)
    return Job(job_id=job_id, kind="abc", seed=job_id, n=n, n_steps=steps,
               k_accept=max(1, int(accept_frac * n)), y_obs=y, theta_star=theta_star,
               model=ou_model(steps))


def batched_jobs(n_jobs: int = 256, n_lo: float = 1e3, n_hi: float = 1e7,
                 s_lo: int = 100, s_hi: int = 10_000, accept_frac: float = 0.01,
                 gen_seed: int = 3) -> list[Job]:
    """Uneven OU-ABC jobs: N log-uniform in [n_lo, n_hi], EM steps uniform in
    {s_lo..s_hi}, dt = 10 / steps, theta* from the prior, 1% accepted."""
    rng = np.random.default_rng(gen_seed)
    return [_abc_job(rng, j, n_lo, n_hi, s_lo, s_hi, accept_frac) for j in range(n_jobs)]


def served_jobs(rate_per_s: float = 200.0, duration_s: float = 60.0, abc_frac: float = 0.7,
                gen_seed: int = 4, abc_n=(1e3, 1e6), abc_steps=(100, 2000),
                pv_m=(1e4, 1e6), pv_lambda=(0.01, 100.0), n_obs: int = 50) -> list[Job]:
    """Poisson arrivals (exponential gaps at rate_per_s) of mixed ABC and
    p-value jobs over duration_s seconds."""
    rng = np.random.default_rng(gen_seed)
    jobs: list[Job] = []
    t = 0.0
    jid = 0
    while True:
        t += float(rng.exponential(1.0 / rate_per_s))
        if t >= duration_s:
            break
        if rng.uniform() < abc_frac:
            job = _abc_job(rng, jid, abc_n[0], abc_n[1], abc_steps[0], abc_steps[1], 0.01)
        else:
            m = _log_uniform_int(rng, pv_m[0], pv_m[1])
            lam = float(np.exp(rng.uniform(np.log(pv_lambda[0]), np.log(pv_lambda[1]))))
            job = Job(job_id=jid, kind="pvalue", seed=jid, n=m, lam=lam, n_obs=n_obs,
                      ybar_obs=pvalue_observed_ybar(seed=jid + 2_000_003, n_obs=n_obs))
        job.arrival_s = t
        jobs.append(job)
        jid += 1
    return jobs


# --------------------------------------------------------------------------
# Genetic toggle switch (the paper's example model).
# --------------------------------------------------------------------------

TOGGLE_PRIOR_LO = (250.0, 0.05, 0.05, 0.0, 0.0, 0.0, 0.0)
TOGGLE_PRIOR_HI = (400.0, 0.5, 0.35, 50.0, 50.0, 7.0, 7.0)


def toggle_model(T: int = 600, C: int = 8000) -> dict:
    """Prior box of the paper's toggle-switch example; T time points, C cells."""
    return {"lo": TOGGLE_PRIOR_LO, "hi": TOGGLE_PRIOR_HI, "T": int(T), "C": int(C)}


def toggle_observed_quantiles(seed: int = 7) -> np.ndarray:
    """A synthetic target for the 19 summary quantiles: the quantiles at levels
    0.05..0.95 of a right-skewed intensity distribution (shifted lognormal,
    PCG64-drawn location and scale), standing in for observed cell data."""
    rng = np.random.default_rng(seed)
    loc = float(rng.uniform(300.0, 350.0))
    scale = float(rng.uniform(0.3, 0.6))
    from scipy import stats
    levels = np.arange(1, 20) / 20.0
    return loc + 100.0 * stats.lognorm.ppf(levels, s=scale)


# BEGE model (Sec. 4.2): parameter order and the paper's uniform prior box
# (p0, sigma_p, rho_p, phi_p+, phi_p-, n0, sigma_n, rho_n, phi_n+, phi_n-, mu).
BEGE_PARAMS = ("p0", "sigma_p", "rho_p", "phi_p_plus", "phi_p_minus",
               "n0", "sigma_n", "rho_n", "phi_n_plus", "phi_n_minus", "mu")
BEGE_PRIOR_LO = (1e-4, 1e-4, 1e-4, 1e-4, 1e-4, 1e-4, 1e-4, 1e-4, -0.2, 1e-4, -0.9)
BEGE_PRIOR_HI = (0.5, 0.3, 0.99, 0.5, 0.5, 1.0, 0.3, 0.99, 0.1, 0.75, 0.9)
BEGE_T = 1099          # months in the paper's return series
BEGE_N_PARTICLES = 1024
BEGE_H = 1e-5          # finite-difference step of the density


def bege_returns(T: int = BEGE_T, seed: int = 5) -> np.ndarray:
    """Synthetic monthly log returns standing in for the paper's S&P series
    (which is not available): mean 0.0075, a two-state volatility regime
    (0.04 calm, 0.09 turbulent, staying with probability 0.97) and Student-t
    (5 degrees of freedom) shocks with a negative skew from a mixture."""
    rng = np.random.default_rng(seed)
    r = np.empty(T)
    state = 0
    for t in range(T):
        if rng.uniform() > 0.97:
            state = 1 - state
        vol = 0.04 if state == 0 else 0.09
        z = rng.standard_t(5) / np.sqrt(5.0 / 3.0)
        if rng.uniform() < 0.05:
            z -= 1.5
        r[t] = 0.0075 + vol * z
    return r


def bege_particles(n: int = BEGE_N_PARTICLES, seed: int = 6, centre=None,
                   rel_spread: float = 0.0) -> np.ndarray:
    """[11, n] parameter vectors: uniform on the paper's prior box, or, with a
    centre, uniform within +-rel_spread of the box width around it (clipped to
    the box), like the particles of a later SMC iteration."""
    rng = np.random.default_rng(seed)
    lo, hi = np.array(BEGE_PRIOR_LO), np.array(BEGE_PRIOR_HI)
    if centre is None:
        return lo[:, None] + (hi - lo)[:, None] * rng.uniform(size=(11, n))
    c = np.asarray(centre, dtype=np.float64)
    half = rel_spread * (hi - lo)
    a, b = np.maximum(lo, c - half), np.minimum(hi, c + half)
    return a[:, None] + (b - a)[:, None] * rng.uniform(size=(11, n))


# A parameter vector in the plausible region for monthly returns (used as the
# centre of the later-iteration particle set).
BEGE_THETA_REF = (0.3, 0.03, 0.6, 0.2, 0.3, 0.5, 0.04, 0.6, 0.02, 0.4, 0.008)
