"""Seeded synthetic inputs for the FM-CFUST workloads.

This module is the only code that both the CUDA path and the CPU oracle see.
It holds no E-step or M-step arithmetic: it draws parameters, samples data
from the latent hierarchy of eq (6), builds starting values (k-means
partition, then the moment-based values of eq (23), Sec. 3.3) and states the
lattice settings that both sides receive as inputs.

Workloads (shapes of the paper's experiments; the HSCT flow-cytometry data
are not available, so draws of the same shape stand in for them):
  two_comp_p2   p=q=g=2, n=1000, the fixed two-component parameters below,
                100 EM iterations, q=2 so T_q is deterministic.
  flow_p4       p=q=g=4 (the HSCT shape: 4 markers, 4 populations),
                n=200,000, lattice 1024 points x 8 shifts, 50 iterations.
  wide_p16      p=16, q=2, g=8, n=2,000,000, y stored FP32, 20 iterations.
  learned_p6    p=q=g=6, n=1,000,000.
"""
from __future__ import annotations

import math

import numpy as np

# Korobov generator for N = 1024 lattice points, from oracle/korobov_search.py
# (minimises the P_2 figure of merit over dimensions 3..8).
DEFAULT_KOROBOV_A = 119
DEFAULT_QMC_POINTS = 1024
DEFAULT_QMC_SHIFTS = 8

SEED_BASE = 1606_0000


def seed_for(stream: int, start: int = 0) -> int:
    return SEED_BASE + 100 * stream + start


def qmc_settings(stream: int = 2, npoints=DEFAULT_QMC_POINTS, nshifts=DEFAULT_QMC_SHIFTS,
                 korobov_a=DEFAULT_KOROBOV_A):
    return dict(npoints=npoints, nshifts=nshifts, korobov_a=korobov_a,
                seed=seed_for(stream) * 7919 + 13)


# ----------------------------------------------------------------------------
# parameters
# ----------------------------------------------------------------------------
def two_comp_params():
    """Fixed two-component parameters (p = q = g = 2)."""
    return dict(
        pi=np.array([0.6, 0.4]),
        mu=np.array([[0.0, 0.0], [4.0, 4.0]]),
        Sigma=np.array([[[1.0, 0.0], [0.0, 1.0]], [[1.0, 0.5], [0.5, 1.0]]]),
        Delta=np.array([[[2.0, 0.0], [0.0, -1.0]], [[1.0, 0.5], [0.0, 1.5]]]),
        nu=np.array([4.0, 10.0]),
    )


def draw_params(rng, p, q, g, mu_range=5.0, wishart_df=8, delta_sd=1.5, nu_range=(3.0, 20.0),
                dirichlet=2.0):
    """mu ~ U[-r, r]^p, Sigma = Wishart(I, df)/df, Delta_ij ~ N(0, sd^2),
    nu ~ U[nu_range], pi ~ Dirichlet(dirichlet, ..., dirichlet)."""
    mu = rng.uniform(-mu_range, mu_range, size=(g, p))
    Sigma = np.empty((g, p, p))
    for h in range(g):
        X = rng.standard_normal((wishart_df, p))
        Sigma[h] = X.T @ X / wishart_df
    Delta = rng.normal(0.0, delta_sd, size=(g, p, q))
    nu = rng.uniform(nu_range[0], nu_range[1], size=g)
    pi = rng.dirichlet(np.full(g, dirichlet))
    return dict(pi=pi, mu=mu, Sigma=Sigma, Delta=Delta, nu=nu)


# ----------------------------------------------------------------------------
# eq (6): Y = mu + Delta |U0| + U1, W ~ gamma(nu/2, nu/2), U0 ~ N(0, I/W),
# U1 ~ N(0, Sigma/W), component label ~ Mult(1, pi)
# ----------------------------------------------------------------------------
def sample(rng, n, params, dtype=np.float64):
    pi, mu, Sigma, Delta, nu = (np.asarray(params[k]) for k in ("pi", "mu", "Sigma", "Delta", "nu"))
    g, p = mu.shape
    q = Delta.shape[-1]
    z = rng.choice(g, size=n, p=pi / pi.sum())
    y = np.empty((n, p))
    for h in range(g):
        idx = np.nonzero(z == h)[0]
        m = idx.size
        if m == 0:
            continue
        w = rng.gamma(shape=nu[h] / 2.0, scale=2.0 / nu[h], size=m)
        u0 = np.abs(rng.standard_normal((m, q))) / np.sqrt(w)[:, None]
        Lc = np.linalg.cholesky(Sigma[h])
        u1 = (rng.standard_normal((m, p)) @ Lc.T) / np.sqrt(w)[:, None]
        y[idx] = mu[h] + u0 @ Delta[h].T + u1
    return y.astype(dtype), z


# ----------------------------------------------------------------------------
# starting values: k-means++ partition, 100 Lloyd steps, then eq (23)
# ----------------------------------------------------------------------------
def _nearest(y, C):
    d = (y * y).sum(1)[:, None] - 2.0 * y @ C.T + (C * C).sum(1)[None, :]
    return d.argmin(1)


def kmeans(rng, y, g, iters=100, max_fit=50_000):
    """k-means++ seeding and Lloyd steps; beyond max_fit observations the
    centres are fitted on a random subsample and every point is then assigned
    to its nearest centre."""
    n = y.shape[0]
    ys = y[rng.choice(n, max_fit, replace=False)] if n > max_fit else y
    m = ys.shape[0]
    centers = [ys[rng.integers(m)]]
    d2 = np.sum((ys - centers[0]) ** 2, axis=1)
    for _ in range(1, g):
        probs = d2 / d2.sum()
        c = ys[rng.choice(m, p=probs)]
        centers.append(c)
        d2 = np.minimum(d2, np.sum((ys - c) ** 2, axis=1))
    C = np.array(centers)
    for _ in range(iters):
        lab = _nearest(ys, C)
        for h in range(g):
            if np.any(lab == h):
                C[h] = ys[lab == h].mean(0)
    return _nearest(y, C)


def moment_start(yc, q, alpha=0.5, nu0=10.0):
    """Eq (23) for one cluster: delta = sign(m3) sqrt(pi (1-alpha) s*/(pi-2)),
    Sigma = S - (1-alpha) diag(s*), mu = ybar - sqrt(2/pi) delta.  Delta is
    diag(delta) when q = p and the single column delta when q = 1; other q
    place delta on the leading diagonal of the p x q matrix."""
    p = yc.shape[1]
    ybar = yc.mean(0)
    S = np.cov(yc, rowvar=False).reshape(p, p)
    s = np.diag(S).copy()
    m3 = ((yc - ybar) ** 3).mean(0)
    sign = np.where(m3 >= 0, 1.0, -1.0)
    # skewed coordinates: all p when q = 1 (one column) or q >= p, else the first q
    skewed = np.ones(p) if (q == 1 or q >= p) else (np.arange(p) < q).astype(float)
    delta = skewed * sign * np.sqrt(math.pi * (1.0 - alpha) * s / (math.pi - 2.0))
    Sig = S - (1.0 - alpha) * np.diag(s * skewed)
    mu = ybar - math.sqrt(2.0 / math.pi) * delta
    D = np.zeros((p, q))
    if q == 1:
        D[:, 0] = delta
    else:
        for i in range(min(p, q)):
            D[i, i] = delta[i]
    return mu, Sig, D, nu0


def init_params(rng, y, g, q, alpha=0.5, nu0=10.0):
    """Starting values for EM: k-means partition, then eq (23) per cluster
    with alpha raised in 0.1 steps (to 0.9) while Sigma is not positive
    definite."""
    return params_from_labels(y, kmeans(rng, y, g), g, q, alpha, nu0)


def random_partition_start(rng, y, g, q, alpha=0.5, nu0=10.0):
    """Starting values from a uniformly random partition into g parts, then
    eq (23) per part (the random-start variant of Algorithm 1)."""
    return params_from_labels(y, rng.integers(0, g, size=y.shape[0]), g, q, alpha, nu0)


def params_from_labels(y, lab, g, q, alpha=0.5, nu0=10.0):
    """Eq (23) per labelled cluster (clusters with fewer than p + 2 points use
    all of y)."""
    n, p = y.shape
    pi = np.zeros(g)
    mu = np.zeros((g, p))
    Sigma = np.zeros((g, p, p))
    Delta = np.zeros((g, p, q))
    nu = np.zeros(g)
    for h in range(g):
        yc = y[lab == h]
        if yc.shape[0] < p + 2:
            yc = y
        pi[h] = max(yc.shape[0], 1) / n
        a = alpha
        while True:
            m, S, D, v = moment_start(yc, q, a, nu0)
            try:
                np.linalg.cholesky(S)
                break
            except np.linalg.LinAlgError:
                if a >= 0.9 - 1e-12:
                    S = np.cov(yc, rowvar=False) + 1e-3 * np.eye(p)
                    D = 0.1 * D
                    break
                a = min(0.9, a + 0.1)
        mu[h], Sigma[h], Delta[h], nu[h] = m, S, D, v
    pi = pi / pi.sum()
    return dict(pi=pi, mu=mu, Sigma=Sigma, Delta=Delta, nu=nu)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------
WORKLOADS = {
    "two_comp_p2": dict(stream=1, p=2, q=2, g=2, n=1000, iters=100),
    "flow_p4": dict(stream=2, p=4, q=4, g=4, n=200_000, iters=50),
    "wide_p16": dict(stream=3, p=16, q=2, g=8, n=2_000_000, iters=20),
    "learned_p6": dict(stream=5, p=6, q=6, g=6, n=1_000_000, iters=30),
}


# Batched fits: nfits independent problems, p uniform on {2..8}, q = p, g
# uniform on {2..6}, n log-uniform on [1e3, 1e5], parameters drawn as for
# flow_p4, `starts` random-partition starts per problem, 30 iterations.
BATCH = dict(stream=4, nfits=256, starts=4, p=(2, 8), g=(2, 6), n=(1_000, 100_000), iters=30)


def make_batch(nfits=None, starts=None, n_range=None, p_range=None, g_range=None):
    """Return dict(fits=[dict(y, truth, starts=[params...], p, q, g, n)], qmc, iters).
    The first k problems are the same for every nfits >= k."""
    B = BATCH
    nfits = B["nfits"] if nfits is None else int(nfits)
    starts = B["starts"] if starts is None else int(starts)
    n_lo, n_hi = B["n"] if n_range is None else n_range
    p_lo, p_hi = B["p"] if p_range is None else p_range
    g_lo, g_hi = B["g"] if g_range is None else g_range
    fits = []
    for f in range(nfits):
        rng = np.random.default_rng([seed_for(B["stream"]), f])
        p = int(rng.integers(p_lo, p_hi + 1))
        g = int(rng.integers(g_lo, g_hi + 1))
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        truth = draw_params(rng, p, p, g)
        y, z = sample(rng, n, truth)
        st = [random_partition_start(np.random.default_rng([seed_for(B["stream"], s + 1), f]), y, g, p)
              for s in range(starts)]
        fits.append(dict(y=y, z=z, truth=truth, starts=st, p=p, q=p, g=g, n=n))
    return dict(fits=fits, qmc=qmc_settings(B["stream"]), iters=B["iters"])


def make_workload(name, n=None, start=0, with_init=True):
    """Return dict(y, truth, init, qmc, p, q, g, n) for a named workload.
    n overrides the size (the first n observations of the same draw are not
    reused; the whole draw is repeated at the new size with the same seed)."""
    w = WORKLOADS[name]
    cfg = w["stream"]
    rng = np.random.default_rng(seed_for(cfg, start))
    p, q, g = w["p"], w["q"], w["g"]
    nn = int(n if n is not None else w["n"])
    if name == "two_comp_p2":
        truth = two_comp_params()
    elif name == "wide_p16":
        truth = draw_params(rng, p, q, g, mu_range=3.0, wishart_df=32)
    else:
        truth = draw_params(rng, p, q, g)
    y, z = sample(rng, nn, truth)
    out = dict(y=y, z=z, truth=truth, qmc=qmc_settings(cfg), p=p, q=q, g=g, n=nn,
               iters=w["iters"])
    if with_init:
        out["init"] = init_params(np.random.default_rng(seed_for(cfg, start) + 1), y, g, q)
    return out
