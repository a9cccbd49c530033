"""Pins for the oracle's M-step (eqs 18-22), Aitken rule (24-26) and EM loop."""
import math

import numpy as np
import pytest
import scipy.special as sp

from paper_1606_02054_gb300 import synth


def _q_block(y, tau, u, e2, e3, mu, Delta, Sigma):
    """Expected complete-data log-likelihood of one component's
    N(y; mu + Delta U, Sigma / W) term of eq (6), written from the hierarchy:
    sum_j tau_j [-1/2 log|Sigma| - 1/2 tr(Sigma^{-1} M_j)],
    M_j = u r r^T - Delta e2 r^T - r e2^T Delta^T + Delta e3 Delta^T, r = y_j - mu."""
    R = y - mu
    M = (np.einsum("j,ja,jb->ab", tau * u, R, R)
         - Delta @ np.einsum("j,jk,jb->kb", tau, e2, R)
         - np.einsum("j,ja,jk->ak", tau, R, e2) @ Delta.T
         + Delta @ np.einsum("j,jkl->kl", tau, e3) @ Delta.T)
    sign, logdet = np.linalg.slogdet(Sigma)
    return -0.5 * tau.sum() * logdet - 0.5 * np.trace(np.linalg.solve(Sigma, M))


def _q_nu(tau, u, el, nu):
    return np.sum(tau * (0.5 * nu * math.log(nu / 2) - sp.gammaln(nu / 2) + 0.5 * nu * (el - u)))


@pytest.fixture(scope="module")
def em_step(oracle):
    w = synth.make_workload("flow_p4", n=400)
    spec = oracle.qmc(**w["qmc"])
    e = oracle.estep(w["y"], w["init"], spec)
    new, flag = oracle.mstep(w["y"], e, w["init"])
    return w, e, new


def test_mstep_blocks_maximise_q(em_step):
    w, e, new = em_step
    y = w["y"]
    old = w["init"]
    rng = np.random.default_rng(0)
    g = old["pi"].size
    for h in range(g):
        args = (y, e["tau"][h], e["u"][h], e["eu"][h], e["euu"][h])
        mu1, D1, S1 = new["mu"][h], new["Delta"][h], new["Sigma"][h]
        D0, S0 = old["Delta"][h], old["Sigma"][h]
        # eq (19): mu^(k+1) maximises Q(mu, Delta^(k), Sigma) for any Sigma
        base = _q_block(*args, mu1, D0, S0)
        for _ in range(4):
            v = rng.standard_normal(mu1.size) * 1e-3
            assert _q_block(*args, mu1 + v, D0, S0) < base
        # eq (20): Delta^(k+1) maximises Q(mu^(k+1), Delta, Sigma) for any Sigma
        base = _q_block(*args, mu1, D1, S0)
        for _ in range(4):
            V = rng.standard_normal(D1.shape) * 1e-3
            assert _q_block(*args, mu1, D1 + V, S0) < base
        # eq (21): Sigma^(k+1) maximises Q(mu^(k+1), Delta^(k+1), Sigma)
        base = _q_block(*args, mu1, D1, S1)
        for _ in range(4):
            A = rng.standard_normal(S1.shape) * 1e-3
            assert _q_block(*args, mu1, D1, S1 + A @ A.T + 1e-4 * (A + A.T)) < base
        # gradient in mu vanishes (central differences)
        gr = []
        for i in range(mu1.size):
            d = np.zeros(mu1.size); d[i] = 1e-5
            gr.append((_q_block(*args, mu1 + d, D0, S0) - _q_block(*args, mu1 - d, D0, S0)) / 2e-5)
        assert np.max(np.abs(gr)) < 1e-5 * e["tau"][h].sum()
        # eq (18)
        assert abs(new["pi"][h] - e["tau"][h].mean()) < 1e-15
        # eq (22): nu^(k+1) maximises the nu part of Q
        t, u, el = e["tau"][h], e["u"][h], e["elogu"][h]
        v1 = new["nu"][h]
        assert _q_nu(t, u, el, v1) >= _q_nu(t, u, el, v1 * (1 + 1e-4))
        assert _q_nu(t, u, el, v1) >= _q_nu(t, u, el, v1 * (1 - 1e-4))


def test_nu_root(oracle):
    for n_h, s_h in [(100.0, -130.0), (5.0, -5.6), (1e4, -1.02e4)]:
        v, fl = oracle.nu_root(n_h, s_h)
        assert fl == 0
        F = n_h * (math.log(v / 2) - sp.digamma(v / 2) + 1) + s_h
        assert abs(F) < 1e-9 * n_h
    # no root in the bracket: clamp and flag
    v, fl = oracle.nu_root(100.0, -100.001)
    assert v == 200.0 and fl == 1
    v, fl = oracle.nu_root(100.0, -1e4)
    assert v == 1.0 and fl == -1


def test_aitken(oracle):
    # l_k = L - C r^k: Aitken's estimate (eqs 25-26) is exactly L
    L, C, r = -1234.5, 10.0, 0.6
    ls = [L - C * r ** k for k in range(80)]
    conv, linf = oracle.aitken_converged(ls[2], ls[3], ls[4], 1e-6)
    assert abs(linf - L) < 1e-9 and not conv
    k = next(k for k in range(2, 80) if oracle.aitken_converged(ls[k - 2], ls[k - 1], ls[k], 1e-6)[0])
    # |l_inf - l_k| = C r^k: the rule (eq 24) stops at the first k with C r^k < eps
    assert abs(ls[k] - L) < 1e-6 <= abs(ls[k - 1] - L)
    # equal consecutive values: treated as converged
    assert oracle.aitken_converged(-5.0, -4.0, -4.0, 1e-6)[0]
    assert oracle.aitken_converged(-4.0, -4.0, -4.0, 1e-6)[0]


def test_ecm_monotone_with_fixed_nu(oracle):
    # q = 2: T_q is deterministic and the E-step exact; with nu held fixed each
    # CM-step maximises Q, so the log-likelihood cannot decrease.
    w = synth.make_workload("two_comp_p2", n=1000)
    spec = oracle.qmc(**w["qmc"])
    _, hist, k = oracle.fit(w["y"], w["init"], 25, spec, nu_min=10.0, nu_max=10.0)
    assert k == 25 and hist.size == 26
    d = np.diff(hist)
    assert np.all(d > -1e-9 * abs(hist[-1])), d


def test_fit_recovers_generating_parameters(oracle):
    w = synth.make_workload("two_comp_p2", n=1500)
    spec = oracle.qmc(**w["qmc"])
    est, hist, k = oracle.fit(w["y"], w["init"], 40, spec)
    t = w["truth"]
    order = [int(np.argmin([np.linalg.norm(est["mu"][h] - t["mu"][s]) for h in range(2)]))
             for s in range(2)]
    assert sorted(order) == [0, 1]
    for s, h in enumerate(order):
        assert abs(est["pi"][h] - t["pi"][s]) < 0.08
        Om_e = est["Sigma"][h] + est["Delta"][h] @ est["Delta"][h].T
        Om_t = t["Sigma"][s] + t["Delta"][s] @ t["Delta"][s].T
        # location of the skewed component: mean = mu + sqrt(2/pi) Delta 1 (nu > 1 factor aside)
        assert np.linalg.norm(est["mu"][h] + est["Delta"][h].sum(1) * 0.8
                              - t["mu"][s] - t["Delta"][s].sum(1) * 0.8) < 0.6
        assert np.linalg.norm(Om_e - Om_t) / np.linalg.norm(Om_t) < 0.5
    assert hist[-1] > hist[0]


def _t_mixture_em(y, pi, mu, Sigma, nu, iters):
    """Textbook ECM for a mixture of multivariate t (McLachlan & Peel), written
    independently: E-step tau, u = (nu+p)/(nu+d); CM-steps pi, mu = sum tau u y /
    sum tau u, Sigma = sum tau u r r^T / sum tau, then nu from
    log(nu/2) - psi(nu/2) + 1 + (1/N) sum tau (log u - u) + psi((nu_k+p)/2) - log((nu_k+p)/2) = 0."""
    import scipy.optimize as so
    import scipy.special as sps
    from scipy.stats import multivariate_t

    n, p = y.shape
    g = len(pi)
    pi, mu, Sigma, nu = pi.copy(), mu.copy(), Sigma.copy(), nu.copy()
    for _ in range(iters):
        logf = np.array([multivariate_t(mu[h], Sigma[h], df=nu[h]).logpdf(y) for h in range(g)])
        a = np.log(pi)[:, None] + logf
        tau = np.exp(a - np.logaddexp.reduce(a, axis=0))
        for h in range(g):
            r = y - mu[h]
            d = np.einsum("ij,jk,ik->i", r, np.linalg.inv(Sigma[h]), r)
            u = (nu[h] + p) / (nu[h] + d)
            N = tau[h].sum()
            pi[h] = N / n
            mu[h] = (tau[h] * u) @ y / (tau[h] * u).sum()
            r = y - mu[h]
            Sigma[h] = (r * (tau[h] * u)[:, None]).T @ r / N
            c = (tau[h] * (np.log(u) - u)).sum() / N + sps.digamma((nu[h] + p) / 2) - np.log((nu[h] + p) / 2)
            f = lambda v: np.log(v / 2) - sps.digamma(v / 2) + 1 + c
            nu[h] = so.brentq(f, 1.0, 200.0, xtol=1e-14, rtol=1e-15) if f(1.0) > 0 > f(200.0) else nu[h]
    return pi, mu, Sigma, nu


def test_held_delta_zero_is_the_t_mixture_em(oracle):
    """Delta^(0) = 0 held by the M-step: the CFUST EM reduces to the t-mixture EM
    (the T_q factor of eq 4 is 2^-q, u is (nu+p)/(nu+d) and eq 15 is exact)."""
    w = synth.make_workload("flow_p4", n=400, with_init=False)
    y = w["y"][:, :3]
    g, q = 2, 2
    rng = np.random.default_rng(8)
    lab = rng.integers(0, g, len(y))
    P = dict(pi=np.array([0.5, 0.5]), mu=np.array([y[lab == h].mean(0) for h in range(g)]),
             Sigma=np.array([np.cov(y[lab == h], rowvar=False) for h in range(g)]),
             Delta=np.zeros((g, 3, q)), nu=np.array([8.0, 12.0]))
    got, hist, it = oracle.fit(y, P, 12, oracle.qmc(**w["qmc"]), hold=oracle.HOLD_DELTA)
    pi, mu, Sigma, nu = _t_mixture_em(y, P["pi"], P["mu"], P["Sigma"], P["nu"], 12)
    assert np.all(got["Delta"] == 0.0)
    np.testing.assert_allclose(got["pi"], pi, rtol=1e-9)
    np.testing.assert_allclose(got["mu"], mu, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(got["Sigma"], Sigma, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(got["nu"], nu, rtol=1e-8)


def test_held_nu_stays(oracle):
    w = synth.make_workload("two_comp_p2", n=300)
    got, hist, it = oracle.fit(w["y"], w["init"], 5, oracle.qmc(**w["qmc"]), hold=oracle.HOLD_NU)
    np.testing.assert_array_equal(got["nu"], np.asarray(w["init"]["nu"], dtype=float))
    assert np.all(np.diff(hist) > -1e-6 * np.abs(hist[:-1]))  # still an ECM (q = 2: exact moments)


def _normal_mixture_em(y, pi, mu, Sigma, iters):
    """Textbook EM for a mixture of multivariate normals, written independently."""
    from scipy.stats import multivariate_normal

    n, p = y.shape
    g = len(pi)
    pi, mu, Sigma = pi.copy(), mu.copy(), Sigma.copy()
    for _ in range(iters):
        a = np.log(pi)[:, None] + np.array([multivariate_normal(mu[h], Sigma[h]).logpdf(y) for h in range(g)])
        tau = np.exp(a - np.logaddexp.reduce(a, axis=0))
        for h in range(g):
            N = tau[h].sum()
            pi[h] = N / n
            mu[h] = tau[h] @ y / N
            r = y - mu[h]
            Sigma[h] = (r * tau[h][:, None]).T @ r / N
    return pi, mu, Sigma


def test_normal_limit_with_delta_zero_is_the_normal_mixture_em(oracle):
    """nu = inf (eq 5) with Delta^(0) = 0 held: the E-step has u = 1 and T_q = 2^-q, so the
    fit is the EM of a normal mixture."""
    w = synth.make_workload("flow_p4", n=400, with_init=False)
    y = w["y"][:, :3]
    g, q = 2, 2
    rng = np.random.default_rng(9)
    lab = rng.integers(0, g, len(y))
    P = dict(pi=np.array([0.5, 0.5]), mu=np.array([y[lab == h].mean(0) for h in range(g)]),
             Sigma=np.array([np.cov(y[lab == h], rowvar=False) for h in range(g)]),
             Delta=np.zeros((g, 3, q)), nu=np.array([np.inf, np.inf]))
    got, hist, it = oracle.fit(y, P, 12, oracle.qmc(**w["qmc"]), hold=oracle.HOLD_DELTA | oracle.HOLD_NU)
    pi, mu, Sigma = _normal_mixture_em(y, P["pi"], P["mu"], P["Sigma"], 12)
    assert np.all(got["Delta"] == 0.0) and np.all(np.isinf(got["nu"]))
    np.testing.assert_allclose(got["pi"], pi, rtol=1e-10)
    np.testing.assert_allclose(got["mu"], mu, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(got["Sigma"], Sigma, rtol=1e-10, atol=1e-12)
