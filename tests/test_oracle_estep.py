"""Pins for the oracle's density and E-step (eqs 4, 12-17), CPU only."""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp
import scipy.stats as st


def _spec(oracle, seed=5):
    return oracle.qmc(1024, 8, 119, seed)


def _rand_spd(rng, p, jitter=0.5):
    A = rng.standard_normal((p, p))
    return A @ A.T / p + jitter * np.eye(p)


@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_delta_zero_is_multivariate_t(oracle, q):
    # Sec. 2: Delta = 0 reduces eq (4) to the multivariate t density (3)
    rng = np.random.default_rng(10 + q)
    p = 4
    S = _rand_spd(rng, p)
    mu = rng.normal(0, 1, p)
    nu = 5.7
    for _ in range(3):
        y = mu + rng.normal(0, 2, p)
        r = oracle.pair(y, mu, S, np.zeros((p, q)), nu, _spec(oracle))
        ref = st.multivariate_t(loc=mu, shape=S, df=nu).logpdf(y)
        assert abs(r["logf"] - ref) < 1e-12 * max(1.0, abs(ref))
        # E-step quantities with Delta = 0 have closed forms: u = (nu+p)/(nu+d),
        # elogu = psi((nu+p)/2) - log((nu+d)/2) (the one-step-late term cancels),
        # U is the positive part of a spherical t, so with m = nu+p+2 and
        # s^2 = (nu+d)/m: E[W U_r] = u s 2 sqrt(m) G((m+1)/2) / (sqrt(pi) (m-1) G(m/2))
        # and E[W U U^T] = I + (2/pi)(1 1^T - I).
        d = float((y - mu) @ np.linalg.solve(S, y - mu))
        u = (nu + p) / (nu + d)
        assert abs(r["u"] - u) < 1e-12 * u
        el = sp.digamma((nu + p) / 2) - math.log((nu + d) / 2)
        assert abs(r["elogu"] - el) < 1e-12 * max(1.0, abs(el))
        m = nu + p + 2
        s = math.sqrt((nu + d) / m)
        e1 = u * s * 2 * math.sqrt(m) * math.exp(sp.gammaln((m + 1) / 2) - sp.gammaln(m / 2)) \
            / (math.sqrt(math.pi) * (m - 1))
        assert np.allclose(r["eu"], e1, rtol=1e-10, atol=0)
        E2 = np.eye(q) + (2 / math.pi) * (np.ones((q, q)) - np.eye(q))
        assert np.allclose(r["euu"], E2, rtol=1e-10, atol=1e-12)


def test_univariate_matches_hierarchy_integral(oracle):
    # p = q = 1: f(y) = int int N(y; mu + delta u, sigma^2/w) 2 N(u; 0, 1/w) 1(u>0)
    #                     gamma(w; nu/2, nu/2) du dw   (eq 6), by 2-D quadrature
    mu, sig2, delta, nu = 0.3, 1.7, 1.4, 6.5
    for y in [-2.0, 0.9, 4.0]:
        def integrand(u, w):
            return (st.norm.pdf(y, mu + delta * u, math.sqrt(sig2 / w))
                    * 2 * st.norm.pdf(u, 0, math.sqrt(1 / w))
                    * st.gamma.pdf(w, nu / 2, scale=2 / nu))
        ref, _ = si.dblquad(integrand, 0, np.inf, 0, np.inf, epsabs=1e-12, epsrel=1e-10)
        r = oracle.pair([y], [mu], [[sig2]], [[delta]], nu, _spec(oracle))
        assert abs(r["logf"] - math.log(ref)) < 1e-7


@pytest.mark.parametrize("q", [1, 2])
def test_density_integrates_to_one(oracle, q):
    # int f(y) dy = 1 by tensor Gauss-Legendre after y = mu + s tan(theta)
    p = 2
    if q == 2:
        Sigma = np.array([[1.0, 0.5], [0.5, 1.0]])
        Delta = np.array([[1.0, 0.5], [0.0, 1.5]])
    else:
        Sigma = np.array([[1.0, 0.3], [0.3, 0.8]])
        Delta = np.array([[1.2], [-0.7]])
    mu = np.array([0.5, -0.2])
    nu = 6.0
    nq = 64
    x, wts = np.polynomial.legendre.leggauss(nq)
    th = x * math.pi / 2
    wt = wts * math.pi / 2
    sc = 3.0
    Y = []
    W = []
    for i in range(nq):
        for j in range(nq):
            Y.append(mu + sc * np.array([math.tan(th[i]), math.tan(th[j])]))
            W.append(wt[i] * wt[j] * sc * sc / (math.cos(th[i]) ** 2 * math.cos(th[j]) ** 2))
    Y = np.array(Y)
    params = dict(pi=[1.0], mu=[mu], Sigma=[Sigma], Delta=[Delta], nu=[nu])
    e = oracle.estep(Y, params, _spec(oracle))
    total = float(np.sum(np.exp(e["logf"][0]) * np.array(W)))
    assert abs(total - 1.0) < 2e-5


def test_skew_normal_limit(oracle):
    # nu -> infinity: 2^q phi_p(y; mu, Omega) Phi_q(c; 0, Lambda), eq (5); gap ~ 1/nu
    p, q = 2, 2
    mu = np.array([0.2, -0.4])
    Sigma = np.array([[1.0, 0.3], [0.3, 1.5]])
    Delta = np.array([[0.8, -0.3], [0.2, 1.1]])
    Om = Sigma + Delta @ Delta.T
    Oi = np.linalg.inv(Om)
    Lam = np.eye(q) - Delta.T @ Oi @ Delta
    for y in [np.array([0.5, 0.5]), np.array([-1.0, 1.3])]:
        c = Delta.T @ Oi @ (y - mu)
        ref = (q * math.log(2) + st.multivariate_normal(mu, Om).logpdf(y)
               + math.log(st.multivariate_normal(np.zeros(q), Lam).cdf(c)))
        g3 = oracle.pair(y, mu, Sigma, Delta, 1e3, _spec(oracle))["logf"] - ref
        g4 = oracle.pair(y, mu, Sigma, Delta, 1e4, _spec(oracle))["logf"] - ref
        assert abs(g4) < 1e-3
        assert abs(g3 / g4 - 10.0) < 0.6, (g3, g4)


def _mc_moments(y, mu, Sigma, Delta, nu, n, seed):
    """Importance sampling from the prior of eq (6): draw (W, U), weight by
    N(y; mu + Delta U, Sigma/W); return estimates and batch standard errors."""
    rng = np.random.default_rng(seed)
    p, q = Delta.shape
    Lc = np.linalg.cholesky(Sigma)
    Li = np.linalg.inv(Lc)
    ld = np.log(np.diag(Lc)).sum()
    nb = 16
    m = n // nb
    rows = []
    for _ in range(nb):
        Wd = np.ones(m) if np.isinf(nu) else rng.gamma(nu / 2, 2 / nu, m)
        U = np.abs(rng.standard_normal((m, q))) / np.sqrt(Wd)[:, None]
        z = (y - mu - U @ Delta.T) @ Li.T
        wt = np.exp(-0.5 * Wd * (z * z).sum(1) + 0.5 * p * np.log(Wd)
                    - 0.5 * p * math.log(2 * math.pi) - ld)
        f = wt.mean()
        rows.append(np.concatenate([[f, (wt * Wd).mean() / f],
                                    (wt * Wd) @ U / m / f,
                                    (np.einsum("i,ij,ik->jk", wt * Wd, U, U) / m / f).ravel()]))
    R = np.array(rows)
    est = R.mean(0)
    se = R.std(0, ddof=1) / math.sqrt(nb)
    return est, se


@pytest.mark.parametrize("case", ["p2q2", "p3q3", "p4q1"])
def test_moments_brute_force(oracle, case):
    rng = np.random.default_rng(20)
    if case == "p2q2":
        y, mu = np.array([5.5, 6.0]), np.array([4.0, 4.0])
        Sigma = np.array([[1.0, 0.5], [0.5, 1.0]])
        Delta = np.array([[1.0, 0.5], [0.0, 1.5]])
        nu = 10.0
    elif case == "p3q3":
        y, mu = np.array([0.8, -0.3, 1.5]), np.zeros(3)
        Sigma = _rand_spd(rng, 3)
        Delta = rng.normal(0, 1, (3, 3))
        nu = 6.3
    else:
        y, mu = np.array([1.0, 0.5, -0.2, 2.0]), np.zeros(4)
        Sigma = _rand_spd(rng, 4)
        Delta = rng.normal(0, 1.2, (4, 1))
        nu = 5.0
    q = Delta.shape[1]
    r = oracle.pair(y, mu, Sigma, Delta, nu, _spec(oracle))
    est, se = _mc_moments(y, mu, Sigma, Delta, nu, 3_200_000, 7)
    got = np.concatenate([[math.exp(r["logf"]), r["u"]], r["eu"], r["euu"].ravel()])
    z = np.abs(got - est) / np.maximum(se, 1e-12)
    assert np.all(z < 5.0), (case, got, est, se)


def test_estep_invariants(oracle):
    from paper_1606_02054_gb300 import synth

    w = synth.make_workload("flow_p4", n=60, with_init=False)
    e = oracle.estep(w["y"], w["truth"], oracle.qmc(**w["qmc"]))
    assert np.allclose(e["tau"].sum(0), 1.0, atol=1e-13)
    assert np.all(e["tau"] >= 0) and np.all(e["u"] > 0)
    g, n, q = e["eu"].shape
    t = w["truth"]
    checked = 0
    for h in range(g):
        Om = t["Sigma"][h] + t["Delta"][h] @ t["Delta"][h].T
        ltp = st.multivariate_t(loc=t["mu"][h], shape=Om, df=t["nu"][h]).logpdf(w["y"])
        alpha_s = np.exp(e["logf"][h] - q * math.log(2) - ltp)
        for j in range(n):
            E3 = e["euu"][h, j]
            assert np.allclose(E3, E3.T, atol=1e-15)
            # E[W] E[W U U^T] - E[W U] E[W U]^T is positive semidefinite.  The
            # lattice estimate of T_q loses relative accuracy far in its tail,
            # where the moment formulas cancel; check where it is accurate.
            if e["se"][h, j] > 1e-3 * alpha_s[j]:
                continue
            checked += 1
            C = e["u"][h, j] * E3 - np.outer(e["eu"][h, j], e["eu"][h, j])
            assert np.linalg.eigvalsh(C).min() > -1e-6 * np.abs(C).max(), (h, j)
    assert checked >= n // 2
    # log-likelihood = sum_j log sum_h pi_h f_h (eq 27)
    lse = sp.logsumexp(np.log(w["truth"]["pi"])[:, None] + e["logf"], axis=0).sum()
    assert abs(e["loglik"] - lse) < 1e-9 * abs(lse)


# ---------------------------------------------------------------------------
# single-pass (ratio-estimator) truncated-t moments, q >= 3
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("q", [3, 4])
def test_single_pass_moments_match_recursion(oracle, q):
    rng = np.random.default_rng(30 + q)
    p = q
    Sigma = _rand_spd(rng, p)
    Delta = rng.normal(0, 1.0, (p, q))
    nu = 6.5
    big = oracle.qmc(16384, 16, 5693, 11, 1)
    for _ in range(3):
        y = rng.normal(0, 1.5, p)
        rec = oracle.pair(y, np.zeros(p), Sigma, Delta, nu, oracle.qmc(16384, 16, 5693, 11, 0))
        sp1 = oracle.pair(y, np.zeros(p), Sigma, Delta, nu, big)
        # alpha: the recursion's T_q at nu+p+2 and the single pass's W/(nu+p)-weighted pass
        # of alpha_s are two unbiased lattice estimates of the same integral (2.6e5 points)
        assert abs(sp1["u"] - rec["u"]) <= 2e-5 * rec["u"] and sp1["logf"] == rec["logf"]
        scale = np.abs(rec["euu"]).max()
        assert np.abs(sp1["eu"] - rec["eu"]).max() <= 2e-3 * np.abs(rec["eu"]).max()
        assert np.abs(sp1["euu"] - rec["euu"]).max() <= 3e-3 * scale


def test_single_pass_moments_are_psd_everywhere(oracle):
    from paper_1606_02054_gb300 import synth

    w = synth.make_workload("flow_p4", n=40, with_init=False)
    e = oracle.estep(w["y"], w["truth"], oracle.qmc(**dict(w["qmc"], moments=1)))
    g, n, q = e["eu"].shape
    for h in range(g):
        for j in range(n):
            C = e["u"][h, j] * e["euu"][h, j] - np.outer(e["eu"][h, j], e["eu"][h, j])
            # a weighted covariance of lattice draws: PSD up to rounding, also far in the tail
            assert np.linalg.eigvalsh(C).min() >= -1e-9 * max(np.abs(C).max(), 1e-300), (h, j)


def test_single_pass_delta_zero(oracle):
    # Delta = 0: E[W U] = u s 2 sqrt(m) G((m+1)/2)/(sqrt(pi)(m-1)G(m/2)), E[W U U^T] = I + (2/pi)(11^T - I)
    p = q = 4
    rng = np.random.default_rng(44)
    S = _rand_spd(rng, p)
    nu = 5.7
    y = rng.normal(0, 2, p)
    r = oracle.pair(y, np.zeros(p), S, np.zeros((p, q)), nu, oracle.qmc(4096, 16, 1517, 3, 1))
    d = float(y @ np.linalg.solve(S, y))
    u = (nu + p) / (nu + d)
    m = nu + p + 2
    s = math.sqrt((nu + d) / m)
    e1 = u * s * 2 * math.sqrt(m) * math.exp(sp.gammaln((m + 1) / 2) - sp.gammaln(m / 2)) \
        / (math.sqrt(math.pi) * (m - 1))
    assert np.allclose(r["eu"], e1, rtol=5e-3)
    E2 = np.eye(q) + (2 / math.pi) * (np.ones((q, q)) - np.eye(q))
    assert np.allclose(r["euu"], E2, rtol=1e-2, atol=1e-2)



# ---------------------------------------------------------------------------
# nu = infinity: the CFUSN model of eq (5)
# ---------------------------------------------------------------------------
def test_phi2_closed_forms_and_scipy(oracle):
    import scipy.stats as st
    for rho in (-0.9, -0.3, 0.0, 0.45, 0.99):
        assert abs(oracle.phi2(0.0, 0.0, rho) - (0.25 + math.asin(rho) / (2 * math.pi))) < 1e-14
    assert abs(oracle.phi2(0.7, -0.4, 0.0) - st.norm.cdf(0.7) * st.norm.cdf(-0.4)) < 1e-15
    assert abs(oracle.phi2(0.3, 1.1, 1.0) - st.norm.cdf(0.3)) < 1e-15
    for h, k, rho in ((0.5, -1.2, 0.6), (-2.0, -1.5, -0.7), (1.3, 0.2, 0.95), (-3.0, 2.0, 0.3)):
        mvn = st.multivariate_normal(mean=[0, 0], cov=[[1, rho], [rho, 1]])
        assert abs(oracle.phi2(h, k, rho) - mvn.cdf([h, k])) < 1e-9
    # T_2 -> Phi_2 at rate 1/nu
    g1 = oracle.t2cdf(0.5, -1.2, 0.6, 1e2) - oracle.phi2(0.5, -1.2, 0.6)
    g2 = oracle.t2cdf(0.5, -1.2, 0.6, 1e3) - oracle.phi2(0.5, -1.2, 0.6)
    assert 7 < g1 / g2 < 13
    assert oracle.t2cdf(0.5, -1.2, 0.6, math.inf) == oracle.phi2(0.5, -1.2, 0.6)


def test_skew_normal_univariate_closed_form(oracle):
    """p = q = 1, nu = inf: Azzalini's skew normal 2 phi(y; mu, omega^2) Phi(a (y - mu)/omega),
    omega^2 = sigma^2 + delta^2, a = delta / sigma."""
    import scipy.stats as st
    mu, sig2, dl = 0.4, 1.3, -0.9
    om = math.sqrt(sig2 + dl * dl)
    a = dl / math.sqrt(sig2)
    for y in (-3.0, -0.5, 0.4, 1.7, 4.0):
        r = oracle.pair(np.array([y]), np.array([mu]), np.array([[sig2]]), np.array([[dl]]), math.inf,
                        _spec(oracle))
        ref = math.log(2 * st.norm.pdf(y, mu, om) * st.norm.cdf(a * (y - mu) / om))
        assert abs(r["logf"] - ref) < 1e-12
        assert r["u"] == 1.0


@pytest.mark.parametrize("q", [1, 2])
def test_skew_normal_density_integrates_to_one(oracle, q):
    p = 2
    if q == 2:
        Sigma = np.array([[1.0, 0.5], [0.5, 1.0]])
        Delta = np.array([[1.0, 0.5], [0.0, 1.5]])
    else:
        Sigma = np.array([[1.0, 0.3], [0.3, 0.8]])
        Delta = np.array([[1.2], [-0.7]])
    mu = np.array([0.5, -0.2])
    x, wts = np.polynomial.legendre.leggauss(64)
    sc = 4.0
    Y, W = [], []
    for i in range(64):
        for j in range(64):
            Y.append(mu + sc * np.array([x[i], x[j]]) * 2.5)
            W.append(wts[i] * wts[j] * (sc * 2.5) ** 2)
    params = dict(pi=[1.0], mu=[mu], Sigma=[Sigma], Delta=[Delta], nu=[math.inf])
    e = oracle.estep(np.array(Y), params, _spec(oracle))
    total = float(np.sum(np.exp(e["logf"][0]) * np.array(W)))
    assert abs(total - 1.0) < 1e-6


@pytest.mark.parametrize("case", ["p2q2", "p3q3"])
def test_skew_normal_moments_brute_force(oracle, case):
    rng = np.random.default_rng(21)
    if case == "p2q2":
        y, mu = np.array([5.5, 6.0]), np.array([4.0, 4.0])
        Sigma = np.array([[1.0, 0.5], [0.5, 1.0]])
        Delta = np.array([[1.0, 0.5], [0.0, 1.5]])
    else:
        y, mu = np.array([0.8, -0.3, 1.5]), np.zeros(3)
        Sigma = _rand_spd(rng, 3)
        Delta = rng.normal(0, 1, (3, 3))
    r = oracle.pair(y, mu, Sigma, Delta, math.inf, _spec(oracle))
    est, se = _mc_moments(y, mu, Sigma, Delta, math.inf, 3_200_000, 9)
    got = np.concatenate([[math.exp(r["logf"]), r["u"]], r["eu"], r["euu"].ravel()])
    z = np.abs(got - est) / np.maximum(se, 1e-12)
    assert np.all(z < 5.0), (case, got, est, se)


def test_skew_normal_single_pass_matches_recursion(oracle):
    rng = np.random.default_rng(22)
    p, q = 3, 3
    Sigma = _rand_spd(rng, p)
    Delta = rng.normal(0, 1, (p, q))
    mu = np.zeros(p)
    for y in (np.array([0.8, -0.3, 1.5]), np.array([-1.0, 2.0, 0.2])):
        a = oracle.pair(y, mu, Sigma, Delta, math.inf, _spec(oracle))
        b = oracle.pair(y, mu, Sigma, Delta, math.inf, oracle.qmc(1024, 8, 119, 5, moments=1))
        assert a["logf"] == b["logf"]
        np.testing.assert_allclose(b["eu"], a["eu"], rtol=0, atol=5e-3 * np.abs(a["eu"]).max())
        np.testing.assert_allclose(b["euu"], a["euu"], rtol=0, atol=5e-3 * np.abs(a["euu"]).max())


PHI2_TAILS = ((-6.27, 7.12, -0.311), (7.1, -6.3, -0.5), (-8.0, -9.0, 0.6), (-6.0, 6.5, -0.95),
              (-30.0, -2.5, 0.93), (3.0, -2.6, -0.999), (-4.0, -4.0, 0.999))


def test_phi2_far_tails(oracle):
    """Far-tail values against a 40-digit integral of phi(x) Phi((k - rho x)/sqrt(1 - rho^2))
    over x <= h: relative 1e-10, including the two lower-tail orientations of the
    rho = -1 bound and values far below 1e-100."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for h, k, rho in PHI2_TAILS:
        H, K, R = mp.mpf(h), mp.mpf(k), mp.mpf(rho)
        f = lambda x: mp.npdf(x) * mp.ncdf((K - R * x) / mp.sqrt(1 - R * R))
        # the integrand falls off over ~1/|h| below h: geometric breakpoints toward h
        pts = [-mp.inf] + [H - mp.mpf(2) ** j for j in range(5, -8, -1)] + [H]
        ref = float(mp.quad(f, pts))
        got = oracle.phi2(h, k, rho)
        assert abs(got - ref) <= 1e-10 * ref, (h, k, rho, got, ref)


def test_null_pair_beyond_fp64(oracle):
    """An observation on the far non-skewed side of a skew-normal component: Phi_q(c)
    is below the FP64 range (log Phi_2 < -745 by the Mills-ratio bound), so the pair has
    log f = -inf, tau = 0 and zeroed expectations, and the E-step and M-step stay finite."""
    Sigma = np.array([[1.0, 0.2], [0.2, 1.0]])
    Delta = np.array([[3.0, 0.0], [0.0, 3.0]])
    mu0, mu1 = np.array([0.0, 0.0]), np.array([-60.0, -60.0])
    y = np.array([-60.0, -60.0])  # 60 units below component 0 on both skewed axes
    r = oracle.pair(y, mu0, Sigma, Delta, math.inf, _spec(oracle))
    Om = Sigma + Delta @ Delta.T
    c = Delta.T @ np.linalg.solve(Om, y - mu0)
    Lam = np.eye(2) - Delta.T @ np.linalg.solve(Om, Delta)
    z = c[0] / math.sqrt(Lam[0, 0])
    # Phi_2(c) <= Phi(z) < phi(z)/|z|
    assert -0.5 * z * z - math.log(-z) - 0.5 * math.log(2 * math.pi) < -745.0
    assert r["logf"] == -math.inf and r["u"] == 1.0 and r["elogu"] == 0.0
    assert np.all(r["eu"] == 0.0) and np.all(r["euu"] == 0.0)
    rng = np.random.default_rng(4)
    Y = np.vstack([rng.normal(0, 1, (50, 2)), rng.normal(-60, 1, (50, 2)), y])
    params = dict(pi=[0.5, 0.5], mu=[mu0, mu1], Sigma=[Sigma, Sigma], Delta=[Delta, Delta],
                  nu=[math.inf, math.inf])
    e = oracle.estep(Y, params, _spec(oracle))
    assert e["logf"][0, -1] == -math.inf and e["tau"][0, -1] == 0.0 and e["tau"][1, -1] == 1.0
    assert np.isfinite(e["loglik"]) and np.all(np.isfinite(e["eu"])) and np.all(np.isfinite(e["euu"]))
    P, _ = oracle.mstep(Y, e, params, hold=oracle.HOLD_NU)
    for key in ("pi", "mu", "Sigma", "Delta"):
        assert np.all(np.isfinite(P[key])), key


def test_joint_pass_change_of_measure(oracle):
    """The single-pass estimator weights alpha_s's lattice pass (chi-square at k1 dof) by
    W/k1, the density ratio of chi-square(k1 + 2) to chi-square(k1).  Pinned against an
    independent plain lattice T_q at k1 + 2 (different points: within 5e-5 relative on
    16384 x 16 points), the old moment pass at k1 + 2 (same quantity, other estimator),
    and the orthant closed form: at c = 0 and equicorrelation 1/2, T_q = 1/(q + 1) for every
    dof."""
    rng = np.random.default_rng(41)
    big = oracle.qmc(16384, 16, 5693, 13)
    for q in (3, 4):
        A = rng.normal(0, 1, (q, q + 2))
        Lam = A @ A.T / (q + 2) + 0.3 * np.eye(q)
        c = rng.normal(0.3, 1.0, q)
        nud, k1 = 9.3, 8.0
        k2 = k1 + 2.0
        a, m1, m2 = oracle.tk_joint(c, Lam, nud, k1, big)
        ref, se = oracle.tkcdf(c * np.sqrt(k2 / nud), Lam, k2, big)
        assert abs(a - ref) <= max(5e-5 * ref, 6 * se), (q, a, ref, se)
        a2, r1, r2 = oracle.tk_moments(c, nud / k2 * Lam, k2, big)
        assert abs(a2 - ref) <= 1e-12 * ref  # the old pass: the same points as the plain T_q
        np.testing.assert_allclose(m1, r1, rtol=0, atol=2e-3 * np.abs(r1).max())
        np.testing.assert_allclose(m2, r2, rtol=0, atol=3e-3 * np.abs(r2).max())
        R = np.full((q, q), 0.5) + 0.5 * np.eye(q)
        a0, _, _ = oracle.tk_joint(np.zeros(q), R, 7.0, 5.0, big)
        assert abs(a0 - 1.0 / (q + 1)) <= 2e-4, (q, a0)


# ---------------------------------------------------------------------------
# Exact E[log W | y] from the single pass (elogw = 1) in place of the OSL eq (15)
# ---------------------------------------------------------------------------
def _elogw_reference(y, mu, Sigma, Delta, nu):
    """E[log W | y] for one component by a 1-D integral over t = log W: the posterior of W
    is the Gamma((nu+p)/2, rate (nu+d)/2) law tilted by Phi_q(sqrt(W) c; 0, Lambda) (the
    hierarchy of eq 6 with U0 integrated out), so in t its density is proportional to
    exp(a t - b e^t) Phi_q(e^(t/2) c), a = (nu+p)/2, b = (nu+d)/2; trapezoid rule on a
    wide uniform grid (exponentially accurate for this smooth, fast-decaying integrand),
    Phi_q by scipy's multivariate normal CDF."""
    p, q = Delta.shape
    Om = Sigma + Delta @ Delta.T
    r = y - mu
    Oir = np.linalg.solve(Om, r)
    d = float(r @ Oir)
    c = Delta.T @ Oir
    Lam = np.eye(q) - Delta.T @ np.linalg.solve(Om, Delta)
    a, b = (nu + p) / 2, (nu + d) / 2
    t0 = math.log(a / b)
    t = np.linspace(t0 - 30.0 / math.sqrt(a) - 8.0, t0 + 20.0 / math.sqrt(a), 120)
    mvn = st.multivariate_normal(mean=np.zeros(q), cov=Lam, abseps=1e-13, releps=1e-6, maxpts=400_000)
    phi = np.array([mvn.cdf(math.exp(0.5 * ti) * c) for ti in t])
    lg = a * t - b * np.exp(t)
    wgt = np.exp(lg - lg.max()) * phi
    return float(np.sum(t * wgt) / np.sum(wgt)), d


def test_exact_elogw_delta_zero(oracle):
    """Delta = 0: the tilt is a constant, the posterior of W is Gamma((nu+p)/2, (nu+d)/2)
    and E[log W | y] = psi((nu+p)/2) - log((nu+d)/2) -- which the OSL form of eq (15)
    also gives here, exactly but for the lattice error of its u.  The lattice mean of
    log W is within its QMC error."""
    p = q = 3
    rng = np.random.default_rng(61)
    S = _rand_spd(rng, p)
    nu = 6.3
    y = rng.normal(0, 1.5, p)
    spec = oracle.qmc(4096, 16, 1517, 3, 1, 1)
    r = oracle.pair(y, np.zeros(p), S, np.zeros((p, q)), nu, spec)
    d = float(y @ np.linalg.solve(S, y))
    ref = sp.digamma((nu + p) / 2) - math.log((nu + d) / 2)
    assert abs(r["elogu"] - ref) <= 2e-4 * max(1.0, abs(ref))
    osl = oracle.pair(y, np.zeros(p), S, np.zeros((p, q)), nu, oracle.qmc(4096, 16, 1517, 3, 1, 0))
    assert abs(osl["elogu"] - ref) <= 1e-5 * max(1.0, abs(ref))


@pytest.mark.parametrize("case", [0, 1, 2])
def test_exact_elogw_matches_tilted_gamma_integral(oracle, case):
    """Skewed components (q = 3, 4): the single-pass E[log W | y] equals the integral of
    log W against the tilted Gamma posterior to the lattice's error (1.5e-3; case 1 puts y
    on the unskewed side, where the tilt is steep and the 4096 x 16 lattice's mean is
    9e-4 off), where the OSL form of eq (15) is off by 7e-3 to 0.43."""
    rng = np.random.default_rng(700 + case)
    p, q = (3, 3) if case < 2 else (4, 4)
    S = _rand_spd(rng, p)
    Delta = rng.normal(0, 1.2, (p, q))
    nu = [4.5, 9.0, 6.0][case]
    mu = np.zeros(p)
    y = rng.normal(0, 1.0, p) + (Delta @ np.abs(rng.normal(0, 1, q))) * (1 if case != 1 else -1)
    ref, d = _elogw_reference(y, mu, S, Delta, nu)
    ex = oracle.pair(y, mu, S, Delta, nu, oracle.qmc(4096, 16, 1517, 9, 1, 1))
    osl = oracle.pair(y, mu, S, Delta, nu, oracle.qmc(4096, 16, 1517, 9, 1, 0))
    assert abs(ex["elogu"] - ref) <= 1.5e-3 * max(1.0, abs(ref)), (ex["elogu"], ref)
    assert abs(osl["elogu"] - ref) > 3 * abs(ex["elogu"] - ref)
    # the same pass's u = E[W | y] (eq 13) is unchanged by the elogw reading
    assert ex["u"] == osl["u"] and np.array_equal(ex["eu"], osl["eu"])
    print(f"case {case}: exact {ex['elogu']:.6f}, integral {ref:.6f}, OSL {osl['elogu']:.6f}")
