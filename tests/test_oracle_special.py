"""Pins for the oracle's special functions (CPU only).

Each check compares the oracle with something other than itself: a
library routine written elsewhere (scipy.special), a closed form, an
identity, or an independent representation of the same quantity.
"""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp
import scipy.stats as st


def test_digamma(oracle):
    xs = [0.1, 0.5, 1.0, 1.7, 3.3, 9.99, 10.0, 47.5, 250.0, 1e4]
    for x in xs:
        assert abs(oracle.digamma(x) - sp.digamma(x)) <= 1e-14 * max(1.0, abs(sp.digamma(x)))
    # psi(1) = -Euler-Mascheroni constant; psi(x+1) = psi(x) + 1/x
    assert abs(oracle.digamma(1.0) + 0.5772156649015329) < 1e-15
    for x in [0.3, 2.2, 11.7]:
        assert abs(oracle.digamma(x + 1) - oracle.digamma(x) - 1 / x) < 1e-13


def test_phi_and_inverse(oracle):
    for x in [-38.0, -20.0, -5.5, -1.0, 0.0, 0.3, 2.0, 8.0]:
        ref = sp.ndtr(x)
        # relative conditioning of Phi in the lower tail is about x^2 * eps
        assert abs(oracle.phi(x) - ref) <= 1e-15 * (1 + x * x) * max(ref, 1e-300) + 1e-300
    for p in [1e-300, 1e-100, 1e-12, 1e-3, 0.02425, 0.3, 0.5, 0.7, 0.97575, 1 - 1e-12]:
        ref = sp.ndtri(p)
        assert abs(oracle.phi_inv(p) - ref) <= 2e-14 * max(1.0, abs(ref)), p


def test_incbeta_incgamma(oracle):
    rng = np.random.default_rng(0)
    for _ in range(200):
        a, b, x = rng.uniform(0.2, 60), rng.uniform(0.2, 30), rng.uniform(0, 1)
        ref = sp.betainc(a, b, x)
        assert abs(oracle.incbeta(a, b, x) - ref) <= 1e-12 * max(ref, 1e-12), (a, b, x)
    for _ in range(200):
        a, x = rng.uniform(0.3, 150), rng.uniform(0, 300)
        ref = sp.gammainc(a, x)
        assert abs(oracle.incgamma_p(a, x) - ref) <= 1e-12 * max(ref, 1e-12), (a, x)


def test_chi2_quantile(oracle):
    for nu in [1.0, 2.5, 7.3, 12.0, 30.0, 205.0]:
        for w in [1e-300, 1e-100, 1e-12, 1e-5, 0.01, 0.3, 0.5]:
            ref = 2 * sp.gammaincinv(nu / 2, w)
            assert abs(oracle.chi2_quantile(w, nu) - ref) <= 1e-12 * ref, (w, nu)
        for wc in [1e-300, 1e-50, 1e-12, 1e-3, 0.4]:
            ref = 2 * sp.gammainccinv(nu / 2, wc)
            assert abs(oracle.chi2_quantile(1 - wc, nu, wc) - ref) <= 1e-12 * ref, (wc, nu)


def test_t1_library_and_closed_forms(oracle):
    rng = np.random.default_rng(1)
    for _ in range(300):
        nu = rng.uniform(0.5, 250)
        x = rng.normal(0, 4)
        ref = sp.stdtr(nu, x)
        assert abs(oracle.t1cdf(x, nu) - ref) <= 1e-12 * max(ref, 1e-10), (x, nu)
        assert abs(oracle.t1pdf(x, nu) - st.t.pdf(x, nu)) <= 1e-12 * st.t.pdf(x, nu)
    for x in [-30.0, -2.0, -0.1, 0.0, 0.7, 5.0]:
        # nu = 1: Cauchy;  nu = 2: x / (2 sqrt(2 + x^2)) + 1/2
        assert abs(oracle.t1cdf(x, 1.0) - (0.5 + math.atan(x) / math.pi)) < 1e-14
        assert abs(oracle.t1cdf(x, 2.0) - (0.5 + x / (2 * math.sqrt(2 + x * x)))) < 1e-14
    assert oracle.t1cdf(0.0, 3.7) == 0.5


# -------------------------------------------------------------------------
# T_2 pins
# -------------------------------------------------------------------------
def _t2_plackett(h, k, rho, nu):
    """Bivariate t CDF from an independent representation: since
    T_2 = E_s[Phi_2(s h, s k; rho)] with s^2 ~ chi2_nu / nu, and
    dPhi_2/drho = phi_2, dT_2/drho = (1 + Q/nu)^(-nu/2) / (2 pi sqrt(1-rho^2))
    with Q = (h^2 - 2 rho h k + k^2) / (1 - rho^2).  Integrate from rho = +-1,
    where T_2 is a univariate t CDF (scipy.special.stdtr); r = sin(phi)."""
    def dens(phi):
        r = math.sin(phi)
        c2 = math.cos(phi) ** 2
        if c2 == 0.0:
            return 0.0 if h != k else (1 + h * h / nu) ** (-nu / 2) / (2 * math.pi)
        Q = (h * h - 2 * r * h * k + k * k) / c2
        return (1 + Q / nu) ** (-nu / 2) / (2 * math.pi)

    a = math.asin(rho)
    if rho >= 0:
        base = sp.stdtr(nu, min(h, k))
        val, _ = si.quad(dens, a, math.pi / 2, epsabs=1e-15, epsrel=1e-13, limit=500)
        return base - val
    base = max(0.0, sp.stdtr(nu, h) + sp.stdtr(nu, k) - 1.0)
    val, _ = si.quad(dens, -math.pi / 2, a, epsabs=1e-15, epsrel=1e-13, limit=500)
    return base + val


def _dunnett_sobel(h, k, r, nu):
    """Dunnett & Sobel (1954) finite series for the standard bivariate t CDF at
    integer nu, in the form given by Genz & Bretz (2009), Sec. 2.2.1."""
    om = 1.0 - r * r
    dh, dk = h - r * k, k - r * h
    if abs(dh) + om > 0:
        xh = dh * dh / (dh * dh + om * (nu + k * k))   # beta argument for the h-term
        xk = dk * dk / (dk * dk + om * (nu + h * h))   # ... and for the k-term
    else:
        xh = xk = 0.0
    sh = math.copysign(1.0, dh) if dh != 0 else 0.0
    sk = math.copysign(1.0, dk) if dk != 0 else 0.0
    if nu % 2 == 0:
        val = math.atan2(math.sqrt(om), -r) / (2 * math.pi)
        gh = h / math.sqrt(16 * (nu + h * h))
        gk = k / math.sqrt(16 * (nu + k * k))
        bk = 2 * math.atan2(math.sqrt(xk), math.sqrt(1 - xk)) / math.pi
        dbk = 2 * math.sqrt(xk * (1 - xk)) / math.pi
        bh = 2 * math.atan2(math.sqrt(xh), math.sqrt(1 - xh)) / math.pi
        dbh = 2 * math.sqrt(xh * (1 - xh)) / math.pi
        for j in range(1, nu // 2 + 1):
            val += gh * (1 + sk * bk) + gk * (1 + sh * bh)
            bk += dbk
            dbk *= 2 * j * (1 - xk) / (2 * j + 1)
            bh += dbh
            dbh *= 2 * j * (1 - xh) / (2 * j + 1)
            gh *= (2 * j - 1) / (2 * j * (1 + h * h / nu))
            gk *= (2 * j - 1) / (2 * j * (1 + k * k / nu))
        return val
    sn = math.sqrt(nu)
    qq = math.sqrt(h * h + k * k - 2 * r * h * k + nu * om)
    a1 = h * k + r * nu
    a2 = h * k - nu
    s = h + k
    val = math.atan2(-sn * (a2 * qq + s * a1), a2 * a1 - nu * s * qq) / (2 * math.pi)
    if val < -1e-15:
        val += 1.0
    gh = h / (2 * math.pi * sn * (1 + h * h / nu))
    gk = k / (2 * math.pi * sn * (1 + k * k / nu))
    bk = dbk = math.sqrt(xk)
    bh = dbh = math.sqrt(xh)
    for j in range(1, (nu - 1) // 2 + 1):
        val += gh * (1 + sk * bk) + gk * (1 + sh * bh)
        dbk *= (2 * j - 1) * (1 - xk) / (2 * j)
        bk += dbk
        dbh *= (2 * j - 1) * (1 - xh) / (2 * j)
        bh += dbh
        gh *= 2 * j / ((2 * j + 1) * (1 + h * h / nu))
        gk *= 2 * j / ((2 * j + 1) * (1 + k * k / nu))
    return val


def test_t2_orthant_and_degenerate(oracle):
    for nu in [1.5, 3.0, 7.7, 40.0]:
        for rho in [-0.95, -0.4, 0.0, 0.3, 0.9, 0.999]:
            ref = 0.25 + math.asin(rho) / (2 * math.pi)
            assert abs(oracle.t2cdf(0.0, 0.0, rho, nu) - ref) < 1e-13
        assert abs(oracle.t2cdf(0.4, -1.3, 1.0, nu) - sp.stdtr(nu, -1.3)) < 1e-14
        assert abs(oracle.t2cdf(0.4, 1.3, -1.0, nu)
                   - (sp.stdtr(nu, 0.4) + sp.stdtr(nu, 1.3) - 1)) < 1e-13


def test_t2_complement_and_symmetry(oracle):
    rng = np.random.default_rng(2)
    for _ in range(20):
        h, k = rng.normal(0, 2, 2)
        rho = rng.uniform(-0.97, 0.97)
        nu = rng.uniform(2, 30)
        a = oracle.t2cdf(h, k, rho, nu)
        # P(X<=h, Y<=k) + P(X<=h, Y>k) = T_1(h); (X, -Y) has correlation -rho
        assert abs(a + oracle.t2cdf(h, -k, -rho, nu) - sp.stdtr(nu, h)) < 1e-12
        assert abs(a - oracle.t2cdf(k, h, rho, nu)) < 1e-12


def test_t2_independent_representation(oracle):
    rng = np.random.default_rng(3)
    for _ in range(40):
        h, k = rng.normal(0, 2.5, 2)
        rho = rng.uniform(-0.99, 0.99)
        nu = rng.uniform(1.0, 60.0)
        ref = _t2_plackett(h, k, rho, nu)
        got = oracle.t2cdf(h, k, rho, nu)
        assert abs(got - ref) <= 1e-11 * max(ref, 1e-6), (h, k, rho, nu, got, ref)


def test_t2_dunnett_sobel(oracle):
    rng = np.random.default_rng(4)
    for nu in [1, 2, 3, 4, 5, 8, 13]:
        for _ in range(8):
            h, k = rng.normal(0, 2, 2)
            rho = rng.uniform(-0.95, 0.95)
            ref = _dunnett_sobel(h, k, rho, nu)
            assert abs(oracle.t2cdf(h, k, rho, nu) - ref) < 1e-12, (h, k, rho, nu)


def test_t2_normal_limit(oracle):
    # nu -> infinity gives the bivariate normal; the gap shrinks like 1/nu
    for h, k, rho in [(0.3, -0.7, 0.5), (-1.2, 0.4, -0.6), (1.5, 2.0, 0.9)]:
        ref = st.multivariate_normal(mean=[0, 0], cov=[[1, rho], [rho, 1]]).cdf([h, k])
        g3 = oracle.t2cdf(h, k, rho, 1e3) - ref
        g4 = oracle.t2cdf(h, k, rho, 1e4) - ref
        assert abs(g4) < 2e-5
        assert abs(g3 / g4 - 10.0) < 0.5, (g3, g4)


# -------------------------------------------------------------------------
# lattice and T_k (k >= 3) pins
# -------------------------------------------------------------------------
def test_splitmix64_published_vector(oracle):
    # SplitMix64 (Steele, Lea & Flood 2014): first output from state 0 is 0xE220A8397B1DCDAF
    assert oracle.splitmix64_u01(0) == (0xE220A8397B1DCDAF >> 11) * 2.0 ** -53


def test_tk_orthants(oracle):
    spec = oracle.qmc(1024, 8, 119, 99)
    # identity correlation, b = 0: every lattice point gives exactly 2^-k
    for k in (3, 4, 5, 6):
        v, se = oracle.tkcdf(np.zeros(k), np.eye(k), 7.3, spec)
        assert abs(v - 2.0 ** -k) < 1e-15 and se < 1e-15
    # equicorrelated rho = 1/2: orthant probability 1/(k+1) for any elliptical law
    for k in (3, 4, 5, 6):
        R = np.full((k, k), 0.5) + 0.5 * np.eye(k)
        v, se = oracle.tkcdf(np.zeros(k), R, 5.5, spec)
        assert abs(v - 1.0 / (k + 1)) < max(4 * se, 1e-6), (k, v, se)
    # k = 3 orthant: 1/8 + sum_{i<j} asin(rho_ij) / (4 pi)
    R = np.array([[1, 0.3, -0.5], [0.3, 1, 0.2], [-0.5, 0.2, 1]])
    v, se = oracle.tkcdf(np.zeros(3), R, 11.0, spec)
    ref = 0.125 + (math.asin(0.3) + math.asin(-0.5) + math.asin(0.2)) / (4 * math.pi)
    assert abs(v - ref) < max(4 * se, 1e-6)


def test_tk_reduces_to_t2(oracle):
    # a third coordinate with an enormous upper limit leaves T_2 of the other two
    spec = oracle.qmc(1024, 8, 119, 7)
    V = np.array([[1.5, 0.4, 0.2], [0.4, 2.0, -0.3], [0.2, -0.3, 1.0]])
    b = np.array([0.4, -0.8, 1e6])
    v, se = oracle.tkcdf(b, V, 6.6, spec)
    ref = oracle.t2cdf(0.4 / math.sqrt(1.5), -0.8 / math.sqrt(2.0), 0.4 / math.sqrt(3.0), 6.6)
    assert abs(v - ref) < max(4 * se, 1e-5)


def test_tk_against_library_and_high_n(oracle):
    rng = np.random.default_rng(5)
    spec = oracle.qmc(1024, 8, 119, 2024)
    big = oracle.qmc(16384, 16, 5693, 11)   # larger lattice, different generator
    for k in (3, 4, 5):
        A = rng.standard_normal((k, k))
        V = A @ A.T + 0.5 * np.eye(k)
        b = rng.normal(0.3, 1.0, k) * np.sqrt(np.diag(V))
        nu = rng.uniform(3, 25)
        v, se = oracle.tkcdf(b, V, nu, spec)
        vb, seb = oracle.tkcdf(b, V, nu, big)
        assert abs(v - vb) < 4 * math.hypot(se, seb) + 1e-7, (k, v, vb, se, seb)
        ref = st.multivariate_t(shape=V, df=nu, seed=1).cdf(b, maxpts=2_000_000)
        assert abs(v - ref) < 4 * se + 2e-4, (k, v, ref, se)


def test_tk_brute_force_mc(oracle):
    rng = np.random.default_rng(6)
    spec = oracle.qmc(1024, 8, 119, 3)
    k, nu = 3, 4.5
    V = np.array([[1.0, 0.6, 0.1], [0.6, 2.0, -0.4], [0.1, -0.4, 0.7]])
    b = np.array([0.2, 0.9, -0.3])
    v, se = oracle.tkcdf(b, V, nu, spec)
    m = 4_000_000
    Z = rng.standard_normal((m, k)) @ np.linalg.cholesky(V).T
    s = np.sqrt(rng.chisquare(nu, m) / nu)
    X = Z / s[:, None]
    hit = np.all(X <= b, axis=1)
    est = hit.mean()
    mc_se = math.sqrt(est * (1 - est) / m)
    assert abs(v - est) < 4 * math.hypot(mc_se, se)
