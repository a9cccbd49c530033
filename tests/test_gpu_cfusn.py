"""GPU: the CFUSN model (eq 5, the nu -> infinity limit; cfust_opts.model =
CFUST_MODEL_CFUSN) against the oracle's nu = inf path (pinned on the CPU in
tests/test_oracle_estep.py).

Tolerances: Phi and the lattice Phi_k (k >= 3, s = 1, same points) 1e-12
relative in FP64; Phi_2 1e-9 relative, the bar for deterministic Phi_q/T_q (two
graded Gauss-Legendre halves of 64 nodes against the oracle's adaptive
quadrature of the same Sheppard integrand: the rule emulated in FP64 on the
host agrees with the oracle to 2e-11 on these cases, far tails included);
per-pair log f 1e-9 (far-tail pairs included; measured 1.8e-10); the moments of
eqs (16)-(17) 1e-7 of the row scale (the recursion's q = 2 moment formulas cancel
in the far tails: measured 6.3e-8 at p = 16), and a pair that is null (T_q = 0 in FP64: log f = -inf) on one side has
log f < -700 on the other; FP32 modes: l 1e-6 relative; fits: final l 1e-6,
parameters 1e-4; the normal mixture (Delta = 0 held, T_q = 2^-q exactly): l 1e-9,
parameters 1e-8.
"""
import math

import numpy as np
import pytest

from paper_1606_02054_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_02054_gb300 import build

    build.build()
    import paper_1606_02054_gb300 as cf

    return cf


def _ctx(cf, w, params, precision=0, moments=1, n=None):
    q = w["qmc"]
    o = cf.cfust_default_opts(precision=precision, qmc_points=q["npoints"], qmc_shifts=q["nshifts"],
                              qmc_korobov_a=q["korobov_a"], seed=q["seed"], moments=moments,
                              model=cf.CFUST_MODEL_CFUSN)
    y = w["y"] if n is None else w["y"][:n]
    c = cf.cfust_create(w["p"], w["q"], w["g"], y.shape[0], o)
    cf.cfust_set_data(c, y)
    cf.cfust_set_params(c, params)
    return c


def _normal(params):
    P = {k: np.array(v, dtype=float) for k, v in params.items()}
    P["nu"] = np.full_like(P["nu"], np.inf)
    return P


PHI2_TAILS = ((-6.27, 7.12, -0.311), (7.1, -6.3, -0.5), (-8.0, -9.0, 0.6), (-6.0, 6.5, -0.95),
              (-30.0, -2.5, 0.93), (3.0, -2.6, -0.999), (-4.0, -4.0, 0.999))


def _logf_close(got, ref, tol):
    """Equal within tol where both are finite; a pair that is -inf (T_q = 0 in FP64, a
    null pair) on one side has log f below -700 (tau 0 in FP64) on the other."""
    fin = np.isfinite(got) & np.isfinite(ref)
    np.testing.assert_allclose(got[fin], ref[fin], rtol=tol, atol=tol)
    assert np.all(np.where(np.isneginf(got), ref < -700, True))
    assert np.all(np.where(np.isneginf(ref), got < -700, True))
    assert not np.any(np.isnan(got)) and not np.any(np.isposinf(got))


def _row_close(got, ref, rtol, axes=(-1,)):
    scale = np.abs(ref).max(axis=axes, keepdims=True)
    assert np.all(np.abs(got - ref) <= rtol * scale + 1e-12), f"worst {np.max(np.abs(got - ref) / (scale + 1e-12)):.3e}"


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_normal_integrators(cf, oracle, k):
    w = synth.make_workload("two_comp_p2", n=10, with_init=False)
    q = w["qmc"]
    ctx = cf.cfust_create(2, 2, 2, 10, cf.cfust_default_opts(qmc_points=q["npoints"], qmc_shifts=q["nshifts"],
                                                          qmc_korobov_a=q["korobov_a"], seed=q["seed"]))
    rng = np.random.default_rng(300 + k)
    cnt = 200 if k <= 2 else 16
    b = np.zeros((cnt, k))
    V = np.zeros((cnt, k, k))
    for i in range(cnt):
        A = rng.standard_normal((k, k))
        V[i] = A @ A.T + 0.3 * np.eye(k)
        b[i] = rng.normal(0.2, 1.3, k) * np.sqrt(np.diag(V[i]))
    if k == 2:  # far tails: both orientations of the rho = -1 bound, values far below 1e-100
        for h, kk, rho in PHI2_TAILS:
            b = np.vstack([b, [h, kk]])
            V = np.concatenate([V, [[[1.0, rho], [rho, 1.0]]]])
        cnt = len(b)
    nu = np.full(cnt, np.inf)
    got, _ = cf.cfust_tk_eval(ctx, b, V, nu)
    spec = oracle.qmc(**q)
    ref = np.array([oracle.tkcdf(b[i], V[i], math.inf, spec)[0] for i in range(cnt)])
    rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)
    print(f"Phi_{k}: worst relative error {rel.max():.2e}")
    np.testing.assert_allclose(got, ref, rtol=1e-9 if k == 2 else 1e-12)


@pytest.mark.parametrize("name,n,moments", [("two_comp_p2", 300, 0), ("flow_p4", 200, 1), ("flow_p4", 120, 0),
                                             ("wide_p16", 400, 0)])
def test_cfusn_estep_fp64(cf, oracle, name, n, moments):
    w = synth.make_workload(name, n=n)
    P = _normal(w["init"])
    c = _ctx(cf, w, P, moments=moments)
    L = cf.cfust_estep(c)
    g = cf.cfust_get_pairs(c)
    o = oracle.estep(w["y"], P, oracle.qmc(**dict(w["qmc"], moments=moments)))
    tol = 1e-9
    fin = np.isfinite(g["logf"]) & np.isfinite(o["logf"])
    print(f"{name} moments={moments}: worst log f error "
          f"{np.max(np.abs(g['logf'][fin] - o['logf'][fin]) / np.maximum(1, np.abs(o['logf'][fin]))):.2e}")
    _logf_close(g["logf"], o["logf"], tol)
    assert np.all(g["u"] == 1.0)
    live = np.isfinite(g["logf"]) & np.isfinite(o["logf"])  # null pairs: tau 0, moments unused
    _row_close(g["eu"][live], o["eu"][live], 1e-7)
    _row_close(g["euu"][live], o["euu"][live], 1e-7, axes=(-1, -2))
    assert abs(L - o["loglik"]) <= tol * abs(o["loglik"])
    got = cf.cfust_get_params(c)
    assert np.all(np.isinf(got["nu"]))


@pytest.mark.parametrize("precision", [1, 2])
def test_cfusn_estep_fp32(cf, oracle, precision):
    w = synth.make_workload("wide_p16", n=400)
    P = _normal(w["init"])
    c = _ctx(cf, w, P, precision=precision)
    L = cf.cfust_estep(c)
    o = oracle.estep(w["y"], P, oracle.qmc(**w["qmc"]))
    assert abs(L - o["loglik"]) <= 1e-6 * abs(o["loglik"])


def test_cfusn_fit(cf, oracle):
    w = synth.make_workload("two_comp_p2", n=400)
    P = _normal(w["init"])
    c = _ctx(cf, w, P)
    it, hist = cf.cfust_fit(c, 10)
    ref, rhist, rit = oracle.fit(w["y"], P, 10, oracle.qmc(**w["qmc"]), hold=oracle.HOLD_NU)
    assert it == rit == 10
    assert abs(hist[-1] - rhist[-1]) <= 1e-6 * abs(rhist[-1])
    got = cf.cfust_get_params(c)
    for k in ("pi", "mu", "Sigma", "Delta"):
        np.testing.assert_allclose(got[k], ref[k], rtol=1e-4, atol=1e-6, err_msg=k)
    assert np.all(np.isinf(got["nu"]))


def test_normal_mixture_fit(cf, oracle):
    """The normal mixture: CFUSN with Delta^(0) = 0 held (cfust_opts.hold =
    CFUST_HOLD_DELTA), against the oracle's held fit (pinned on the CPU against a
    textbook normal-mixture EM): final l 1e-9, parameters 1e-8."""
    w = synth.make_workload("flow_p4", n=600, with_init=False)
    y = np.ascontiguousarray(w["y"][:, :3])
    g, q = 2, 2
    lab = np.random.default_rng(9).integers(0, g, len(y))
    P = dict(pi=np.array([0.5, 0.5]), mu=np.array([y[lab == h].mean(0) for h in range(g)]),
             Sigma=np.array([np.cov(y[lab == h], rowvar=False) for h in range(g)]),
             Delta=np.zeros((g, 3, q)), nu=np.array([np.inf, np.inf]))
    qm = w["qmc"]
    o = cf.cfust_default_opts(qmc_points=qm["npoints"], qmc_shifts=qm["nshifts"], qmc_korobov_a=qm["korobov_a"],
                              seed=qm["seed"], model=cf.CFUST_MODEL_CFUSN, hold=cf.CFUST_HOLD_DELTA)
    c = cf.cfust_create(3, q, g, len(y), o)
    cf.cfust_set_data(c, y)
    cf.cfust_set_params(c, P)
    it, hist = cf.cfust_fit(c, 12)
    ref, rhist, rit = oracle.fit(y, P, 12, oracle.qmc(**qm), hold=oracle.HOLD_DELTA | oracle.HOLD_NU)
    assert it == rit == 12
    assert abs(hist[-1] - rhist[-1]) <= 1e-9 * abs(rhist[-1])
    got = cf.cfust_get_params(c)
    assert np.all(got["Delta"] == 0.0) and np.all(np.isinf(got["nu"]))
    for k in ("pi", "mu", "Sigma"):
        np.testing.assert_allclose(got[k], ref[k], rtol=1e-8, atol=1e-10, err_msg=k)
