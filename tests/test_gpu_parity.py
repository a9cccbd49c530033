"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on
the same seeded inputs and the same lattice.

Tolerances:
  FP64 mode, q <= 2 (T_q deterministic): per-pair log-density
      |diff| <= 1e-9 max(1, |ref|); other per-pair quantities 1e-9 relative.
  FP64 mode, q >= 3: both sides evaluate the same lattice points, so they
      agree far inside 3 standard errors; asserted at 1e-8 relative.
  FP32 mode: |alpha_s diff| <= 3 SE + 5e-5 alpha_s (FP32 rounding of the
      lattice products and of the T_2 quadrature).
  Fits: final log-likelihood relative error <= 1e-6, parameters <= 1e-4
      after the same iteration count.
"""
import math

import numpy as np
import pytest
import scipy.special as sp
import scipy.stats as st

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


def _opts(cf, w, precision=0, **kw):
    q = w["qmc"]
    return cf.cfust_default_opts(precision=precision, qmc_points=q["npoints"],
                                 qmc_shifts=q["nshifts"], qmc_korobov_a=q["korobov_a"],
                                 seed=q["seed"], **kw)


def _ctx(cf, w, params, precision=0, y=None, **kw):
    y = w["y"] if y is None else y
    ctx = cf.cfust_create(w["p"], w["q"], w["g"], y.shape[0], _opts(cf, w, precision, **kw))
    cf.cfust_set_data(ctx, y)
    cf.cfust_set_params(ctx, params)
    return ctx


def _close(a, b, rtol, atol=0.0):
    a, b = np.asarray(a), np.asarray(b)
    err = np.abs(a - b)
    lim = rtol * np.abs(b) + atol
    bad = err > lim
    assert not bad.any(), f"max err {err.max():.3e} (worst rel {np.max(err / (np.abs(b) + 1e-300)):.3e}) at {np.argwhere(bad)[:5].tolist()}"


def _compare_pairs(g, o, rtol=1e-9, q=None):
    _close(g["logf"], o["logf"], rtol, rtol)      # |d| <= rtol max(1,|ref|) (approx.)
    _close(g["tau"], o["tau"], 0.0, rtol)
    _close(g["u"], o["u"], rtol, 1e-12)
    _close(g["elogu"], o["elogu"], rtol, rtol)
    _close(g["eu"], o["eu"], rtol, 1e-11)
    _close(g["euu"], o["euu"], rtol, 1e-11)


# ---------------------------------------------------------------------------
# integrators
# ---------------------------------------------------------------------------
def _rand_cases(rng, k, count, nu_lo=3.0, nu_hi=40.0):
    b = np.zeros((count, k))
    V = np.zeros((count, k, k))
    nu = rng.uniform(nu_lo, nu_hi, count)
    for i in range(count):
        A = rng.standard_normal((k, k))
        V[i] = A @ A.T + 0.3 * np.eye(k)
        b[i] = rng.normal(0.2, 1.3, k) * np.sqrt(np.diag(V[i]))
    return b, V, nu


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7, 8])
def test_tk_integrators_fp64(cf, oracle, k):
    w = synth.make_workload("two_comp_p2", n=10, with_init=False)
    ctx = cf.cfust_create(2, 2, 2, 10, _opts(cf, w, 0))
    rng = np.random.default_rng(100 + k)
    b, V, nu = _rand_cases(rng, k, 24 if k >= 3 else 200)
    got, gse = cf.cfust_tk_eval(ctx, b, V, nu)
    spec = oracle.qmc(**w["qmc"])
    ref = np.array([oracle.tkcdf(b[i], V[i], nu[i], spec)[0] for i in range(len(nu))])
    rse = np.array([oracle.tkcdf(b[i], V[i], nu[i], spec)[1] for i in range(len(nu))]) if k >= 3 else None
    _close(got, ref, 1e-12 if k == 1 else (2e-10 if k == 2 else 1e-9))
    if k >= 3:
        _close(gse, rse, 1e-6, 1e-15)


@pytest.mark.parametrize("k", [1, 2, 4])
def test_tk_integrators_fp32(cf, oracle, k):
    w = synth.make_workload("two_comp_p2", n=10, with_init=False)
    ctx = cf.cfust_create(2, 2, 2, 10, _opts(cf, w, 1))
    rng = np.random.default_rng(200 + k)
    b, V, nu = _rand_cases(rng, k, 24 if k >= 3 else 200)
    got, gse = cf.cfust_tk_eval(ctx, b, V, nu)
    spec = oracle.qmc(**w["qmc"])
    res = [oracle.tkcdf(b[i], V[i], nu[i], spec) for i in range(len(nu))]
    ref = np.array([r[0] for r in res])
    se = np.array([r[1] for r in res])
    err = np.abs(got - ref)
    lim = 3 * se + 5e-5 * ref + 1e-12
    assert np.all(err <= lim), f"worst rel err {np.max(err / ref):.3e}, worst err/lim {np.max(err / lim):.3f}"


def test_tk_integrator_edge_cases(cf, oracle):
    w = synth.make_workload("two_comp_p2", n=10, with_init=False)
    ctx = cf.cfust_create(2, 2, 2, 10, _opts(cf, w, 0))
    # orthant of an equicorrelated (rho = 1/2) law: 1/(k+1); identity & b=0: 2^-k
    for k in (3, 4, 6):
        R = np.full((k, k), 0.5) + 0.5 * np.eye(k)
        v, s = cf.cfust_tk_eval(ctx, np.zeros((1, k)), R[None], [7.0])
        assert abs(v[0] - 1 / (k + 1)) < 4 * s[0] + 1e-9
        v, s = cf.cfust_tk_eval(ctx, np.zeros((1, k)), np.eye(k)[None], [7.0])
        assert v[0] == 2.0 ** -k and s[0] == 0.0
    # strong correlations in T_2 (graded nodes) and far tails
    cases = [(-3.0, -3.0, 0.999, 5.0), (2.0, -2.0, -0.9999, 7.0), (-8.0, -7.0, 0.5, 6.0),
             (-20.0, 3.0, 0.3, 9.0), (0.0, 0.0, 0.0, 4.0)]
    for h, kk, rho, nu in cases:
        V = np.array([[1.0, rho], [rho, 1.0]])
        v, _ = cf.cfust_tk_eval(ctx, np.array([[h, kk]]), V[None], [nu])
        ref = oracle.t2cdf(h, kk, rho, nu)
        assert abs(v[0] - ref) <= 1e-9 * ref, (h, kk, rho, nu, v[0], ref)


def test_t2_fp32_edge_cases(cf, oracle):
    """FP32 T_2 (quadrature with the tabulated inner T_1) at strong correlations
    on both sides of the node-grading threshold |rho| = 0.99, far tails down to
    ~1e-20, and dofs from 1.5 to 200: FP32 bound 5e-5 relative."""
    w = synth.make_workload("two_comp_p2", n=10, with_init=False)
    ctx = cf.cfust_create(2, 2, 2, 10, _opts(cf, w, 1))
    cases = [(-3.0, -3.0, 0.999, 5.0), (2.0, -2.0, -0.9999, 7.0), (-8.0, -7.0, 0.5, 6.0),
             (-20.0, 3.0, 0.3, 9.0), (0.0, 0.0, 0.0, 4.0), (-6.0, -6.0, 0.95, 200.0),
             (1.5, 0.5, 0.985, 1.5), (-30.0, -30.0, 0.2, 2.5), (0.3, -0.2, -0.989, 30.0),
             (-4.0, 6.0, -0.7, 60.0), (5.0, 5.0, 0.1, 3.0), (-12.0, -9.0, 0.9, 15.0),
             (-10.0, -10.0, 0.5, 60.0), (-14.0, -12.0, 0.3, 40.0)]
    b = np.array([[h, kk] for h, kk, _, _ in cases])
    V = np.array([[[1.0, r], [r, 1.0]] for _, _, r, _ in cases])
    nu = np.array([c[3] for c in cases])
    got, _ = cf.cfust_tk_eval(ctx, b, V, nu)
    ref = np.array([oracle.t2cdf(h, kk, r, v) for h, kk, r, v in cases])
    rel = np.abs(got - ref) / ref
    assert np.all(rel <= 5e-5), list(zip(cases, rel))


def test_t2_fp32_piece_classes(cf, oracle):
    """FP32 T_2 where each quadrature piece takes 8 to 32 nodes by its class (4 <= dof
    <= 64, |rho| < 0.9): the region's edges, lower tails of h down to T_1 = 1e-12 (short
    pieces that end at phi = 0, where the dof caps of the small classes hold) and h up
    to 12 (long pieces at large dof, which take 32 nodes).  The FP32 bound 5e-5 relative
    holds wherever T_2 > 1e-12."""
    from scipy.special import stdtrit
    w = synth.make_workload("two_comp_p2", n=10, with_init=False)
    ctx = cf.cfust_create(2, 2, 2, 10, _opts(cf, w, 1))
    rng = np.random.default_rng(2424)
    n = 600
    edge_nu = [4.0, 4.0, 64.0, 64.0, 3.99, 64.5, 20.0, 40.0]
    edge_rho = [0.899, -0.899, 0.899, -0.899, 0.5, -0.5, 0.3, -0.3]
    nu = np.concatenate([edge_nu, np.exp(rng.uniform(np.log(4.0), np.log(64.0), n - 8))])
    rho = np.concatenate([edge_rho, rng.uniform(-0.9, 0.9, n - 8)])
    b = rng.uniform(-8.0, 8.0, (n, 2))
    tail = rng.uniform(size=n) < 0.3
    b[tail, 0] = stdtrit(nu[tail], 10.0 ** rng.uniform(-12.0, -3.0, tail.sum()))
    far = rng.uniform(size=n) < 0.15
    b[far, 0] = rng.uniform(4.0, 12.0, far.sum())
    V = np.array([[[1.0, r], [r, 1.0]] for r in rho])
    got, _ = cf.cfust_tk_eval(ctx, b, V, nu)
    ref = np.array([oracle.t2cdf(b[i, 0], b[i, 1], rho[i], nu[i]) for i in range(n)])
    keep = ref > 1e-12
    rel = np.abs(got - ref)[keep] / ref[keep]
    print(f"T_2 piece classes: worst rel err {rel.max():.3e} over {keep.sum()} cases")
    assert keep.sum() > n // 2 and np.all(rel <= 5e-5), f"worst rel err {rel.max():.3e}"


# ---------------------------------------------------------------------------
# E-step, M-step, fit
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def two_comp():
    return synth.make_workload("two_comp_p2")


def test_estep_two_comp_fp64(cf, oracle, two_comp):
    w = two_comp
    ctx = _ctx(cf, w, w["init"])
    L = cf.cfust_estep(ctx)
    g = cf.cfust_get_pairs(ctx)
    o = oracle.estep(w["y"], w["init"], oracle.qmc(**w["qmc"]))
    _compare_pairs(g, o, 1e-9)
    assert abs(L - o["loglik"]) <= 1e-11 * abs(o["loglik"])
    assert np.all(g["se"] == 0.0)


def test_stats_match_sums_of_oracle_pairs(cf, oracle, two_comp):
    w = two_comp
    ctx = _ctx(cf, w, w["init"])
    cf.cfust_estep(ctx)
    S = cf.cfust_get_stats(ctx)
    o = oracle.estep(w["y"], w["init"], oracle.qmc(**w["qmc"]))
    p, q = w["p"], w["q"]
    for h in range(w["g"]):
        t, u = o["tau"][h], o["u"][h]
        r = w["y"] - w["init"]["mu"][h]
        ref = np.concatenate([[t.sum(), (t * u).sum(), (t * (o["elogu"][h] - u)).sum()],
                              (t * u) @ r, t @ o["eu"][h],
                              np.einsum("j,ja,jb->ab", t, r, o["eu"][h]).ravel(),
                              np.einsum("j,jab->ab", t, o["euu"][h]).ravel(),
                              np.einsum("j,ja,jb->ab", t * u, r, r).ravel()])
        _close(S[h], ref, 1e-9, 1e-9)


def test_mstep_two_comp(cf, oracle, two_comp):
    w = two_comp
    ctx = _ctx(cf, w, w["init"])
    cf.cfust_estep(ctx)
    cf.cfust_mstep(ctx)
    got = cf.cfust_get_params(ctx)
    o = oracle.estep(w["y"], w["init"], oracle.qmc(**w["qmc"]))
    ref, _ = oracle.mstep(w["y"], o, w["init"])
    for k in ("pi", "mu", "Sigma", "Delta", "nu"):
        _close(got[k], ref[k], 1e-8, 1e-10)


def test_fit_two_comp_fp64(cf, oracle, two_comp):
    w = two_comp
    iters = w["iters"]
    ctx = _ctx(cf, w, w["init"])
    it, hist = cf.cfust_fit(ctx, iters)
    got = cf.cfust_get_params(ctx)
    ref, rhist, rit = oracle.fit(w["y"], w["init"], iters, oracle.qmc(**w["qmc"]))
    assert it == rit == iters
    assert abs(hist[-1] - rhist[-1]) <= 1e-6 * abs(rhist[-1])
    _close(hist, rhist, 1e-6)
    for k in ("pi", "mu", "Sigma", "Delta", "nu"):
        _close(got[k], ref[k], 1e-4, 1e-6)


def test_fit_aitken_stop(cf, oracle, two_comp):
    # this fit converges slowly (ratio ~0.98), so |l_inf - l| falls below 0.5
    # only after ~80 iterations; both sides must stop at the same iteration
    w = two_comp
    ctx = _ctx(cf, w, w["init"])
    it, hist = cf.cfust_fit(ctx, 200, 0.5)
    _, rhist, rit = oracle.fit(w["y"], w["init"], 200, oracle.qmc(**w["qmc"]), tol=0.5)
    assert it == rit and 2 < it < 200
    _close(hist, rhist, 1e-7)


@pytest.fixture(scope="module")
def flow_small():
    return synth.make_workload("flow_p4", n=300)


def test_estep_flow_p4_fp64(cf, oracle, flow_small):
    w = flow_small
    ctx = _ctx(cf, w, w["init"])
    L = cf.cfust_estep(ctx)
    g = cf.cfust_get_pairs(ctx)
    o = oracle.estep(w["y"], w["init"], oracle.qmc(**w["qmc"]))
    _close(g["logf"], o["logf"], 1e-9, 1e-9)
    _close(g["se"], o["se"], 1e-6, 1e-15)
    _close(g["tau"], o["tau"], 0.0, 1e-9)
    _close(g["u"], o["u"], 1e-8, 1e-12)
    # eu, euu combine many integrals; same lattice points on both sides
    scale = np.abs(o["euu"]).max(axis=(-1, -2), keepdims=True)
    assert np.all(np.abs(g["euu"] - o["euu"]) <= 1e-7 * scale + 1e-10)
    scale = np.abs(o["eu"]).max(axis=-1, keepdims=True)
    assert np.all(np.abs(g["eu"] - o["eu"]) <= 1e-7 * scale + 1e-10)
    assert abs(L - o["loglik"]) <= 1e-10 * abs(o["loglik"])


def _alpha_s(w, params, logf):
    q = w["q"]
    out = np.zeros_like(logf)
    for h in range(w["g"]):
        Om = params["Sigma"][h] + params["Delta"][h] @ params["Delta"][h].T
        ltp = st.multivariate_t(loc=params["mu"][h], shape=Om, df=params["nu"][h]).logpdf(w["y"])
        out[h] = np.exp(logf[h] - q * math.log(2) - ltp)
    return out


def test_estep_flow_p4_fp32(cf, oracle, flow_small):
    w = flow_small
    ctx = _ctx(cf, w, w["init"], precision=1)
    L = cf.cfust_estep(ctx)
    g = cf.cfust_get_pairs(ctx)
    o = oracle.estep(w["y"], w["init"], oracle.qmc(**w["qmc"]))
    a_ref = _alpha_s(w, w["init"], o["logf"])
    a_got = _alpha_s(w, w["init"], g["logf"])
    assert np.all(np.abs(a_got - a_ref) <= 3 * o["se"] + 5e-5 * a_ref + 1e-300)
    assert abs(L - o["loglik"]) <= 1e-6 * abs(o["loglik"])


def test_fit_flow_p4_fp64(cf, oracle, flow_small):
    w = flow_small
    iters = 8
    ctx = _ctx(cf, w, w["init"])
    it, hist = cf.cfust_fit(ctx, iters)
    got = cf.cfust_get_params(ctx)
    ref, rhist, _ = oracle.fit(w["y"], w["init"], iters, oracle.qmc(**w["qmc"]))
    assert abs(hist[-1] - rhist[-1]) <= 1e-6 * abs(rhist[-1])
    for k in ("pi", "mu", "Sigma", "Delta", "nu"):
        _close(got[k], ref[k], 1e-4, 1e-6)


def test_full_size_flow_p4_sampled(cf, oracle):
    """The benchmarked configuration (n = 200,000, FP32 integrals): sampled
    pairs against the oracle, and the eq (27) identity at full size."""
    w = synth.make_workload("flow_p4")
    ctx = _ctx(cf, w, w["init"], precision=1)
    L = cf.cfust_estep(ctx)
    g = cf.cfust_get_pairs(ctx)
    lse = sp.logsumexp(np.log(w["init"]["pi"])[:, None] + g["logf"], axis=0)
    assert abs(lse.sum() - L) <= 1e-9 * abs(L)
    assert np.allclose(g["tau"].sum(0), 1.0, atol=1e-12)
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(w["n"], 40, replace=False))
    idx = np.concatenate([[0, w["n"] - 1], idx])
    sub = dict(w, y=w["y"][idx], n=len(idx))
    o = oracle.estep(sub["y"], w["init"], oracle.qmc(**w["qmc"]))
    a_ref = _alpha_s(sub, w["init"], o["logf"])
    a_got = _alpha_s(sub, w["init"], g["logf"][:, idx])
    assert np.all(np.abs(a_got - a_ref) <= 3 * o["se"] + 5e-5 * a_ref + 1e-300)


@pytest.mark.parametrize("p,q,g,n", [(1, 1, 1, 1), (3, 1, 2, 257), (3, 3, 2, 33), (5, 5, 2, 9),
                                     (8, 8, 1, 3), (6, 2, 3, 70), (2, 2, 16, 5)])
def test_estep_shapes_fp64(cf, oracle, p, q, g, n):
    rng = np.random.default_rng(1000 + 97 * p + 13 * q + g)
    params = synth.draw_params(rng, p, q, g, delta_sd=0.8)
    y, _ = synth.sample(rng, n, params)
    w = dict(p=p, q=q, g=g, n=n, y=y, qmc=synth.qmc_settings(2, npoints=256, nshifts=4))
    ctx = _ctx(cf, w, params)
    L = cf.cfust_estep(ctx)
    gp = cf.cfust_get_pairs(ctx)
    o = oracle.estep(y, params, oracle.qmc(**w["qmc"]))
    _close(gp["logf"], o["logf"], 1e-9, 1e-9)
    _close(gp["u"], o["u"], 1e-8, 1e-12)
    scale = np.abs(o["euu"]).max(axis=(-1, -2), keepdims=True)
    assert np.all(np.abs(gp["euu"] - o["euu"]) <= 1e-7 * scale + 1e-10)
    assert abs(L - o["loglik"]) <= 1e-10 * abs(o["loglik"])
    assert abs(cf.cfust_loglik(ctx) - L) <= 1e-12 * abs(L)


@pytest.mark.parametrize("moments", [0, 1])
def test_fp32_far_tail_pairs_use_fp64(cf, oracle, moments):
    # an observation far on the wrong side of the skewing directions makes
    # alpha_s tiny; the FP32 mode recomputes such pairs in FP64 (in the single-pass
    # form with the shared pass of alpha_s weighted to dof nu+p+2, as the FP64 mode)
    p = q = 3
    params = dict(pi=[1.0], mu=[np.zeros(3)], Sigma=[0.3 * np.eye(3)],
                  Delta=[3.0 * np.eye(3)], nu=[30.0])
    y = np.array([[-40.0, -40.0, -40.0], [0.5, 0.2, 0.1]])
    w = dict(p=p, q=q, g=1, n=2, y=y, qmc=synth.qmc_settings(2))
    c32 = _ctx(cf, w, params, precision=1, moments=moments)
    c64 = _ctx(cf, w, params, precision=0, moments=moments)
    cf.cfust_estep(c32)
    cf.cfust_estep(c64)
    g32, g64 = cf.cfust_get_pairs(c32), cf.cfust_get_pairs(c64)
    o = oracle.estep(y, params, oracle.qmc(**dict(w["qmc"], moments=moments)))
    assert o["logf"][0, 0] < -100
    _close(g32["logf"][0, 0], g64["logf"][0, 0], 1e-12)
    _close(g64["logf"], o["logf"], 1e-9, 1e-9)
    # the far pair's E-step values: FP32-mode fix-up (FP64) against the FP64 mode
    _close(g32["u"][0, 0], g64["u"][0, 0], 1e-10)
    _close(g32["eu"][0, 0], g64["eu"][0, 0], 1e-9, 1e-9 * np.abs(g64["eu"][0, 0]).max())
    _close(g32["euu"][0, 0], g64["euu"][0, 0], 1e-9, 1e-9 * np.abs(g64["euu"][0, 0]).max())
    _close(g64["u"][0, 0], o["u"][0, 0], 1e-8)


def test_determinism(cf, flow_small):
    w = flow_small
    ctx = _ctx(cf, w, w["init"], precision=1)
    L1 = cf.cfust_estep(ctx)
    S1 = cf.cfust_get_stats(ctx)
    L2 = cf.cfust_estep(ctx)
    S2 = cf.cfust_get_stats(ctx)
    assert L1 == L2 and np.array_equal(S1, S2)


def test_error_paths(cf, two_comp):
    w = two_comp
    ctx = cf.cfust_create(2, 2, 2, w["n"], _opts(cf, w))
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_estep(ctx)
    assert e.value.status == cf.CFUST_ESTATE
    cf.cfust_set_data(ctx, w["y"])
    bad = {k: np.array(v, dtype=float) for k, v in w["init"].items()}
    bad["nu"] = np.array([0.5, 10.0])
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_set_params(ctx, bad)
    assert e.value.status == cf.CFUST_EINVAL
    bad = {k: np.array(v, dtype=float) for k, v in w["init"].items()}
    bad["Sigma"][1] = np.array([[1.0, 2.0], [2.0, 1.0]])
    bad["Delta"][1] = 0.0
    cf.cfust_set_params(ctx, bad)
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_estep(ctx)
    assert e.value.status == cf.CFUST_ENOTPD
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_mstep(ctx)
    assert e.value.status == cf.CFUST_ESTATE


def test_device_resident_input(cf, oracle, two_comp):
    import torch

    w = two_comp
    yt = torch.tensor(w["y"], dtype=torch.float32, device="cuda")
    ctx = cf.cfust_create(2, 2, 2, w["n"], _opts(cf, w))
    cf.cfust_set_data(ctx, yt)
    cf.cfust_set_params(ctx, w["init"])
    L = cf.cfust_estep(ctx)
    o = oracle.estep(w["y"].astype(np.float32).astype(np.float64), w["init"], oracle.qmc(**w["qmc"]))
    assert abs(L - o["loglik"]) <= 1e-11 * abs(o["loglik"])
