"""GPU parity of the single-pass moment reading (opts.moments = 1): the CUDA
ratio estimators against the oracle's, on the same lattice points."""
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


def _ctx(cf, w, params, precision=0, y=None):
    y = w["y"] if y is None else y
    q = w["qmc"]
    opts = cf.cfust_default_opts(precision=precision, qmc_points=q["npoints"],
                                 qmc_shifts=q["nshifts"], qmc_korobov_a=q["korobov_a"],
                                 seed=q["seed"], moments=1)
    ctx = cf.cfust_create(w["p"], w["q"], w["g"], y.shape[0], opts)
    cf.cfust_set_data(ctx, y)
    cf.cfust_set_params(ctx, params)
    return ctx


def _spec(oracle, w):
    return oracle.qmc(**dict(w["qmc"], moments=1))


def _row_close(got, ref, rtol, atol=1e-10, axes=(-1,)):
    scale = np.abs(ref).max(axis=axes, keepdims=True)
    err = np.abs(got - ref)
    assert np.all(err <= rtol * scale + atol), f"worst {np.max(err / (scale + atol)):.3e}"


@pytest.fixture(scope="module")
def flow_small():
    return synth.make_workload("flow_p4", n=300)


def test_single_pass_fp64(cf, oracle, flow_small):
    w = flow_small
    ctx = _ctx(cf, w, w["init"])
    L = cf.cfust_estep(ctx)
    g = cf.cfust_get_pairs(ctx)
    o = oracle.estep(w["y"], w["init"], _spec(oracle, w))
    np.testing.assert_allclose(g["logf"], o["logf"], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(g["u"], o["u"], rtol=1e-8, atol=1e-12)
    _row_close(g["eu"], o["eu"], 1e-8)
    _row_close(g["euu"], o["euu"], 1e-8, axes=(-1, -2))
    assert abs(L - o["loglik"]) <= 1e-10 * abs(o["loglik"])
    # a weighted covariance of lattice draws: PSD for every pair
    C = g["u"][..., None, None] * g["euu"] - np.einsum("hja,hjb->hjab", g["eu"], g["eu"])
    ev = np.linalg.eigvalsh(C)
    assert np.all(ev.min(-1) >= -1e-9 * np.abs(C).max(axis=(-1, -2)))


def test_single_pass_fp32(cf, oracle, flow_small):
    w = flow_small
    ctx = _ctx(cf, w, w["init"], precision=1)
    L = cf.cfust_estep(ctx)
    g = cf.cfust_get_pairs(ctx)
    o = oracle.estep(w["y"], w["init"], _spec(oracle, w))
    assert abs(L - o["loglik"]) <= 1e-6 * abs(o["loglik"])
    np.testing.assert_allclose(g["u"], o["u"], rtol=1e-4)
    _row_close(g["eu"], o["eu"], 2e-4)
    _row_close(g["euu"], o["euu"], 2e-4, axes=(-1, -2))


def test_single_pass_fit_fp64(cf, oracle, flow_small):
    w = flow_small
    iters = 8
    ctx = _ctx(cf, w, w["init"])
    it, hist = cf.cfust_fit(ctx, iters)
    got = cf.cfust_get_params(ctx)
    ref, rhist, _ = oracle.fit(w["y"], w["init"], iters, _spec(oracle, w))
    assert abs(hist[-1] - rhist[-1]) <= 1e-6 * abs(rhist[-1])
    for k in ("pi", "mu", "Sigma", "Delta", "nu"):
        np.testing.assert_allclose(got[k], ref[k], rtol=1e-4, atol=1e-6)


@pytest.mark.parametrize("p,q,g,n", [(3, 3, 2, 33), (5, 5, 2, 9), (8, 7, 1, 4), (8, 8, 1, 3)])
def test_single_pass_shapes_fp64(cf, oracle, p, q, g, n):
    rng = np.random.default_rng(2000 + 97 * p + 13 * q + g)
    params = synth.draw_params(rng, p, q, g, delta_sd=0.8)
    y, _ = synth.sample(rng, n, params)
    w = dict(p=p, q=q, g=g, n=n, y=y, qmc=synth.qmc_settings(2, npoints=256, nshifts=4))
    ctx = _ctx(cf, w, params)
    L = cf.cfust_estep(ctx)
    gp = cf.cfust_get_pairs(ctx)
    o = oracle.estep(y, params, _spec(oracle, w))
    np.testing.assert_allclose(gp["logf"], o["logf"], rtol=1e-9, atol=1e-9)
    _row_close(gp["eu"], o["eu"], 1e-8)
    _row_close(gp["euu"], o["euu"], 1e-8, axes=(-1, -2))
    assert abs(L - o["loglik"]) <= 1e-10 * abs(o["loglik"])


@pytest.mark.parametrize("p,q,g,n", [(5, 5, 2, 40), (7, 6, 2, 24), (8, 7, 2, 24), (8, 8, 2, 20)])
def test_single_pass_shapes_fp32(cf, oracle, p, q, g, n):
    """FP32 moment kernels of every record dimension up to 8 (K = 7, 8 run in 4-warp
    blocks) against the FP64 oracle on the same lattice: FP32 bounds."""
    rng = np.random.default_rng(3000 + 97 * p + 13 * q + g)
    params = synth.draw_params(rng, p, q, g, delta_sd=0.8)
    y, _ = synth.sample(rng, n, params)
    w = dict(p=p, q=q, g=g, n=n, y=y, qmc=synth.qmc_settings(2))
    ctx = _ctx(cf, w, params, precision=1)
    L = cf.cfust_estep(ctx)
    gp = cf.cfust_get_pairs(ctx)
    o = oracle.estep(y, params, _spec(oracle, w))
    assert abs(L - o["loglik"]) <= 1e-6 * abs(o["loglik"])
    np.testing.assert_allclose(gp["u"], o["u"], rtol=2e-4)
    _row_close(gp["eu"], o["eu"], 5e-4)
    _row_close(gp["euu"], o["euu"], 5e-4, axes=(-1, -2))
