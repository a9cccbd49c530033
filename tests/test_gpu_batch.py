"""GPU: the batched form (cfust_fit_batch) -- every fit of a batch captured as
one CUDA graph with its loop control on the device, all fits run concurrently.

Its results must equal those of the host-driven cfust_fit on the same inputs
bit for bit (same kernels, same order, deterministic reductions), including
the Aitken stopping iteration (eqs 24-26) and the failure paths; and a
batched fit must meet the oracle's fit tolerances (final l 1e-6 relative,
parameters 1e-4) like cfust_fit does.
"""
import numpy as np
import pytest

from paper_1606_02054_gb300 import synth

pytestmark = pytest.mark.gpu

KEYS = ("pi", "mu", "Sigma", "Delta", "nu")


@pytest.fixture(scope="module")
def cf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_02054_gb300 import build

    build.build()
    import paper_1606_02054_gb300 as cf

    return cf


@pytest.fixture(scope="module")
def batch():
    # ragged shapes: p = q in {2..8}, g in {2..6}, small n
    return synth.make_batch(nfits=6, starts=2, n_range=(150, 600))


def _ctx(cf, p, q, g, y, params, qmc, precision=0, moments=1):
    o = cf.cfust_default_opts(precision=precision, qmc_points=qmc["npoints"],
                              qmc_shifts=qmc["nshifts"], qmc_korobov_a=qmc["korobov_a"],
                              seed=qmc["seed"], moments=moments)
    c = cf.cfust_create(p, q, g, y.shape[0], o)
    cf.cfust_set_data(c, y)
    cf.cfust_set_params(c, params)
    return c


def _pairs(cf, batch, precision, moments=1):
    """Two contexts per (problem, start) with identical inputs."""
    out = []
    for f in batch["fits"]:
        for st in f["starts"]:
            a = _ctx(cf, f["p"], f["q"], f["g"], f["y"], st, batch["qmc"], precision, moments)
            b = _ctx(cf, f["p"], f["q"], f["g"], f["y"], st, batch["qmc"], precision, moments)
            out.append((a, b))
    return out


def _host_fit(cf, ctx, max_iter, tol):
    try:
        it, hist = cf.cfust_fit(ctx, max_iter, tol)
        return it, hist, cf.CFUST_OK
    except cf.CfustError as e:
        return None, None, e.status


@pytest.mark.parametrize("precision,tol,max_iter", [(0, 0.0, 5), (1, 0.0, 5), (2, 0.0, 5), (1, 0.1, 40)])
def test_batch_equals_host_loop(cf, batch, precision, tol, max_iter):
    pairs = _pairs(cf, batch, precision)
    iters, hist, status = cf.cfust_fit_batch([b for _, b in pairs], max_iter, tol)
    for i, (a, b) in enumerate(pairs):
        it, h, s = _host_fit(cf, a, max_iter, tol)
        assert status[i] == s, (i, cf.cfust_last_error(b))
        if s != cf.CFUST_OK:
            continue
        assert iters[i] == it
        np.testing.assert_array_equal(hist[i, : it + 1], h)
        assert np.all(np.isnan(hist[i, it + 1:]))
        pa, pb = cf.cfust_get_params(a), cf.cfust_get_params(b)
        for k in KEYS:
            np.testing.assert_array_equal(pb[k], pa[k], err_msg=k)
    if tol > 0:
        assert np.any(iters < max_iter), "the Aitken rule never fired; pick a larger tol"


def test_batch_repeat_continues_from_current_params(cf, batch):
    """A second call reuses the cached graph and continues from Psi^(K)."""
    f = batch["fits"][0]
    qmc = batch["qmc"]
    a = _ctx(cf, f["p"], f["q"], f["g"], f["y"], f["starts"][0], qmc, 1)
    b = _ctx(cf, f["p"], f["q"], f["g"], f["y"], f["starts"][0], qmc, 1)
    for _ in range(2):
        it, h = cf.cfust_fit(a, 3, 0.0)
        iters, hist, status = cf.cfust_fit_batch([b], 3, 0.0)
        assert status[0] == cf.CFUST_OK and iters[0] == it
        np.testing.assert_array_equal(hist[0], h)
    pa, pb = cf.cfust_get_params(a), cf.cfust_get_params(b)
    for k in KEYS:
        np.testing.assert_array_equal(pb[k], pa[k])


def test_batch_zero_iterations_is_one_density_pass(cf, batch):
    f = batch["fits"][1]
    c = _ctx(cf, f["p"], f["q"], f["g"], f["y"], f["starts"][0], batch["qmc"], 0)
    L = cf.cfust_loglik(c)
    iters, hist, status = cf.cfust_fit_batch([c], 0, 0.0)
    assert status[0] == cf.CFUST_OK and iters[0] == 0
    assert hist.shape == (1, 1) and hist[0, 0] == L


def test_batch_no_final_pass(cf, batch):
    f = batch["fits"][2]
    a = _ctx(cf, f["p"], f["q"], f["g"], f["y"], f["starts"][0], batch["qmc"], 1)
    b = _ctx(cf, f["p"], f["q"], f["g"], f["y"], f["starts"][0], batch["qmc"], 1)
    it, h = cf.cfust_fit(a, 4, 0.0)
    iters, hist, status = cf.cfust_fit_batch([b], 4, 0.0, flags=cf.CFUST_FIT_NO_FINAL)
    assert status[0] == cf.CFUST_OK and iters[0] == 4
    np.testing.assert_array_equal(hist[0, :4], h[:4])
    assert np.isnan(hist[0, 4])
    pa, pb = cf.cfust_get_params(a), cf.cfust_get_params(b)
    for k in KEYS:
        np.testing.assert_array_equal(pb[k], pa[k])


def test_batch_empty_component_keeps_last_good_params(cf):
    """A component far from every observation gets sum tau = 0 (its densities
    underflow): the first M-step fails with CFUST_EEMPTY, exactly as in the
    host loop, and Psi^(0) is kept."""
    w = synth.make_workload("two_comp_p2", n=300)
    params = {k: np.array(v, dtype=float) for k, v in w["init"].items()}
    params["mu"][1] = [1.0e3, 1.0e3]
    params["nu"][1] = 200.0
    params["Sigma"][1] = np.eye(2)
    params["Delta"][1] = 0.0  # keeps T_q finite: log f_2 ~ -930, tau_2 = 0 in FP64
    params["pi"] = np.array([0.99, 0.01])
    qmc = w["qmc"]
    a = _ctx(cf, 2, 2, 2, w["y"], params, qmc, 0)
    b = _ctx(cf, 2, 2, 2, w["y"], params, qmc, 0)
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_fit(a, 5, 0.0)
    assert e.value.status == cf.CFUST_EEMPTY
    ok = _ctx(cf, 2, 2, 2, w["y"], w["init"], qmc, 0)
    iters, hist, status = cf.cfust_fit_batch([ok, b], 5, 0.0)
    assert status[0] == cf.CFUST_OK and iters[0] == 5
    assert status[1] == cf.CFUST_EEMPTY and iters[1] == 0
    assert "component 1" in cf.cfust_last_error(b)
    assert np.isfinite(hist[1, 0]) and np.all(np.isnan(hist[1, 1:]))
    pb = cf.cfust_get_params(b)
    for k in KEYS:
        np.testing.assert_array_equal(pb[k], params[k])


def test_batch_fit_matches_oracle(cf, oracle):
    """A batched fit of a ragged batch against the oracle's fits (FP64, same
    lattice): final l <= 1e-6 relative, parameters <= 1e-4."""
    b = synth.make_batch(nfits=3, starts=1, n_range=(120, 250), p_range=(2, 4), g_range=(2, 3))
    qmc = b["qmc"]
    oq = oracle.qmc(qmc["npoints"], qmc["nshifts"], qmc["korobov_a"], qmc["seed"], moments=1)
    ctxs, refs = [], []
    for f in b["fits"]:
        st = f["starts"][0]
        ctxs.append(_ctx(cf, f["p"], f["q"], f["g"], f["y"], st, qmc, 0))
        rp, rh, _ = oracle.fit(f["y"], st, 6, oq)
        refs.append((rh, rp))
    iters, hist, status = cf.cfust_fit_batch(ctxs, 6, 0.0)
    assert np.all(status == cf.CFUST_OK)
    for i, c in enumerate(ctxs):
        rh, rp = refs[i]
        assert abs(hist[i, -1] - rh[-1]) <= 1e-6 * abs(rh[-1])
        got = cf.cfust_get_params(c)
        for k in KEYS:
            np.testing.assert_allclose(got[k], rp[k], rtol=1e-4, atol=1e-6, err_msg=k)


def test_batch_rejects_duplicates_and_bad_args(cf, batch):
    f = batch["fits"][0]
    c = _ctx(cf, f["p"], f["q"], f["g"], f["y"], f["starts"][0], batch["qmc"], 0)
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_fit_batch([c, c], 2, 0.0)
    assert e.value.status == cf.CFUST_EINVAL
    with pytest.raises(cf.CfustError):
        cf.cfust_fit_batch([c], -1, 0.0)
    with pytest.raises(cf.CfustError):
        cf.cfust_fit_batch([c], 2, 0.0, flags=8)
