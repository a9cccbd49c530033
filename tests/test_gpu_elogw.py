"""GPU: the exact E[log W | y] (opts.elogw = CFUST_ELOGW_EXACT) in place of the
one-step-late eq (15) of Sec. 3.1: the f-weighted mean of log W over the points of
the single-pass lattice pass of alpha_s, against the oracle's estimator on the same
points (pinned on the CPU against the tilted-Gamma integral in
tests/test_oracle_estep.py).

Tolerances: FP64 per pair 1e-9 (log W's mean over the same points); FP32 integrals
2e-5 absolute (log s^2 and the weights in FP32 over 8192 points); the other E-step
outputs are those of the OSL reading bit for bit (FP64); 10-iteration fits: final l
1e-6 relative, parameters 1e-4, and nu moves away from the OSL fit's."""
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


def _ctx(cf, w, precision, elogw, moments=1, n=None):
    q = w["qmc"]
    o = cf.cfust_default_opts(precision=precision, qmc_points=q["npoints"], qmc_shifts=q["nshifts"],
                              qmc_korobov_a=q["korobov_a"], seed=q["seed"], moments=moments, elogw=elogw)
    y = w["y"] if n is None else w["y"][:n]
    c = cf.cfust_create(w["p"], w["q"], w["g"], y.shape[0], o)
    cf.cfust_set_data(c, y)
    cf.cfust_set_params(c, w["init"])
    return c


@pytest.mark.parametrize("name,n", [("flow_p4", 300), ("learned_p6", 60)])
def test_exact_elogw_pairs(cf, oracle, name, n):
    w = synth.make_workload(name, n=n)
    spec = oracle.qmc(**dict(w["qmc"], moments=1, elogw=1))
    o = oracle.estep(w["y"], w["init"], spec)
    c64 = _ctx(cf, w, 0, 1)
    L = cf.cfust_estep(c64)
    g = cf.cfust_get_pairs(c64)
    np.testing.assert_allclose(g["elogu"], o["elogu"], rtol=1e-9, atol=1e-9)
    assert abs(L - o["loglik"]) <= 1e-10 * abs(o["loglik"])
    # everything but E[log W] is the OSL reading's, bit for bit
    osl = _ctx(cf, w, 0, 0)
    assert cf.cfust_estep(osl) == L
    go = cf.cfust_get_pairs(osl)
    for k in ("logf", "u", "eu", "euu", "tau"):
        assert np.array_equal(go[k], g[k]), k
    assert np.max(np.abs(go["elogu"] - g["elogu"])) > 1e-4  # the readings differ
    # FP32 integrals
    c32 = _ctx(cf, w, 1, 1)
    cf.cfust_estep(c32)
    g32 = cf.cfust_get_pairs(c32)
    live = np.isfinite(o["logf"])
    err = np.abs(g32["elogu"] - o["elogu"])[live]
    print(f"{name}: FP32 exact E[log W] worst abs err {err.max():.2e}")
    assert err.max() <= 2e-5


@pytest.mark.parametrize("precision", [1, 2])
def test_exact_elogw_fit(cf, oracle, precision):
    w = synth.make_workload("flow_p4", n=600)
    y = w["y"].astype(np.float32) if precision == 2 else w["y"]
    iters = 10
    c = _ctx(cf, dict(w, y=y), precision, 1)
    _, hist = cf.cfust_fit(c, iters)
    got = cf.cfust_get_params(c)
    ref, rhist, _ = oracle.fit(y.astype(np.float64), w["init"], iters,
                               oracle.qmc(**dict(w["qmc"], moments=1, elogw=1)))
    rel = abs(hist[-1] - rhist[-1]) / abs(rhist[-1])
    perr = max(float(np.linalg.norm(np.atleast_1d(got[k][h] - ref[k][h])) / np.linalg.norm(np.atleast_1d(ref[k][h])))
               for k in ("pi", "mu", "Sigma", "Delta", "nu") for h in range(w["g"]))
    print(f"exact E[log W] fit, precision {precision}: l rel err {rel:.2e}, parameters {perr:.2e}")
    assert rel <= 1e-6 and perr <= 1e-4
    osl = _ctx(cf, dict(w, y=y), precision, 0)
    cf.cfust_fit(osl, iters)
    nu_osl = cf.cfust_get_params(osl)["nu"]
    assert np.max(np.abs(got["nu"] - nu_osl) / nu_osl) > 1e-3  # the nu update sees the exact term


def test_exact_elogw_errors(cf):
    w = synth.make_workload("flow_p4", n=50)
    q = w["qmc"]
    for kw in (dict(moments=0, elogw=1), dict(moments=1, elogw=2),
               dict(moments=1, elogw=1, model=cf.CFUST_MODEL_CFUSN)):
        with pytest.raises(cf.CfustError) as e:
            cf.cfust_create(4, 4, 4, 50, cf.cfust_default_opts(**kw))
        assert e.value.status == cf.CFUST_EINVAL
    c = _ctx(cf, w, 1, 1)
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_surrogate_train(c)
    assert e.value.status == cf.CFUST_EINVAL
    w2 = synth.make_workload("two_comp_p2", n=50)
    with pytest.raises(cf.CfustError):
        cf.cfust_create(2, 2, 2, 50, cf.cfust_default_opts(moments=1, elogw=1))
