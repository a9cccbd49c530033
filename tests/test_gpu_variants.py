"""GPU: fits with parameters held by the M-step (cfust_opts.hold) against the
oracle's held fits.  From Delta^(0) = 0 with Delta held, the CFUST EM is the EM
of a mixture of multivariate t (pinned on the CPU against a textbook t-mixture
EM in tests/test_oracle_mstep.py).  FP64, q = 2 (deterministic T_2): final l
within 1e-8 relative and parameters within 1e-6 after 10 iterations; held
values stay bit-identical.
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


def _ctx(cf, w, params, hold):
    q = w["qmc"]
    o = cf.cfust_default_opts(qmc_points=q["npoints"], qmc_shifts=q["nshifts"],
                              qmc_korobov_a=q["korobov_a"], seed=q["seed"], hold=hold)
    c = cf.cfust_create(w["p"], w["q"], w["g"], w["y"].shape[0], o)
    cf.cfust_set_data(c, w["y"])
    cf.cfust_set_params(c, params)
    return c


@pytest.mark.parametrize("hold", [1, 2, 3])
def test_held_fit_matches_oracle(cf, oracle, hold):
    w = synth.make_workload("two_comp_p2", n=500)
    P = {k: np.array(v, dtype=float) for k, v in w["init"].items()}
    if hold & 1:
        P["Delta"][:] = 0.0  # the t mixture
    c = _ctx(cf, w, P, hold)
    it, hist = cf.cfust_fit(c, 10)
    ref, rhist, rit = oracle.fit(w["y"], P, 10, oracle.qmc(**w["qmc"]), hold=hold)
    assert it == rit == 10
    assert abs(hist[-1] - rhist[-1]) <= 1e-8 * abs(rhist[-1])
    got = cf.cfust_get_params(c)
    for k in KEYS:
        np.testing.assert_allclose(got[k], ref[k], rtol=1e-6, atol=1e-9, err_msg=k)
    if hold & 1:
        assert np.all(got["Delta"] == 0.0)
    if hold & 2:
        np.testing.assert_array_equal(got["nu"], P["nu"])


def test_held_fit_batched_equals_host_loop(cf):
    w = synth.make_workload("two_comp_p2", n=400)
    P = {k: np.array(v, dtype=float) for k, v in w["init"].items()}
    P["Delta"][:] = 0.0
    a = _ctx(cf, w, P, cf.CFUST_HOLD_DELTA)
    b = _ctx(cf, w, P, cf.CFUST_HOLD_DELTA)
    it, h = cf.cfust_fit(a, 6)
    iters, hist, status = cf.cfust_fit_batch([b], 6)
    assert status[0] == cf.CFUST_OK and iters[0] == it
    np.testing.assert_array_equal(hist[0], h)
    pa, pb = cf.cfust_get_params(a), cf.cfust_get_params(b)
    for k in KEYS:
        np.testing.assert_array_equal(pb[k], pa[k])


def test_hold_rejects_unknown_bits(cf):
    w = synth.make_workload("two_comp_p2", n=50)
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_create(2, 2, 2, 50, cf.cfust_default_opts(hold=4))
    assert e.value.status == cf.CFUST_EINVAL
