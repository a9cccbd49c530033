"""GPU: cfust_autotune, the launch-shape tuner of the integrators (FP32 T_2 records:
lanes per record; the FP32 single-pass moment pass at q <= 4: lattice points per
lane).  Every candidate shape computes the same integrals (the lanes' partial sums are
added in a different order), so after tuning the E-step still matches the oracle at
the FP32 bounds of the parity tests, and a fit equals the untuned fit to rounding."""
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


def _ctx(cf, w, precision, moments, y):
    q = w["qmc"]
    o = cf.cfust_default_opts(precision=precision, qmc_points=q["npoints"], qmc_shifts=q["nshifts"],
                              qmc_korobov_a=q["korobov_a"], seed=q["seed"], moments=moments)
    c = cf.cfust_create(w["p"], w["q"], w["g"], y.shape[0], o)
    cf.cfust_set_data(c, y)
    cf.cfust_set_params(c, w["init"])
    return c


@pytest.mark.parametrize("name,n,precision,moments", [("wide_p16", 20000, 2, 1), ("flow_p4", 8000, 1, 1),
                                                      ("two_comp_p2", 4000, 1, 0)])
def test_autotune_choices_and_results(cf, oracle, name, n, precision, moments):
    w = synth.make_workload(name, n=n)
    y = w["y"].astype(np.float32) if precision == 2 else w["y"]
    c = _ctx(cf, w, precision, moments, y)
    L_before = cf.cfust_estep(c)
    choices, ms = cf.cfust_autotune(c, reps=2)
    print(name, choices, {k: v for k, v in ms.items() if v is not None})
    has_t2 = w["q"] == 2
    has_mom = moments == 1 and 3 <= w["q"] <= 4
    assert (choices["t2_lanes"] in (2, 4, 8, 16, 32)) == has_t2
    assert (choices["mom_points"] in (1, 2)) == has_mom
    t2 = [ms[f"t2_lanes_{l}"] for l in (2, 4, 8, 16, 32)]
    mp = [ms["mom_points_1"], ms["mom_points_2"]]
    assert all((v is not None and v > 0) == has_t2 for v in t2)
    assert all((v is not None and v > 0) == has_mom for v in mp)
    if has_t2:
        assert ms[f"t2_lanes_{choices['t2_lanes']}"] == min(t2)
    # after tuning: the same E-step to FP32 rounding, and the oracle's at the FP32 bound
    with pytest.raises(cf.CfustError):
        cf.cfust_mstep(c)  # tuning leaves no E-step results
    L_after = cf.cfust_estep(c)
    assert abs(L_after - L_before) <= 1e-8 * abs(L_before)
    o = oracle.estep(y[:400].astype(np.float64), w["init"], oracle.qmc(**dict(w["qmc"], moments=moments)))
    c2 = _ctx(cf, w, precision, moments, y[:400])  # a second context, created after the tuning run
    L2 = cf.cfust_estep(c2)
    assert abs(L2 - o["loglik"]) <= 1e-6 * abs(o["loglik"])


def test_autotuned_fit_matches_untuned(cf):
    w = synth.make_workload("wide_p16", n=12000)
    y = w["y"].astype(np.float32)
    a = _ctx(cf, w, 2, 1, y)
    b = _ctx(cf, w, 2, 1, y)
    cf.cfust_autotune(b, reps=1)
    _, ha = cf.cfust_fit(a, 5)
    _, hb = cf.cfust_fit(b, 5)
    np.testing.assert_allclose(hb, ha, rtol=1e-8)
    pa, pb = cf.cfust_get_params(a), cf.cfust_get_params(b)
    for k in ("pi", "mu", "Sigma", "Delta", "nu"):
        np.testing.assert_allclose(pb[k], pa[k], rtol=1e-5, atol=1e-8)


def test_autotune_errors(cf):
    w = synth.make_workload("two_comp_p2", n=100)
    c = cf.cfust_create(2, 2, 2, 100, cf.cfust_default_opts(precision=1))
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_autotune(c)
    assert e.value.status == cf.CFUST_ESTATE
    cf.cfust_set_data(c, w["y"])
    cf.cfust_set_params(c, w["init"])
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_autotune(c, reps=0)
    assert e.value.status == cf.CFUST_EINVAL
