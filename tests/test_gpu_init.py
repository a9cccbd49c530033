"""GPU: initialisation by Algorithm 1 (Sec. 3.3, eq 23) through cfust_init against
the oracle's Algorithm 1 on the same partitions and lattice.

Tolerances: each candidate's log-likelihood within 1e-9 relative (FP64 density
pass; -inf for the same invalid candidates), the same chosen candidate, and the
chosen parameters within 1e-10 relative (the cluster sums differ only in
summation order).
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


def _ctx(cf, w, y, precision=0):
    q = w["qmc"]
    o = cf.cfust_default_opts(precision=precision, qmc_points=q["npoints"], qmc_shifts=q["nshifts"],
                              qmc_korobov_a=q["korobov_a"], seed=q["seed"], moments=1)
    c = cf.cfust_create(w["p"], w["q"], w["g"], y.shape[0], o)
    cf.cfust_set_data(c, y)
    return c


def _compare(cf, c, ll, ib, ref):
    rbest, rll, rib = ref
    fin = np.isfinite(rll)
    assert np.array_equal(np.isfinite(ll), fin)
    np.testing.assert_allclose(ll[fin], rll[fin], rtol=1e-9)
    assert ib == rib
    got = cf.cfust_get_params(c)
    for k in KEYS:
        np.testing.assert_allclose(got[k], rbest[k], rtol=1e-10, atol=1e-12, err_msg=k)


@pytest.mark.parametrize("name,n,alphas", [("flow_p4", 1500, None), ("two_comp_p2", 600, (0.6, 0.75, 0.9))])
def test_init_random_partitions(cf, oracle, name, n, alphas):
    w = synth.make_workload(name, n=n, with_init=False)
    c = _ctx(cf, w, w["y"])
    ll, ib = cf.cfust_init(c, nstarts=3, seed=99, alphas=alphas)
    spec = oracle.qmc(**dict(w["qmc"], moments=1))
    ref = oracle.init(w["y"], w["g"], w["q"], spec, nstarts=3, seed=99,
                      alphas=oracle.ALPHAS if alphas is None else alphas)
    _compare(cf, c, ll, ib, ref)


def test_init_given_labels_wide(cf, oracle):
    """p = 16, q = 2, g = 8 with k-means partitions (the 1 < q < p shape of Delta)."""
    w = synth.make_workload("wide_p16", n=4000, with_init=False)
    y = w["y"]
    labels = np.stack([synth.kmeans(np.random.default_rng(s), y, w["g"]) for s in range(2)]).astype(np.int32)
    c = _ctx(cf, w, y)
    ll, ib = cf.cfust_init(c, nstarts=2, labels=labels, alphas=(0.9, 0.95, 0.99))
    ref = oracle.init(y, w["g"], w["q"], oracle.qmc(**w["qmc"]), nstarts=2, labels=labels,
                      alphas=(0.9, 0.95, 0.99))
    _compare(cf, c, ll, ib, ref)


def test_init_then_fit(cf):
    w = synth.make_workload("two_comp_p2", n=600, with_init=False)
    c = _ctx(cf, w, w["y"])
    ll, ib = cf.cfust_init(c, nstarts=4, seed=3)
    it, hist = cf.cfust_fit(c, 20)
    assert hist[0] == pytest.approx(ll.flat[ib], rel=1e-12)
    assert hist[-1] > hist[0]


def test_init_errors(cf):
    w = synth.make_workload("two_comp_p2", n=200, with_init=False)
    c = _ctx(cf, w, w["y"])
    bad = np.full((1, 200), 2, dtype=np.int32)  # g = 2: labels must be 0 or 1
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_init(c, nstarts=1, labels=bad)
    assert e.value.status == cf.CFUST_EINVAL
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_init(c, nstarts=1, alphas=(0.5, 1.0))
    assert e.value.status == cf.CFUST_EINVAL
    # every cluster but one empty: no valid candidate
    one = np.zeros((1, 200), dtype=np.int32)
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_init(c, nstarts=1, labels=one)
    assert e.value.status == cf.CFUST_ENOTPD


# ---- k-means partitions on the device (Algorithm 1's clusterings) ------------------
def _near_ties(y, centres, rel=1e-9):
    """Observations whose two nearest centres are within rel in squared distance: there
    the assignment may differ by the order of the cluster sums' rounding."""
    d = np.sort(((y[:, None, :] - centres[None]) ** 2).sum(-1), axis=1)
    return d[:, 1] - d[:, 0] <= rel * d[:, 0]


@pytest.mark.parametrize("name,n,starts", [("flow_p4", 20000, 3), ("wide_p16", 20000, 2), ("two_comp_p2", 5000, 2)])
def test_kmeans_matches_oracle(cf, oracle, name, n, starts):
    """Same starting centres, same Lloyd iteration: labels identical (but for near-ties,
    which rounding may decide either way), centres within 1e-9 relative, same count of
    assignments when no label differs."""
    w = synth.make_workload(name, n=n, with_init=False)
    c = _ctx(cf, w, w["y"])
    lab, its, cen = cf.cfust_kmeans(c, nstarts=starts, seed=2024, max_iter=300)
    rlab, rits, rcen = oracle.kmeans(w["y"], w["g"], nstarts=starts, seed=2024, max_iter=300)
    for s in range(starts):
        diff = lab[s] != rlab[s]
        tie = _near_ties(w["y"], rcen[s])
        assert np.all(tie[diff]), f"start {s}: {diff.sum()} labels differ, {np.sum(diff & ~tie)} not at ties"
        np.testing.assert_allclose(cen[s], rcen[s], rtol=1e-9, atol=1e-12)
        if not diff.any():
            assert its[s] == rits[s]
        assert its[s] < 300


def test_kmeans_partitions_for_init(cf, oracle):
    """Algorithm 1 on device k-means partitions: the candidates and the chosen start
    match the oracle's Algorithm 1 on the oracle's k-means partitions."""
    w = synth.make_workload("flow_p4", n=3000, with_init=False)
    c = _ctx(cf, w, w["y"])
    lab, _, _ = cf.cfust_kmeans(c, nstarts=2, seed=5, max_iter=200)
    rlab, _, _ = oracle.kmeans(w["y"], w["g"], nstarts=2, seed=5, max_iter=200)
    assert np.array_equal(lab, rlab)
    ll, ib = cf.cfust_init(c, nstarts=2, labels=lab)
    ref = oracle.init(w["y"], w["g"], w["q"], oracle.qmc(**dict(w["qmc"], moments=1)), nstarts=2, labels=rlab)
    _compare(cf, c, ll, ib, ref)


def test_kmeans_errors(cf):
    w = synth.make_workload("two_comp_p2", n=200, with_init=False)
    c = _ctx(cf, w, w["y"])
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_kmeans(c, nstarts=0)
    assert e.value.status == cf.CFUST_EINVAL
    c1 = cf.cfust_create(2, 2, 2, 1, cf.cfust_default_opts())
    cf.cfust_set_data(c1, w["y"][:1])
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_kmeans(c1)
    assert e.value.status == cf.CFUST_EINVAL
