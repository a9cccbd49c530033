"""The row-sharded fit on one GPU: two library contexts hold the two shards of
the observations (rows split on a segment boundary), the exchange is a
concatenation on the device, and the sharded EM (paper_1606_02054_gb300.shard)
must reproduce cfust_fit on the whole problem bit for bit: the same statistics,
log-likelihoods l(Psi^(k)) and parameters after every iteration.  Only the final
density-pass log-likelihood is summed per shard (to rounding)."""
import numpy as np
import pytest
import torch

from paper_1606_02054_gb300 import shard, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_02054_gb300 import build

    build.build()
    import paper_1606_02054_gb300 as cf

    return cf


def _opts(cf, w, precision, moments):
    q = w["qmc"]
    return cf.cfust_default_opts(precision=precision, qmc_points=q["npoints"], qmc_shifts=q["nshifts"],
                                 qmc_korobov_a=q["korobov_a"], seed=q["seed"], moments=moments)


@pytest.mark.parametrize("name,n,precision,moments,world",
                         [("flow_p4", 20000, 1, 1, 2), ("wide_p16", 30000, 2, 1, 2), ("two_comp_p2", 20000, 0, 0, 3)])
def test_sharded_fit_reproduces_cfust_fit(cf, name, n, precision, moments, world):
    w = synth.make_workload(name, n=n)
    y = w["y"].astype(np.float32) if precision == 2 else w["y"]
    opts = _opts(cf, w, precision, moments)
    iters = 4
    # the whole problem in one context
    whole = cf.cfust_create(w["p"], w["q"], w["g"], n, opts)
    cf.cfust_set_data(whole, y)
    cf.cfust_set_params(whole, w["init"])
    it_ref, hist_ref = cf.cfust_fit(whole, iters)
    ref = cf.cfust_get_params(whole)
    # the same rows in `world` shards
    rps = cf.cfust_rows_per_segment(w["p"], w["q"], w["g"], precision)
    bounds, per = shard.shard_bounds(n, world, rps)
    assert all(lo % rps == 0 for lo, _ in bounds)
    engines = [shard.CudaShard(cf, w["p"], w["q"], w["g"], lo, hi, opts, np.ascontiguousarray(y[lo:hi]),
                               w["init"], per, n) for lo, hi in bounds]
    it, hist = shard.sharded_fit(engines, torch.cat, iters)
    assert it == it_ref == iters
    assert np.array_equal(hist[:-1], hist_ref[:-1])
    assert abs(hist[-1] - hist_ref[-1]) <= 1e-13 * abs(hist_ref[-1])
    for e in engines:
        got = cf.cfust_get_params(e.ctx)
        for k in ("pi", "mu", "Sigma", "Delta", "nu"):
            assert np.array_equal(got[k], ref[k]), (k, np.max(np.abs(got[k] - ref[k])))


def test_sharded_statistics_equal_whole(cf):
    """One E-step: the statistics reduced from the gathered shard segments equal
    cfust_get_stats of the whole problem bit for bit, with uneven shards."""
    w = synth.make_workload("flow_p4", n=30001)
    opts = _opts(cf, w, 1, 1)
    whole = cf.cfust_create(w["p"], w["q"], w["g"], w["n"], opts)
    cf.cfust_set_data(whole, w["y"])
    cf.cfust_set_params(whole, w["init"])
    L = cf.cfust_estep(whole)
    S = cf.cfust_get_stats(whole)
    rps = cf.cfust_rows_per_segment(w["p"], w["q"], w["g"], 1)
    bounds, per = shard.shard_bounds(w["n"], 3, rps)
    engines = [shard.CudaShard(cf, w["p"], w["q"], w["g"], lo, hi, opts, w["y"][lo:hi], w["init"], per, w["n"])
               for lo, hi in bounds]
    allseg = torch.cat([e.estep_segments() for e in engines])
    for e in engines:
        assert e.reduce_segments(allseg) == L
        assert np.array_equal(cf.cfust_get_stats(e.ctx), S)
