"""cfust_reduce_stats_noalloc against the allocating path.

Callers that cannot allocate device memory (their own memory pool owns the
device, or a latency-critical loop must not pay the synchronisation of
cudaMalloc/cudaFree) use cfust_reduce_stats_noalloc, whose scratch is a fixed
device array inside the library.  This test runs the ordinary E-step of a
context, hands its per-pair arrays (as device tensors) to the allocation-free
entry point, and checks posterior weights, statistics and log-likelihood
against cfust_estep / cfust_get_stats / cfust_get_pairs on two calls in a row.
It lives in its own file so that it is collected after every other test.
"""
import numpy as np
import pytest

from paper_1606_02054_gb300 import synth

pytestmark = pytest.mark.gpu


def test_reduce_stats_noalloc_matches_allocating_path():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1606_02054_gb300 import build

    build.build()
    import paper_1606_02054_gb300 as cf

    w = synth.make_workload("flow_p4", n=3000)
    p, q, g, n = w["p"], w["q"], w["g"], w["n"]
    qs = w["qmc"]
    opts = cf.cfust_default_opts(precision=cf.CFUST_PREC_FP32, qmc_points=qs["npoints"],
                                 qmc_shifts=qs["nshifts"], qmc_korobov_a=qs["korobov_a"],
                                 seed=qs["seed"])
    ctx = cf.cfust_create(p, q, g, n, opts)
    cf.cfust_set_data(ctx, w["y"])
    cf.cfust_set_params(ctx, w["init"])
    L = cf.cfust_estep(ctx)
    S_ref = cf.cfust_get_stats(ctx)
    pairs = cf.cfust_get_pairs(ctx)

    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    y, pi, mu = dev(w["y"]), dev(w["init"]["pi"]), dev(w["init"]["mu"])
    logf, u, el = dev(pairs["logf"]), dev(pairs["u"]), dev(pairs["elogu"])
    eu, euu = dev(pairs["eu"]), dev(pairs["euu"])
    S = 3 + p + q + p * q + q * q + p * p
    for call in range(2):
        tau = torch.full((g * n,), float("nan"), dtype=torch.float64, device="cuda")
        stats = torch.full((g * S + 1,), float("nan"), dtype=torch.float64, device="cuda")
        cf.cfust_reduce_stats_noalloc(p, q, g, n, y, pi, mu, logf, u, el, eu, euu, tau, stats)
        got = stats.cpu().numpy()
        np.testing.assert_allclose(got[:-1].reshape(g, S), S_ref, rtol=1e-12, atol=1e-9)
        assert abs(got[-1] - L) <= 1e-12 * abs(L), (call, got[-1], L)
        np.testing.assert_allclose(tau.cpu().numpy().reshape(g, n), pairs["tau"], rtol=0, atol=1e-14)

    # beyond the fixed scratch: a clear error from the library itself, nothing launched
    # (called through ctypes directly: the Python wrapper would already reject the
    # tensors as shorter than n = 10^7 needs)
    import ctypes as C

    big_n = 10_000_000
    vp = lambda t: C.c_void_p(t.data_ptr())
    st = cf.lib().cfust_reduce_stats_noalloc(p, q, g, big_n, vp(y), vp(pi), vp(mu), vp(logf), vp(u),
                                             vp(el), vp(eu), vp(euu), None, vp(stats), None)
    assert st == cf.CFUST_EINVAL and "scratch" in cf.cfust_last_error(None)

    # a tensor shorter than its stated size: rejected before the library is called
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_reduce_stats_noalloc(p, q, g, n, y, pi, mu, logf, u, el, eu[:-1], euu, None, stats)
    assert e.value.status == cf.CFUST_EINVAL and "eu holds" in str(e.value)
