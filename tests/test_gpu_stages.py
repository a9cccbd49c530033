"""GPU stage checks: the per-component factor blocks written by the set-up
kernel and the per-pair quantities of the plan kernel, read back through
cfust_debug_read, against their definitions (under eq 4) evaluated with numpy."""
import math

import numpy as np
import pytest
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


def _layout(p, q):
    o = 0
    L = {}
    for name, size in (("mu", p), ("Linv", p * p), ("A", p * q), ("scal", 4), ("Lam", q * q),
                       ("dq", q), ("Lq", q * q)):
        L[name] = o
        o += size
    q1, q2 = q - 1, max(q - 2, 0)
    L["l1s"] = 2 * q1 + 2 * q1 * q1 if q1 > 0 else 0
    L["l1"] = o
    o += q * L["l1s"]
    L["l2s"] = 2 * q2 + q2 * q2 if q2 > 0 else 0
    L["l2"] = o
    o += q * (q - 1) * L["l2s"]
    L["stride"] = (o + 1) & ~1
    return L


def _corr_chol(S):
    d = 1 / np.sqrt(np.diag(S))
    R = S * np.outer(d, d)
    np.fill_diagonal(R, 1.0)
    return d, np.linalg.cholesky(R)


def _schur(S, r):
    idx = [i for i in range(S.shape[0]) if i != r]
    m = S[idx, r] / S[r, r]
    return S[np.ix_(idx, idx)] - np.outer(S[idx, r], S[r, idx]) / S[r, r], m


@pytest.mark.parametrize("name,n", [("two_comp_p2", 30), ("flow_p4", 30)])
def test_factor_blocks_and_plan(cf, name, n):
    w = synth.make_workload(name, n=n)
    p, q, g = w["p"], w["q"], w["g"]
    qs = w["qmc"]
    ctx = cf.cfust_create(p, q, g, n, cf.cfust_default_opts(
        qmc_points=qs["npoints"], qmc_shifts=qs["nshifts"], qmc_korobov_a=qs["korobov_a"],
        seed=qs["seed"]))
    cf.cfust_set_data(ctx, w["y"])
    P = w["init"]
    cf.cfust_set_params(ctx, P)
    cf.cfust_estep(ctx)
    assert cf.cfust_debug_read(ctx, 9, 4, np.int32)[0] == 0
    F = cf.cfust_debug_read(ctx, 0)
    Ly = _layout(p, q)
    assert F.size == g * Ly["stride"]
    pd = cf.cfust_debug_read(ctx, 1, 16 * n * g).reshape(g, n, 2)
    pc = cf.cfust_debug_read(ctx, 2, 8 * n * g * q).reshape(g, n, q)
    for h in range(g):
        Fh = F[h * Ly["stride"]:(h + 1) * Ly["stride"]]
        blk = lambda k, sz: Fh[Ly[k]:Ly[k] + sz]
        Om = P["Sigma"][h] + P["Delta"][h] @ P["Delta"][h].T
        Linv = np.linalg.inv(np.linalg.cholesky(Om))
        Lam = np.eye(q) - P["Delta"][h].T @ np.linalg.solve(Om, P["Delta"][h])
        np.testing.assert_allclose(blk("mu", p), P["mu"][h], rtol=0, atol=0)
        np.testing.assert_allclose(blk("Linv", p * p).reshape(p, p), Linv, rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(blk("A", p * q).reshape(p, q), Linv @ P["Delta"][h],
                                   rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(blk("Lam", q * q).reshape(q, q), Lam, rtol=1e-11, atol=1e-13)
        d, Lc = _corr_chol(Lam)
        np.testing.assert_allclose(blk("dq", q), d, rtol=1e-11)
        np.testing.assert_allclose(blk("Lq", q * q).reshape(q, q), Lc, rtol=1e-10, atol=1e-12)
        for r in range(q if q > 1 else 0):
            q1 = q - 1
            b = Fh[Ly["l1"] + r * Ly["l1s"]:Ly["l1"] + (r + 1) * Ly["l1s"]]
            S1, m1 = _schur(Lam, r)
            np.testing.assert_allclose(b[:q1], m1, rtol=1e-10, atol=1e-13)
            np.testing.assert_allclose(b[q1:q1 + q1 * q1].reshape(q1, q1), S1, rtol=1e-10, atol=1e-13)
            d1, L1 = _corr_chol(S1)
            np.testing.assert_allclose(b[q1 + q1 * q1:2 * q1 + q1 * q1], d1, rtol=1e-10)
            np.testing.assert_allclose(b[2 * q1 + q1 * q1:].reshape(q1, q1), L1, rtol=1e-9, atol=1e-12)
            for s in range(q1 if q > 2 else 0):
                q2 = q - 2
                off = Ly["l2"] + (r * q1 + s) * Ly["l2s"]
                b2 = Fh[off:off + Ly["l2s"]]
                S2, m2 = _schur(S1, s)
                d2, L2 = _corr_chol(S2)
                np.testing.assert_allclose(b2[:q2], m2, rtol=1e-9, atol=1e-12)
                np.testing.assert_allclose(b2[q2:2 * q2], d2, rtol=1e-9)
                np.testing.assert_allclose(b2[2 * q2:].reshape(q2, q2), L2, rtol=1e-9, atol=1e-12)
        # plan: d, log t_p and c per pair
        R = w["y"] - P["mu"][h]
        dref = np.einsum("ja,ab,jb->j", R, np.linalg.inv(Om), R)
        np.testing.assert_allclose(pd[h, :, 0], dref, rtol=1e-11)
        ltp = st.multivariate_t(loc=P["mu"][h], shape=Om, df=P["nu"][h]).logpdf(w["y"])
        np.testing.assert_allclose(pd[h, :, 1], ltp, rtol=1e-11)
        np.testing.assert_allclose(pc[h], R @ np.linalg.solve(Om, P["Delta"][h]), rtol=1e-10, atol=1e-12)
