"""GPU: the learned surrogate's kernels (BF16 tensor-core MLP, Adam, fused record
inference) through the C ABI against the oracle's network (oracle/mlp.py, pinned
on the CPU in tests/test_oracle_mlp.py), and the surrogate E-step and EM against
the lattice.

Tolerances.  The device rounds every hidden activation to BF16 from an FP32 sum
(and tanhf) where the oracle rounds from an FP64 sum (and tanh); where the two
sums straddle a BF16 rounding boundary one activation differs by one BF16 ulp
(2^-8 relative), which moves an output by ~1e-4.  Such flips are rare (the sums
agree to ~1e-7 relative against a half-ulp of 2e-3), so outputs are compared by
their 95th percentile (1e-5, FP32 accumulation alone) and their maximum (3e-3,
flips).  Gradients: 1e-2 norm-wise per tensor (the same flips in the BF16-rounded
backward operands).  Adam: FP32 against FP64, 1e-5 of the step plus one FP32 ulp
of the updated parameter; second moments 1e-4 (1 - 0.999f is 4.7e-5 above 1e-3).
Initialiser:
bit-identical after rounding the oracle's FP64 draw to FP32.
"""
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


@pytest.fixture(scope="module")
def M():
    from oracle import mlp

    return mlp


def _theta(M, seed, nin, nout):
    rng = np.random.default_rng(seed)
    th = M.init(seed, nin, nout)
    P = M.unpack(th)
    for b in ("b1", "b2", "b3"):
        P[b][:] = rng.normal(0, 0.1, P[b].shape)
    P["b4"][:nout] = rng.normal(0, 0.1, nout)
    return np.float32(M.pack(P)).astype(np.float64)


def _close(got, ref, p95=1e-5, mx=3e-3):
    d = np.abs(np.asarray(got, dtype=np.float64) - ref)
    assert np.percentile(d, 95) <= p95, np.percentile(d, 95)
    assert d.max() <= mx, d.max()


def test_init_matches_oracle(cf, M):
    for seed, nin, nout in ((7, 22, 28), (123456789, 11, 15), (3, 37, 45)):
        got = cf.cfust_mlp_init(seed, nin, nout)
        np.testing.assert_array_equal(got, np.float32(M.init(seed, nin, nout)))


@pytest.mark.parametrize("rows", [300, 4096])
def test_forward_backward_match_oracle(cf, M, rows):
    nin, nout = 22, 28
    th = _theta(M, 11, nin, nout)
    rng = np.random.default_rng(rows)
    f = np.zeros((rows, M.IN), np.float32)
    f[:, :nin] = rng.normal(0, 1, (rows, nin))
    t = np.zeros((rows, M.OUT), np.float32)
    t[:, :nout] = rng.normal(0, 1, (rows, nout))
    m = np.zeros((rows, M.OUT), np.float32)
    m[:, 0] = 1
    m[rows // 3:, :nout] = 1
    g, y, loss = cf.cfust_mlp_grad(th, f, t, m, nout)
    ry, _ = M.forward(th, f.astype(np.float64))
    rg, rloss = M.grad(th, f.astype(np.float64), t.astype(np.float64), m.astype(np.float64), nout)
    _close(y[:, :nout], ry[:, :nout])
    assert np.all(y[:, nout:] == np.float32(ry[:, nout:]))  # padding: bias only (zero)
    assert abs(loss - rloss) <= 1e-3 * rloss
    G, RG = M.unpack(g.astype(np.float64)), M.unpack(rg)
    for name, _ in M.SHAPES:
        assert np.linalg.norm(G[name] - RG[name]) <= 1e-2 * np.linalg.norm(RG[name]) + 1e-12, name


def test_adam_matches_oracle(cf, M):
    rng = np.random.default_rng(5)
    n = M.NPARAM
    th = rng.normal(0, 0.1, n).astype(np.float32)
    g = rng.normal(0, 1e-3, n).astype(np.float32)
    m = rng.normal(0, 1e-3, n).astype(np.float32)
    v = np.abs(rng.normal(0, 1e-6, n)).astype(np.float32)
    th1, m1, v1 = cf.cfust_mlp_adam(th, g, m, v, 5, 1e-3)
    rth, rm, rv = M.adam(th.astype(np.float64), g.astype(np.float64), m.astype(np.float64),
                         v.astype(np.float64), 5, 1e-3)
    step = rth - th
    # FP32 step within 1e-5 of the FP64 step, plus the FP32 rounding of the new value
    ulp = np.spacing(np.abs(th1).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs((th1.astype(np.float64) - th) - step) <= 1e-5 * np.abs(step) + ulp)
    # FP32 moment update: relative to the magnitude of its two terms (they may cancel)
    assert np.all(np.abs(m1 - rm) <= 1e-6 * (0.9 * np.abs(m) + 0.1 * np.abs(g)))
    # 1 - beta2 in FP32 (1 - 0.999f) is 4.7e-5 above 0.001
    np.testing.assert_allclose(v1, rv, rtol=1e-4, atol=1e-15)


def _records(q, rows, seed):
    rng = np.random.default_rng(seed)
    bt = rng.normal(0.3, 1.2, (rows, q))
    Lc = np.zeros((rows, q, q))
    for i in range(rows):
        A = rng.normal(0, 1, (q, q + 2))
        S = A @ A.T
        d = np.sqrt(np.diag(S))
        Lc[i] = np.linalg.cholesky(S / np.outer(d, d))
    dof = rng.uniform(8, 30, rows)
    return bt, Lc, dof


def test_record_inference_matches_oracle(cf, M):
    q, rows = 6, 2000
    nin, nout, W = q + q * (q - 1) // 2 + 1, 1 + q + q * (q + 1) // 2, q + q * (q + 1) // 2
    bt, Lc, dof = _records(q, rows, 9)
    F = M.features(bt, Lc, dof)
    f32 = F.astype(np.float32)
    mean = f32.mean(0).astype(np.float32)
    sd = f32.std(0).astype(np.float32)
    z = ((f32 - mean) / sd).astype(np.float32)
    zlo, zhi = z.min(0), z.max(0)
    zhi[0] = np.float32(np.median(z[:, 0]))  # half the records leave the range on feature 0
    margin = np.float32(0.05)
    stats = np.zeros(M.IN * 4 + M.OUT * 2, np.float32)
    stats[:nin] = mean
    stats[M.IN:M.IN + nin] = sd
    stats[M.IN + nin:2 * M.IN] = 1
    stats[2 * M.IN:2 * M.IN + nin] = zlo
    stats[3 * M.IN:3 * M.IN + nin] = zhi
    tm = np.linspace(-2, 1, M.OUT).astype(np.float32)
    ts = np.linspace(0.5, 2, M.OUT).astype(np.float32)
    stats[4 * M.IN:4 * M.IN + M.OUT] = tm
    stats[4 * M.IN + M.OUT:] = ts
    th = _theta(M, 17, nin, nout)
    logT, mom, inbox = cf.cfust_mlp_records(th, stats, margin, bt, Lc, dof)
    lo, hi = zlo - margin, zhi + margin
    ref_in = np.all((z >= lo) & (z <= hi), axis=1)
    clear = np.all((np.abs(z - lo) > 1e-4) & (np.abs(z - hi) > 1e-4), axis=1)
    assert np.array_equal(inbox[clear].astype(bool), ref_in[clear])
    assert 0.3 < ref_in.mean() < 0.7
    fz = np.zeros((rows, M.IN))
    fz[:, :nin] = z
    y, _ = M.forward(th, fz)
    ref_logT = y[:, 0] * ts[0] + tm[0]
    ok = inbox.astype(bool)
    ref_mom = np.array([M.targets_to_moments(y[i, 1:1 + W] * ts[1:1 + W] + tm[1:1 + W], q) for i in range(rows)])
    _close(logT[ok], ref_logT[ok], 1e-5 * ts[0], 3e-3 * ts[0])
    # moments: the same flips, through exp of the log diagonal and L L^T (relative to the row scale)
    scale = np.abs(ref_mom[ok]).max(axis=1, keepdims=True)
    _close(mom[ok] / scale, ref_mom[ok] / scale, 2e-5, 1e-2)
    assert np.all(np.isnan(logT[~ok]))


def _ctx(cf, w, n, precision=1):
    q = w["qmc"]
    o = cf.cfust_default_opts(precision=precision, qmc_points=q["npoints"], qmc_shifts=q["nshifts"],
                              qmc_korobov_a=q["korobov_a"], seed=q["seed"], moments=1)
    c = cf.cfust_create(w["p"], w["q"], w["g"], n, o)
    cf.cfust_set_data(c, w["y"][:n])
    cf.cfust_set_params(c, w["init"])
    return c


def test_surrogate_estep_and_em(cf):
    """learned_p6 subsample (p = q = g = 6), FP32: after training at Psi^(0) the
    surrogate E-step reproduces the lattice l within 1e-3 relative with under 5 %
    fallbacks; every M-step after a surrogate E-step succeeds (the predicted
    covariances are positive definite by construction); 20 surrogate iterations
    followed by 20 lattice iterations keep at least half the l gain of 40 lattice
    iterations (measured: ~90 %; the surrogate's E-step error slows each
    iteration's progress, so this is a sanity bound, not a claim of parity)."""
    n = 20000
    w = synth.make_workload("learned_p6", n=n)
    a = _ctx(cf, w, n)
    b = _ctx(cf, w, n)
    ll0, losses = cf.cfust_surrogate_train(b, seed=3)
    assert np.all(np.isfinite(losses)) and losses[-1] < losses[0]
    L_sur = cf.cfust_estep(b)
    recs, fb = cf.cfust_surrogate_info(b)
    assert recs == 2 * n * w["g"] and fb < 0.05 * recs
    print(f"surrogate E-step l relative error {abs(L_sur - ll0) / abs(ll0):.2e}, fallbacks {fb / recs:.2e}")
    assert abs(L_sur - ll0) <= 1e-3 * abs(ll0)
    for _ in range(20):
        cf.cfust_mstep(b)
        cf.cfust_estep(b)
    cf.cfust_surrogate_use(b, 0)
    _, hist_b = cf.cfust_fit(b, 20)
    _, hist_a = cf.cfust_fit(a, 40)
    assert hist_a[-1] > ll0 and hist_b[-1] > ll0
    assert hist_b[-1] - ll0 >= 0.5 * (hist_a[-1] - ll0)


def test_surrogate_errors(cf):
    w = synth.make_workload("learned_p6", n=500)
    q = w["qmc"]
    o = cf.cfust_default_opts(qmc_points=q["npoints"], qmc_shifts=q["nshifts"], moments=0)
    c = cf.cfust_create(w["p"], w["q"], w["g"], 500, o)
    cf.cfust_set_data(c, w["y"])
    cf.cfust_set_params(c, w["init"])
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_surrogate_train(c)
    assert e.value.status == cf.CFUST_EINVAL
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_surrogate_use(c, 1)
    assert e.value.status == cf.CFUST_ESTATE
    d = _ctx(cf, w, 500)
    with pytest.raises(cf.CfustError) as e:
        cf.cfust_surrogate_train(d, batch=100)
    assert e.value.status == cf.CFUST_EINVAL
