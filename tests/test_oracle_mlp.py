"""Pins of the oracle's surrogate network (oracle/mlp.py), CPU only.

The network is not in the paper; its oracle is pinned by what fixes it
independently: torch's bfloat16 conversion for the rounding, central finite
differences of the unrounded FP64 loss for the backward pass, Adam's closed
forms (the first step moves every coordinate by lr sign(g); with a constant
gradient the bias-corrected step stays lr g / (|g| + eps)), the initialiser's
bounds, the correlation features against a matrix built by hand, and the moment
parametrisation (mean and log-diagonal Cholesky factor of the covariance) by its
round trip and the positive definiteness of every output's covariance.
"""
import math

import numpy as np
import pytest

from oracle import mlp as M


def test_bf16_matches_torch_and_ties_to_even():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-20, 100), rng.normal(0, 1e20, 100),
                        [0.0, -0.0, 1.0, -2.5, 65504.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.bf16(x), ref)
    one = 1.0
    assert M.bf16(one + 2.0 ** -8) == 1.0                     # tie between 1 and 1 + 2^-7: even
    assert M.bf16(one + 3 * 2.0 ** -8) == one + 2.0 ** -6       # tie: rounds up to the even mantissa
    assert M.bf16(one + 2.0 ** -8 + 2.0 ** -20) == one + 2.0 ** -7


def _problem(seed=1, B=7, nin=9, nout=5):
    rng = np.random.default_rng(seed)
    theta = M.init(seed, nin, nout)
    theta[M.NPARAM - M.OUT:] = rng.normal(0, 0.1, M.OUT)  # non-zero biases too
    f = np.zeros((B, M.IN))
    f[:, :nin] = rng.normal(0, 1, (B, nin))
    t = np.zeros((B, M.OUT))
    t[:, :nout] = rng.normal(0, 1, (B, nout))
    m = np.zeros((B, M.OUT))
    m[:, 0] = 1.0
    m[B // 2:, :nout] = 1.0
    return theta, f, t, m, nout


def test_backward_matches_finite_differences():
    theta, f, t, m, nout = _problem()
    g, L = M.grad(theta, f, t, m, nout, rounding=False)
    y, _ = M.forward(theta, f, rounding=False)
    assert L == pytest.approx(M.loss(y, t, m, nout))
    rng = np.random.default_rng(2)
    P = M.unpack(theta)
    offs, o = {}, 0
    for name, shape in M.SHAPES:
        offs[name] = o
        o += int(np.prod(shape))
    picks = []
    for name, shape in M.SHAPES:
        rows = shape[0]
        for _ in range(6):
            if len(shape) == 2:
                i = rng.integers(0, 9 if name == "W1" else rows)
                j = rng.integers(0, 5 if name == "W4" else shape[1])
                picks.append(offs[name] + i * shape[1] + j)
            else:
                picks.append(offs[name] + rng.integers(0, 5 if name == "b4" else shape[0]))
    h = 1e-6
    for e in picks:
        tp, tm = theta.copy(), theta.copy()
        tp[e] += h
        tm[e] -= h
        fd = (M.loss(M.forward(tp, f, False)[0], t, m, nout) - M.loss(M.forward(tm, f, False)[0], t, m, nout)) / (2 * h)
        assert abs(g[e] - fd) <= 1e-7 + 1e-5 * abs(fd), (e, g[e], fd)
    # padding rows of W1 and padding columns of W4 get no gradient through masked outputs
    gW4 = M.unpack(g)["W4"]
    assert np.all(gW4[:, nout:] == 0.0)


def test_rounded_backward_is_close_to_exact():
    theta, f, t, m, nout = _problem(seed=3, B=64)
    g0, _ = M.grad(theta, f, t, m, nout, rounding=False)
    g1, _ = M.grad(theta, f, t, m, nout, rounding=True)
    assert np.linalg.norm(g1 - g0) <= 0.03 * np.linalg.norm(g0)


def test_adam_closed_forms():
    rng = np.random.default_rng(4)
    theta = rng.normal(0, 1, 50)
    g = rng.normal(0, 1, 50)
    m = np.zeros(50)
    v = np.zeros(50)
    th1, m1, v1 = M.adam(theta, g, m, v, 1, 1e-3)
    np.testing.assert_allclose(th1, theta - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    th, mm, vv = theta, m, v
    for step in range(1, 40):
        th_new, mm, vv = M.adam(th, g, mm, vv, step, 1e-3)
        np.testing.assert_allclose(th - th_new, 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
        th = th_new


def test_init_bounds_and_padding():
    nin, nout = 22, 28
    P = M.unpack(M.init(9, nin, nout))
    assert np.all(np.abs(P["W1"][:nin]) <= 1 / math.sqrt(nin)) and np.all(P["W1"][nin:] == 0)
    assert np.all(np.abs(P["W2"]) <= 1 / 16) and np.all(np.abs(P["W3"]) <= 1 / 16)
    assert np.all(P["W4"][:, nout:] == 0) and np.all(np.abs(P["W4"]) <= 1 / 16)
    for b in ("b1", "b2", "b3", "b4"):
        assert np.all(P[b] == 0)
    # uniform: mean ~ 0, variance 1/(3 fan_in)
    w = P["W2"].ravel() * 16
    assert abs(w.mean()) < 0.01 and abs(w.var() - 1 / 3) < 0.01
    assert not np.array_equal(M.init(9, nin, nout), M.init(10, nin, nout))


def test_features_order():
    q = 4
    R = np.array([[1.0, 0.2, -0.3, 0.1], [0.2, 1.0, 0.4, -0.2], [-0.3, 0.4, 1.0, 0.25], [0.1, -0.2, 0.25, 1.0]])
    L = np.linalg.cholesky(R)
    bt = np.array([[0.5, -1.0, 2.0, 0.0]])
    f = M.features(bt, L[None], np.array([12.0]))
    np.testing.assert_allclose(f[0], [0.5, -1.0, 2.0, 0.0, 0.2, -0.3, 0.4, 0.1, -0.2, 0.25, 1 / 12.0], atol=1e-15)


def test_moment_targets_round_trip_and_psd():
    rng = np.random.default_rng(6)
    q = 5
    ii, jj = np.tril_indices(q)
    for _ in range(20):
        m1 = rng.normal(0, 1, q)
        A = rng.normal(0, 1, (q, q))
        C = A @ A.T + 0.1 * np.eye(q)
        M2 = C + np.outer(m1, m1)
        m = np.concatenate([m1, M2[ii, jj]])
        t = M.moments_to_targets(m, q)
        np.testing.assert_allclose(M.targets_to_moments(t, q), m, rtol=1e-12, atol=1e-12)
        # any output vector maps to a positive definite covariance
        back = M.targets_to_moments(rng.normal(0, 2, t.size), q)
        S = np.zeros((q, q))
        S[ii, jj] = back[q:]
        S[jj, ii] = back[q:]
        assert np.all(np.linalg.eigvalsh(S - np.outer(back[:q], back[:q])) > 0)
    bad = np.concatenate([np.ones(q), np.zeros(q * (q + 1) // 2)])  # E[X X^T] = 0 < m1 m1^T
    assert M.moments_to_targets(bad, q) is None
