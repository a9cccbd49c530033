"""Plain FP64 restatement of the learned surrogate's network (numpy).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it, and it shares no code with the CUDA path.

The surrogate is not part of the paper.  It approximates, per integral record,
the quantities the E-step takes from the lattice integrator: log T_q (eq 4 at
dof nu + p; eq 13 at nu + p + 2) and the standardised truncated moments that
enter eqs 16-17 (single-pass form).  The network:

  features f = (b_1..b_q, R_ij for i > j (row-major), 1/dof), standardised by
  (f - fmean) / fstd and zero-padded to IN = 48 columns;
  z1 = bf16(f) bf16(W1) + b1,  h1 = bf16(tanh z1),  IN -> 256
  z2 = h1 bf16(W2) + b2,       h2 = bf16(tanh z2),  256 -> 256
  z3 = h2 bf16(W3) + b3,       h3 = bf16(tanh z3),  256 -> 256
  y  = h3 bf16(W4) + b4,                          256 -> OUT = 48 (the first
  1 + q + q(q+1)/2 used, standardised: log T, the conditional mean m1 = E[X | X <= b],
  and the lower Cholesky factor L of the conditional covariance, row-major, with
  log of its diagonal -- so that every predicted covariance is positive definite)

with bf16 = round to nearest even to bfloat16 (via float32), at exactly the
points where the device rounds; every sum here is FP64.  Loss: the masked squared
error L = sum m (y - t)^2 / (2 B nout) over B rows and the nout used outputs.
Backward: dy = m (y - t) / (B nout),
each GEMM operand rounded to bfloat16 where the device rounds it.  Adam
(Kingma & Ba, 2015) with bias correction, in FP64.
"""
from __future__ import annotations

import numpy as np

IN, H, OUT = 48, 256, 48
SHAPES = (("W1", (IN, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
          ("W4", (H, OUT)), ("b4", (OUT,)))
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def bf16(x):
    """Round to nearest even to bfloat16, through float32 (returned as float64)."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    nan = np.isnan(a)
    if nan.any():
        out[nan] = np.nan
    return out


def unpack(theta):
    """Flat parameter vector (float32 layout W1, b1, W2, b2, W3, b3, W4, b4; matrices
    row-major with the input index first) -> dict of float64 arrays."""
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


def pack(P):
    return np.concatenate([np.asarray(P[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def init(seed, nin, nout):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights over the used rows/columns, zero
    padding and biases (the device's initialiser draws the same numbers from the same
    counter-based SplitMix64 stream: element e of the flat vector uses key seed ^ (e + 1))."""
    theta = np.zeros(NPARAM)
    o = 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        if name[0] == "W":
            fan_in = nin if name == "W1" else H
            u = _splitmix_u01(np.uint64(seed) ^ (np.arange(k, dtype=np.uint64) + np.uint64(o + 1)))
            w = (2.0 * u - 1.0) / np.sqrt(fan_in)
            rows, cols = np.divmod(np.arange(k), shape[1])
            live = np.ones(k, bool)
            if name == "W1":
                live = rows < nin
            if name == "W4":
                live = cols < nout
            theta[o:o + k] = np.where(live, w, 0.0)
        o += k
    return theta


def _splitmix_u01(key):
    """SplitMix64 (Steele, Lea & Flood 2014) output of one step from state key (uint64
    array; arithmetic wraps mod 2^64), top 53 bits as a double in [0, 1)."""
    with np.errstate(over="ignore"):
        z = key + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def forward(theta, f, rounding=True):
    """f: B x IN standardised features.  Returns (y, cache)."""
    P = unpack(theta)
    r = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    x = r(f)
    hs = [x]
    for l in (1, 2, 3):
        z = hs[-1] @ r(P[f"W{l}"]) + P[f"b{l}"]
        hs.append(r(np.tanh(z)))
    y = hs[-1] @ r(P["W4"]) + P["b4"]
    return y, hs


def loss(y, t, m, nout):
    return float(np.sum(m * (y - t) ** 2) / (2.0 * y.shape[0] * nout))


def grad(theta, f, t, m, nout, rounding=True):
    """Gradient of the masked loss with respect to theta (flat), and the loss."""
    P = unpack(theta)
    r = bf16 if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    y, hs = forward(theta, f, rounding)
    dy = m * (y - t) / (y.shape[0] * nout)
    g = {}
    dz = r(dy)
    for l in (4, 3, 2, 1):
        g[f"W{l}"] = hs[l - 1].T @ dz
        g[f"b{l}"] = dz.sum(axis=0)
        if l > 1:
            dh = dz @ r(P[f"W{l}"]).T
            dz = r(dh * (1.0 - hs[l - 1] ** 2))
    return pack(g), loss(y, t, m, nout)


def adam(theta, g, mom, vel, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (step number t >= 1); returns new (theta, mom, vel)."""
    mom = beta1 * mom + (1.0 - beta1) * g
    vel = beta2 * vel + (1.0 - beta2) * g * g
    mh = mom / (1.0 - beta1 ** t)
    vh = vel / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), mom, vel


def features(bt, Lc, dof):
    """Unstandardised features of records: bt (B x q) standardised limits, Lc (B x q x q)
    lower Cholesky factors of the correlation matrices, dof (B,).  Returns B x nin,
    nin = q + q(q-1)/2 + 1."""
    bt = np.asarray(bt, dtype=np.float64)
    B, q = bt.shape
    R = np.einsum("bik,bjk->bij", Lc, Lc)
    cols = [bt]
    ii, jj = np.tril_indices(q, -1)
    cols.append(R[:, ii, jj])
    cols.append((1.0 / np.asarray(dof, dtype=np.float64))[:, None])
    return np.concatenate(cols, axis=1)


def moments_to_targets(m, q):
    """Lattice moments (E[X] (q), lower triangle of E[X X^T] row-major) -> network
    targets (m1, rows of the Cholesky factor of E[X X^T] - m1 m1^T with log diagonal).
    Returns None where the covariance is not positive definite."""
    m = np.asarray(m, dtype=np.float64)
    m1 = m[:q]
    M2 = np.zeros((q, q))
    ii, jj = np.tril_indices(q)
    M2[ii, jj] = m[q:]
    M2[jj, ii] = m[q:]
    try:
        L = np.linalg.cholesky(M2 - np.outer(m1, m1))
    except np.linalg.LinAlgError:
        return None
    t = L[ii, jj].copy()
    t[ii == jj] = np.log(np.diag(L))
    return np.concatenate([m1, t])


def targets_to_moments(t, q):
    """Inverse of moments_to_targets: m1 and E[X X^T] = L L^T + m1 m1^T (lower triangle)."""
    t = np.asarray(t, dtype=np.float64)
    m1 = t[:q]
    ii, jj = np.tril_indices(q)
    L = np.zeros((q, q))
    v = t[q:].copy()
    v[ii == jj] = np.exp(v[ii == jj])
    L[ii, jj] = v
    M2 = L @ L.T + np.outer(m1, m1)
    return np.concatenate([m1, M2[ii, jj]])
