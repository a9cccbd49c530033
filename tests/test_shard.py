"""CPU tests of the row-sharded EM driver (paper_1606_02054_gb300.shard): the
shard bounds, and two gloo ranks on host tensors.

The sharded fit splits the observations by rows (Sec. 4's once-per-iteration
collection, over processes instead of threads).  Here the per-shard work is the
FP64 oracle's (no GPU): each rank runs the oracle E-step on its rows, the
driver's exchange gathers every rank's rows in rank order (zero padding), and
each rank runs the oracle M-step on the gathered arrays, so the sharded fit
must equal the single-process oracle fit.  The statistics check sums each
rank's segments of the sufficient statistics (blocks of rows, segments of
blocks, in the library's order) and gathers them: the rank-ordered sum equals
the single-process segment reduction bit for bit."""
import os
import socket

import numpy as np
import pytest

from paper_1606_02054_gb300 import shard, synth


def test_shard_bounds():
    for n, world, rps in [(20000, 2, 7168), (7168 * 4, 4, 7168), (100_000, 3, 8192), (9000, 2, 4096)]:
        b, per = shard.shard_bounds(n, world, rps)
        assert b[0][0] == 0 and b[-1][1] == n
        for (lo, hi), (lo2, _) in zip(b, b[1:]):
            assert hi == lo2  # contiguous
        for lo, hi in b:
            assert lo % rps == 0 and hi > lo
            assert -(-(hi - lo) // rps) <= per
    with pytest.raises(ValueError):
        shard.shard_bounds(100, 2, 4096)  # one segment cannot feed two ranks


# ---- stand-ins used by the gloo ranks (module level: spawned processes import them) ----
CHUNK, SEG = 64, 4  # rows per block and blocks per segment of the stand-in reduction


def _stats_rows(y, params, e):
    """Per-observation rows of the sufficient statistics (the layout of
    cfust_get_stats per component, then the log-likelihood term)."""
    g = params["pi"].size
    n = y.shape[0]
    rows = []
    for h in range(g):
        t, u = e["tau"][h], e["u"][h]
        r = y - params["mu"][h]
        rows += [t[:, None], (t * u)[:, None], (t * (e["elogu"][h] - u))[:, None], (t * u)[:, None] * r,
                 t[:, None] * e["eu"][h], (t[:, None, None] * r[:, :, None] * e["eu"][h][:, None, :]).reshape(n, -1),
                 (t[:, None, None] * e["euu"][h]).reshape(n, -1),
                 ((t * u)[:, None, None] * r[:, :, None] * r[:, None, :]).reshape(n, -1)]
    lp = np.log(params["pi"])[:, None] + e["logf"]
    m = lp.max(0)
    rows.append((m + np.log(np.exp(lp - m).sum(0)))[:, None])
    return np.concatenate(rows, axis=1)


def _segments(rows):
    """Block sums (CHUNK rows, in order), then segment sums (SEG blocks, in order)."""
    nb = -(-rows.shape[0] // CHUNK)
    blocks = np.zeros((nb, rows.shape[1]))
    for b in range(nb):
        for r in rows[b * CHUNK:(b + 1) * CHUNK]:
            blocks[b] += r
    ns = -(-nb // SEG)
    segs = np.zeros((ns, rows.shape[1]))
    for s in range(ns):
        for b in blocks[s * SEG:(s + 1) * SEG]:
            segs[s] += b
    return segs


def _ordered_sum(segs):
    out = np.zeros(segs.shape[1])
    for s in segs:
        out += s
    return out


class OracleShard:
    """The driver's engine interface over the FP64 oracle: rows [lo, hi) of y.  Its
    'segments' are the E-step's per-observation arrays of its rows (padded to the
    largest shard); reducing them reassembles the arrays of every row."""

    def __init__(self, oracle, y, lo, hi, bounds, params, spec):
        self.o, self.y, self.lo, self.hi, self.bounds, self.spec = oracle, y, lo, hi, bounds, spec
        self.params = {k: np.array(v, dtype=float) for k, v in params.items()}
        self.maxrows = max(b - a for a, b in bounds)

    def _pack(self, e):
        g = self.params["pi"].size
        n = self.hi - self.lo
        lp = np.log(self.params["pi"])[:, None] + e["logf"]
        m = lp.max(0)
        parts = [e["logf"].T, e["tau"].T, e["u"].T, e["elogu"].T,
                 e["eu"].transpose(1, 0, 2).reshape(n, -1), e["euu"].transpose(1, 0, 2, 3).reshape(n, -1),
                 (m + np.log(np.exp(lp - m).sum(0)))[:, None]]
        out = np.zeros((self.maxrows, sum(p.shape[1] for p in parts)))
        out[:n] = np.concatenate(parts, axis=1)
        return out

    def estep_segments(self):
        import torch

        e = self.o.estep(self.y[self.lo:self.hi], self.params, self.spec, nthreads=1)
        return torch.from_numpy(self._pack(e))

    def reduce_segments(self, allseg):
        a = allseg.numpy()
        g, q = self.params["pi"].size, self.params["Delta"].shape[-1]
        rows = np.concatenate([a[r * self.maxrows:r * self.maxrows + (hi - lo)]
                               for r, (lo, hi) in enumerate(self.bounds)])
        n = rows.shape[0]
        o, e = 0, {}
        for key, w in (("logf", g), ("tau", g), ("u", g), ("elogu", g)):
            e[key] = rows[:, o:o + w].T.copy()
            o += w
        e["eu"] = rows[:, o:o + g * q].reshape(n, g, q).transpose(1, 0, 2).copy()
        o += g * q
        e["euu"] = rows[:, o:o + g * q * q].reshape(n, g, q, q).transpose(1, 0, 2, 3).copy()
        o += g * q * q
        self.e = e
        total = 0.0
        for v in rows[:, o]:
            total += v
        return total

    def mstep(self):
        self.params, _ = self.o.mstep(self.y, self.e, self.params)

    def loglik_local(self):
        import torch

        return torch.tensor([self.o.loglik(self.y[self.lo:self.hi], self.params, self.spec, nthreads=1)],
                            dtype=torch.float64)

    def aitken(self, a, b, c, tol):
        return self.o.aitken_converged(a, b, c, tol)[0]


def _rank_main(rank, world, port, outdir):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import oracle

    oracle.build()
    grp = shard.TorchGroup.from_env("gloo")
    w = synth.make_workload("two_comp_p2", n=700)
    spec = oracle.qmc(**w["qmc"])
    bounds, per = shard.shard_bounds(w["n"], world, CHUNK * SEG)
    lo, hi = bounds[rank]
    # (a) statistics: this rank's segments, gathered in rank order (padded), summed in order
    e = oracle.estep(w["y"][lo:hi], w["init"], spec, nthreads=1)
    segs = _segments(_stats_rows(w["y"][lo:hi], w["init"], e))
    pad = np.zeros((per, segs.shape[1]))
    pad[:segs.shape[0]] = segs
    allseg = grp.gather([torch.from_numpy(pad)]).numpy()
    stats = _ordered_sum(allseg)
    # (b) the sharded fit with the oracle as each shard's engine
    eng = OracleShard(oracle, w["y"], lo, hi, bounds, w["init"], spec)
    it, hist = shard.sharded_fit([eng], grp.gather, 4)
    np.savez(os.path.join(outdir, f"rank{rank}.npz"), stats=stats, hist=hist, it=it,
             **{"p_" + k: v for k, v in eng.params.items()})
    grp.barrier()
    grp.close()


def test_gloo_two_ranks(tmp_path, oracle):
    import torch.multiprocessing as mp

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    world = 2
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn")
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    w = synth.make_workload("two_comp_p2", n=700)
    spec = oracle.qmc(**w["qmc"])
    # single process: the same segment reduction over all rows
    e = oracle.estep(w["y"], w["init"], spec, nthreads=1)
    rows = _stats_rows(w["y"], w["init"], e)
    ref = _ordered_sum(_segments(rows))
    for r in res:
        assert np.array_equal(r["stats"], ref)  # bit for bit
        np.testing.assert_allclose(r["stats"], rows.sum(0), rtol=1e-12, atol=1e-9)
    # both ranks hold identical fits, equal to the single-process oracle fit
    ref_p, ref_h, _ = oracle.fit(w["y"], w["init"], 4, spec)
    for r in res:
        assert int(r["it"]) == 4
        for k in ("pi", "mu", "Sigma", "Delta", "nu"):
            assert np.array_equal(r["p_" + k], res[0]["p_" + k])
            np.testing.assert_allclose(r["p_" + k], ref_p[k], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(r["hist"], ref_h, rtol=1e-12)
