"""Row-sharded EM over several processes, one GPU each.

The paper's parallel EM (Sec. 4) runs the per-component work of an iteration in
threads and collects the partial results once per iteration (Sec. 4.3).  Here
the observations are split by rows instead: every process holds a contiguous
range of rows, computes the sufficient statistics of eqs (18)-(22) for them,
and one all-gather per iteration gives every process the segment sums of every
shard; each process reduces them in rank order and runs the identical M-step,
so the parameters stay the same everywhere without a broadcast.

Shard boundaries are multiples of `cfust_rows_per_segment`, so the gathered
segments are exactly the segments of the whole problem and the reduction
reproduces the single-process statistics bit for bit (include/cfust.h).  Every
rank contributes the same number of segment rows (zero rows pad the shorter
last shard; adding +0.0 leaves a sum unchanged).

This module holds the plumbing only -- shard bounds, the exchange through
torch.distributed and the iteration order; every statistic, reduction and
M-step runs in the CUDA library, and the stopping rule is the library's
(cfust_aitken_converged).
"""
from __future__ import annotations

import math
import os

import numpy as np


def shard_bounds(n, world, rows_per_segment):
    """Row ranges [(lo, hi)] of the `world` shards of n observations, each starting
    on a multiple of rows_per_segment, and the segments per rank (the largest
    shard's count, the common padded count)."""
    if world < 1 or rows_per_segment < 1:
        raise ValueError("world and rows_per_segment must be positive")
    nseg = math.ceil(n / rows_per_segment)
    per = math.ceil(nseg / world)
    out = []
    for r in range(world):
        s0, s1 = min(r * per, nseg), min((r + 1) * per, nseg)
        out.append((min(s0 * rows_per_segment, n), min(s1 * rows_per_segment, n)))
    if any(hi <= lo for lo, hi in out):
        raise ValueError(f"n = {n} gives fewer than {world} segments of {rows_per_segment} rows: "
                         "too few observations to shard")
    return out, per


def sharded_fit(engines, gather, max_iter, tol=0.0):
    """The EM loop of cfust_fit over shards: per iteration every local engine
    enqueues its E-step segments, `gather` returns the segments of all shards in
    rank order, every engine reduces them (l(Psi^(k)) of eq (27)) and, unless
    Aitken's rule (eqs 24-26) stops the fit, runs its M-step.  Without
    convergence a density pass gives l(Psi^(max_iter)), summed over shards in
    rank order.  Returns (M-steps run, log-likelihood history), as cfust_fit.

    engines: this process's shards in rank order (one per process in a
    multi-process run; several in a single-process emulation);
    gather(list of local tensors) -> the rank-ordered concatenation over all
    processes."""
    hist = []
    it = 0
    converged = False
    for it in range(max_iter):
        allseg = gather([e.estep_segments() for e in engines])
        Ls = [e.reduce_segments(allseg) for e in engines]
        hist.append(Ls[0])
        if tol > 0 and it >= 2 and engines[0].aitken(hist[-3], hist[-2], hist[-1], tol):
            converged = True
            break
        for e in engines:
            e.mstep()
    if not converged:
        parts = gather([e.loglik_local() for e in engines])
        total = 0.0
        for v in parts.reshape(-1).tolist():  # rank order
            total += v
        hist.append(total)
        it = max_iter
    return it, np.array(hist)


class CudaShard:
    """One shard of the observations on this process's GPU: a library context
    over rows [lo, hi) and its padded segment buffer."""

    def __init__(self, cf, p, q, g, lo, hi, opts, y_rows, params, seg_per_rank, n_total):
        import torch

        self.cf, self.lo, self.hi, self.n_total = cf, lo, hi, n_total
        self.ctx = cf.cfust_create(p, q, g, hi - lo, opts)
        cf.cfust_set_data(self.ctx, y_rows)
        cf.cfust_set_params(self.ctx, params)
        nseg, width = cf.cfust_segment_count(self.ctx)
        if nseg > seg_per_rank:
            raise ValueError(f"shard has {nseg} segments, more than the {seg_per_rank} per rank")
        self.local = torch.zeros((seg_per_rank, width), dtype=torch.float64, device="cuda")

    def estep_segments(self):
        self.cf.cfust_estep_segments(self.ctx, self.local)
        return self.local

    def reduce_segments(self, allseg):
        return self.cf.cfust_reduce_segments(self.ctx, allseg, self.n_total)

    def mstep(self):
        self.cf.cfust_mstep(self.ctx)

    def loglik_local(self):
        import torch

        return torch.tensor([self.cf.cfust_loglik(self.ctx)], dtype=torch.float64, device="cuda")

    def aitken(self, a, b, c, tol):
        return self.cf.cfust_aitken_converged(a, b, c, tol)


class TorchGroup:
    """The exchange between processes: torch.distributed (NCCL between GPUs, gloo
    on host tensors), one process per rank."""

    def __init__(self, dist, rank, world):
        self.dist, self.rank, self.world = dist, rank, world

    @classmethod
    def from_env(cls, backend, local=None):
        import torch
        import torch.distributed as dist

        if not dist.is_initialized():
            kw = {}
            if backend == "nccl" and local is not None:
                kw["device_id"] = torch.device("cuda", local)
            dist.init_process_group(backend, **kw)
        return cls(dist, dist.get_rank(), dist.get_world_size())

    def gather(self, tensors):
        """All ranks' tensors (this rank's `tensors` concatenated first), in rank order."""
        import torch

        mine = torch.cat(tensors) if len(tensors) > 1 else tensors[0]
        out = [torch.empty_like(mine) for _ in range(self.world)]
        self.dist.all_gather(out, mine)
        return torch.cat(out)

    def barrier(self):
        self.dist.barrier()

    def max_over_ranks(self, x):
        import torch

        dev = "cuda" if self.dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist.is_initialized():
            self.dist.destroy_process_group()

    # ---- the benchmark's view: this rank's rows and one EM iteration as a step ----
    def rows(self, n, cf, w, opts):
        rps = cf.cfust_rows_per_segment(w["p"], w["q"], w["g"], opts.precision)
        bounds, self.seg_per_rank = shard_bounds(n, self.world, rps)
        return bounds[self.rank]

    def make_fit(self, cf, w, opts, y_rows):
        lo, hi = self.rows(w["n"], cf, w, opts)
        eng = CudaShard(cf, w["p"], w["q"], w["g"], lo, hi, opts, y_rows, w["init"], self.seg_per_rank, w["n"])
        group = self

        class Step:
            ctx = eng.ctx

            @staticmethod
            def step():
                L = eng.reduce_segments(group.gather([eng.estep_segments()]))
                eng.mstep()
                return L

        return Step


def world_from_env():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0"))
