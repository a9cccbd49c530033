"""Benchmark of the FM-CFUST EM hot path on GB300 (one JSON line on stdout).

A step is one EM iteration -- the E-step over every observation-component pair
with the tau-weighted sufficient statistics (Sec. 3.1, 3.2), then the M-step --
over the whole synthetic workload.  The default workload is `wide_p16`
(p = 16, q = 2, g = 8, n = 2,000,000 observations stored in FP32, drawn from
the latent hierarchy of eq (6)): the largest single-GPU configuration.  The
line reports, on that workload,
  - the chosen form (value, ms_per_step): the mixed-precision form (FP32
    whitening, integrals and compensated statistics; FP64 factorisations, tau,
    log-likelihood, M-step and nu);
  - `plain_gpu`: the plain method (moments by the T_{q-1}/T_{q-2} recursion,
    FP32 integrals, FP64 everything else) timed the same way;
  - `loglik_err`: each form's final log-likelihood and parameters after the
    same EM iterations on a sample of the workload, against the FP64 oracle fit
    in the same reading (computed in the CPU leg, before the GPU work);
  - `roofline`: the dominant kernel's counted algorithmic work per second
    (T_2 quadrature nodes, or lattice points) over the rate of the same
    per-unit arithmetic alone, measured on this GPU in this run
    (cfust_measure_rates);
  - `sub`: the same for flow_p4 (p = q = g = 4, n = 200,000; single-pass vs
    recursion moments), learned_p6 (p = q = g = 6, n = 1,000,000) and the batch
    of concurrent fits (cfust_fit_batch against the fit-by-fit loop).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--sub LIST]
  python bench.py --workload batch [--nfits 64 --starts 4]
  python bench.py --impl reference ...   (the FP64 CPU oracle, bounded sample)

Under torchrun (N > 1) the observations are split by rows across the ranks
and one all-gather of the per-segment statistics per iteration gives every
rank the same sums (paper_1606_02054_gb300.shard): strong scaling, value =
all pairs per second of the slowest rank.  Inputs are resident in HBM; L2
(129 MB) is flushed before every timed step.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

# concurrent fits of the batch workload use many streams: give them more
# hardware work queues than the default 8 (read when the CUDA context starts)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "E-step obs·comp/s and EM iter/s: chosen form vs plain GPU at stated loglik err"
UNIT = "obs·comp/s"

PRECISION_NOTE = {
    "fp64": "fp64 throughout",
    "fp32": "fp32 lattice/quadrature integrals; fp64 whitening, densities, tau, loglik, "
            "statistics, M-step",
    "mixed": "fp32 whitening, integrals and compensated statistics; fp64 factorisations, "
             "tau, loglik, M-step, nu",
}

# (chosen form, plain form) per workload; the plain method is the moment recursion with
# FP32 integrals and FP64 everything else
FORMS = {
    "wide_p16": (dict(label="mixed precision", precision="mixed", moments=1),
                 dict(label="plain: recursion moments, fp32 integrals, fp64 rest", precision="fp32", moments=0)),
    "flow_p4": (dict(label="single-pass moments, fp32 integrals", precision="fp32", moments=1),
                dict(label="plain: recursion moments, fp32 integrals, fp64 rest", precision="fp32", moments=0)),
    "learned_p6": (dict(label="single-pass moments, fp32 integrals", precision="fp32", moments=1),
                   dict(label="plain: recursion moments, fp32 integrals, fp64 rest", precision="fp32", moments=0)),
    "two_comp_p2": (dict(label="fp64", precision="fp64", moments=0),
                    dict(label="plain: fp64", precision="fp64", moments=0)),
}
Y32_WORKLOADS = ("wide_p16",)  # observations stored in FP32
# CPU samples (observations) and sample fits (observations, EM iterations) per workload,
# sized for a few seconds of oracle time on 16 host cores
CPU_SAMPLE = {"wide_p16": 20000, "flow_p4": 2000, "learned_p6": 120, "two_comp_p2": 1000}
REF_SAMPLE = {"wide_p16": 8000, "flow_p4": 400, "learned_p6": 40, "two_comp_p2": 1000}
FIT_SAMPLE = {"wide_p16": (1000, 8), "flow_p4": (200, 6), "learned_p6": (240, 3), "two_comp_p2": (1000, 20)}
# the oracle's recursion at q = 6 (38 lattice integrals per pair) is too slow for a sample fit
# inside the benchmark: there only the chosen form's fit is checked
FIT_CHOSEN_ONLY = ("learned_p6",)
# the plain recursion at p = q = g = 6 takes seconds per iteration (2 T_6 + 6 T_5 + 30 T_4
# lattice integrals per pair): one warm-up and one timed step
SUB_PLAIN_STEPS = {"learned_p6": 1}
# DRAM bytes per algorithmic unit of the dominant kernels, from ncu captures of this
# build (dram__bytes_read.sum + dram__bytes_write.sum of one launch / its units); None
# where no capture of the current kernel exists
TRAFFIC_PER_UNIT = {
    # t2_pieces_kernel<2, 1>, wide_p16 shape at n = 200,000 (mixed form, 8-32 nodes per piece
    # by its class, 64 graded): 115.28 MB read + 5.56 MB written for 83.24 M nodes; the
    # records (FP32 fields in, FP32 result out) scale with the nodes at any n
    ("level0_Tq", 2): (115.277056e6 + 5.564672e6) / 83239548,
    # lattice_mom_kernel_32<4, 0, 0, 2>, flow_p4 shape at n = 4,000: 1.07 MB read, nothing
    # written to DRAM, for 131.07 M lattice points (the records, 67 B each, scale with them)
    ("moments_Tq", 4): 1.070080e6 / 131072000,
}


class Clocks:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
            return
        # the sampler's start-up (driver queries) stays out of the timed region
        t0 = time.time()
        while not self.lines and self.proc.poll() is None and time.time() - t0 < 5.0:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names[1:], parts[5:9]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _prec(cf, name):
    return {"fp32": cf.CFUST_PREC_FP32, "fp64": cf.CFUST_PREC_FP64, "mixed": cf.CFUST_PREC_MIXED}[name]


def _opts(cf, w, form, profile=0, stream=None):
    q = w["qmc"]
    return cf.cfust_default_opts(precision=_prec(cf, form["precision"]), qmc_points=q["npoints"],
                                 qmc_shifts=q["nshifts"], qmc_korobov_a=q["korobov_a"],
                                 seed=q["seed"], profile=profile, cuda_stream=stream,
                                 moments=form["moments"])


def _y_store(w):
    """The observations as the workload stores them (FP32 for the wide workload)."""
    return np.ascontiguousarray(w["y"], dtype=np.float32 if w["name"] in Y32_WORKLOADS else np.float64)


def _form_name(w, form):
    m = "single-pass moments" if form["moments"] and w["q"] >= 3 else "moment recursion"
    return f"{form['label']} ({m}; {PRECISION_NOTE[form['precision']]})"


# ---------------------------------------------------------------------------
# CPU leg: the FP64 oracle (timed baseline, and the reference fits of every form)
# ---------------------------------------------------------------------------
def cpu_baseline(w, nsample, moments):
    """The FP64 oracle, as it stands, on the first `nsample` observations of the
    workload: one E-step + M-step (the same moment reading as the timed form)."""
    import oracle

    sub = _y_store(w)[:nsample].astype(np.float64)
    spec = oracle.qmc(**dict(w["qmc"], moments=moments))
    cores = os.cpu_count() or 1
    params = {k: np.array(v, dtype=float) for k, v in w["init"].items()}
    t0 = time.perf_counter()
    e = oracle.estep(sub, params, spec, nthreads=cores)
    oracle.mstep(sub, e, params)
    dt = time.perf_counter() - t0
    return {"value": nsample * w["g"] / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {nsample} of {w['n']} observations of {w['name']}, one E-step + "
                      f"M-step in FP64 on {cores} host threads",
            "ms_per_step": dt * 1e3}


def oracle_fits(w, forms, nsample, iters):
    """Oracle fits of the first `nsample` observations (as the workload stores them)
    from the workload's starting values, one per distinct moment reading."""
    import oracle

    y = _y_store(w)[:nsample].astype(np.float64)
    out = {}
    if w["name"] in FIT_CHOSEN_ONLY:
        forms = forms[:1]
    for f in forms:
        m = f["moments"] if w["q"] >= 3 else 0
        if m not in out:
            ref, hist, _ = oracle.fit(y, w["init"], iters, oracle.qmc(**dict(w["qmc"], moments=m)),
                                      nthreads=os.cpu_count() or 1)
            out[m] = (ref, hist)
    return out


def fit_error(cf, w, form, refs, nsample, iters):
    """The GPU fit of the same sample in `form` against the oracle's."""
    m = form["moments"] if w["q"] >= 3 else 0
    ref, rhist = refs[m]
    ctx = cf.cfust_create(w["p"], w["q"], w["g"], nsample, _opts(cf, w, form))
    cf.cfust_set_data(ctx, _y_store(w)[:nsample])
    cf.cfust_set_params(ctx, w["init"])
    _, hist = cf.cfust_fit(ctx, iters)
    got = cf.cfust_get_params(ctx)
    perr = max(float(np.linalg.norm(np.atleast_1d(got[k][h] - ref[k][h])) /
                     max(float(np.linalg.norm(np.atleast_1d(ref[k][h]))), 1e-300))
               for k in ("pi", "mu", "Sigma", "Delta", "nu") for h in range(w["g"]))
    return {"loglik_rel_err": abs(hist[-1] - rhist[-1]) / abs(rhist[-1]), "param_rel_err": perr,
            "loglik_gpu": float(hist[-1]), "loglik_oracle": float(rhist[-1]),
            "sample": f"first {nsample} observations, {iters} EM iterations from the same start, "
                      f"oracle in the same moment reading and lattice"}


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
def measure(cf, torch, w, form, y_dev, flush, stream, steps, warmup, with_clocks=False, shard=None):
    """`warmup` untimed, then `steps` timed EM iterations (CUDA events on the launching
    stream around each step, L2 flushed before each); the library's kernel profile and
    algorithmic work counts of the timed steps."""
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if shard is not None:
        fit = shard.make_fit(cf, w, _opts(cf, w, form, profile=1, stream=stream.cuda_stream), y_dev)
        step = fit.step
        ctx = fit.ctx
    else:
        ctx = cf.cfust_create(w["p"], w["q"], w["g"], w["n"],
                              _opts(cf, w, form, profile=1, stream=stream.cuda_stream))
        cf.cfust_set_data(ctx, y_dev)
        cf.cfust_set_params(ctx, w["init"])

        def step():
            L = cf.cfust_estep(ctx)
            cf.cfust_mstep(ctx)
            return L

    # the integrators' launch shapes for this workload, timed on its own records (untimed)
    tuned = cf.cfust_autotune(ctx, reps=2)[0]
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    cf.cfust_profile(ctx, reset=True)
    n0 = cf.cfust_launch_count(ctx)
    clocks = Clocks(local) if with_clocks else None
    if clocks:
        clocks.start()
    if shard is not None:
        shard.barrier()
    torch.cuda.synchronize()
    total_ms, lls, each = 0.0, [], []
    for _ in range(steps):
        flush.fill_(1.0)  # evict L2 before each timed step
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lls.append(step())
        e1.record(stream)
        e1.synchronize()
        each.append(e0.elapsed_time(e1))
        total_ms += each[-1]
    torch.cuda.synchronize()
    if shard is not None:
        shard.barrier()
    clk = clocks.stop() if clocks else None
    ms = total_ms / steps
    if shard is not None:
        ms = shard.max_over_ranks(ms)
    prof = cf.cfust_profile(ctx)
    work = cf.cfust_profile_work(ctx)
    estep_ms = sum(v[0] for k, v in prof.items() if k != "mstep") / steps
    each.sort()
    spread = {"min": each[0], "median": each[len(each) // 2], "max": each[-1]}
    return dict(ms=ms, estep_ms=estep_ms, prof=prof, work=work, ll=lls[-1], clk=clk, spread=spread,
                launches=cf.cfust_launch_count(ctx) - n0, ctx=ctx, tuned=tuned)


def roofline(w, run, rates):
    """The dominant integrator class of a run: counted algorithmic units per second
    (lattice points, T_2 quadrature nodes) over the measured rate of the same per-unit
    arithmetic alone (cfust_measure_rates)."""
    prof, work = run["prof"], run["work"]
    classes = [k for k in ("level0_Tq", "level1_Tq-1", "level2_Tq-2", "moments_Tq")
               if prof[k][1] > 0 and work[k] > 0]
    if not classes:
        return None
    dom = max(classes, key=lambda k: prof[k][0])
    ms_launch = prof[dom][0] / prof[dom][1]
    units_launch = work[dom] / prof[dom][1]
    dims = {"level0_Tq": w["q"], "level1_Tq-1": w["q"] - 1, "level2_Tq-2": w["q"] - 2, "moments_Tq": w["q"]}
    k = dims[dom]
    if k == 2:
        unit, peak_rate = "T_2 quadrature node", rates.get("t2_nodes")
        basis = ("cfust_measure_rates t2_nodes: the FP32 T_2 node alone (two sines, sin^(nu-1), "
                 "tabulated inner T_1), measured on this GPU in this run")
    else:
        unit, peak_rate = "lattice point", rates.get("mix_points", {}).get(k)
        basis = (f"cfust_measure_rates mix_points[{k}]: the single-pass integrand of dimension {k} "
                 f"alone ({k} Phi, {k} Phi^-1, {k * (k - 1) // 2 + 3 * k} + {2 + k + k * (k + 1) // 2} FMA "
                 f"per point), measured on this GPU in this run")
        if dom != "moments_Tq":
            basis += " (an upper bound of the plain T_k integrand's rate: it has one Phi^-1 and the moment sums more)"
    achieved = units_launch / (ms_launch / 1e3) / 1e9
    peak = peak_rate / 1e9 if peak_rate else None
    tb = TRAFFIC_PER_UNIT.get((dom, k))
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": f"G{unit.split()[-1]}s/s",
            "frac": achieved / peak if peak else None,
            "traffic": tb * units_launch if tb else None,
            "kernel": dom, "k": k, "unit_of_work": unit, "units_per_launch": units_launch,
            "ms_per_launch": ms_launch, "peak_basis": basis}


def form_summary(w, run, pairs, world):
    return {"value": pairs / (run["ms"] / 1e3), "unit": UNIT, "ms_per_step": run["ms"],
            "steps": run["steps"], "warmup": run["warmup"], "launch_shapes": run["tuned"],
            "em_iter_per_s": 1e3 / run["ms"], "step_ms_spread": run["spread"],
            "estep_obs_comp_per_s": pairs / (run["estep_ms"] / 1e3),
            "loglik_last": run["ll"], "gpu_launches": int(run["launches"]),
            "kernel_ms_per_step": {k: v[0] / max(1, run["steps"]) for k, v in run["prof"].items()}}


def run_workload(cf, torch, name, args, stream, flush, steps, warmup, with_clocks, refs, fitcfg,
                 rates, shard=None, w=None, plain_steps=None, plain_warmup=None):
    """Chosen and plain forms of one workload, each with its fit error."""
    from paper_1606_02054_gb300 import synth

    if w is None:
        w = synth.make_workload(name)
        w["name"] = name
    chosen, plain = FORMS[name]
    ydt = torch.float32 if name in Y32_WORKLOADS else torch.float64
    if shard is not None:
        lo, hi = shard.rows(w["n"], cf, w, _opts(cf, w, chosen))
        y_dev = torch.tensor(_y_store(w)[lo:hi], dtype=ydt, device="cuda")
    else:
        y_dev = torch.tensor(_y_store(w), dtype=ydt, device="cuda")
    pairs = w["n"] * w["g"]
    runs = {}
    for key, form in (("chosen", chosen), ("plain", plain)):
        st = steps if key == "chosen" or plain_steps is None else plain_steps
        wu = warmup if key == "chosen" or plain_warmup is None else plain_warmup
        r = measure(cf, torch, w, form, y_dev, flush, stream, st, wu,
                    with_clocks=with_clocks and key == "chosen", shard=shard)
        r["steps"], r["warmup"] = st, wu
        runs[key] = r
    out = {"workload": name, "n": w["n"], "p": w["p"], "q": w["q"], "g": w["g"],
           "qmc": f"{w['qmc']['npoints']}x{w['qmc']['nshifts']}"}
    for key, form in (("chosen", chosen), ("plain", plain)):
        s = form_summary(w, runs[key], pairs, 1)
        s["form"] = _form_name(w, form)
        s["roofline"] = roofline(w, runs[key], rates) if key == "chosen" else None
        if refs is not None and (form["moments"] if w["q"] >= 3 else 0) in refs:
            ns, it = fitcfg
            s["loglik_err"] = fit_error(cf, w, form, refs, ns, it)
        out[key] = s
    out["speedup_of_chosen"] = runs["plain"]["ms"] / runs["chosen"]["ms"]
    return out, runs, w, y_dev


def run_batch(args, cf, torch, stream, flush, with_clocks=False, steps=None, warmup=None):
    """Batched fits (p = q uniform on 2..8, g on 2..6, n log-uniform on 1e3..1e5): every
    fit's EM loop is one device-controlled CUDA graph and all fits run concurrently
    (cfust_fit_batch).  One step = one EM iteration of every fit; value = sum over fits
    of n*g per second.  The same iteration run fit by fit through cfust_estep /
    cfust_mstep is timed beside it."""
    from paper_1606_02054_gb300 import synth

    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    B = synth.make_batch(nfits=args.nfits, starts=args.starts)
    qmc = B["qmc"]
    ctxs, pairs, shapes_of = [], 0, []
    for f in B["fits"]:
        for st in f["starts"]:
            shapes_of.append((f["p"], f["g"], f["n"]))
            o = cf.cfust_default_opts(precision=cf.CFUST_PREC_FP32, qmc_points=qmc["npoints"],
                                      qmc_shifts=qmc["nshifts"], qmc_korobov_a=qmc["korobov_a"],
                                      seed=qmc["seed"], moments=1)
            c = cf.cfust_create(f["p"], f["q"], f["g"], f["n"], o)
            cf.cfust_set_data(c, f["y"])
            cf.cfust_set_params(c, st)
            ctxs.append(c)
            pairs += f["n"] * f["g"]

    # launch shapes: the library keeps one choice per (kernel, record dimension, precision),
    # so one tuning run per dimension q (= p here), on that dimension's largest fit; the
    # other fits take it when their graphs are captured (first batch call)
    largest = {}
    for c, (p_, g_, n_) in zip(ctxs, shapes_of):
        if p_ not in largest or n_ * g_ > largest[p_][1]:
            largest[p_] = (c, n_ * g_)
    t_tune = time.perf_counter()
    for c, _ in largest.values():
        cf.cfust_autotune(c, reps=1)
    tuned = len(largest)
    t_tune = time.perf_counter() - t_tune

    def batched():
        it, hist, status = cf.cfust_fit_batch(ctxs, 1, 0.0, flags=cf.CFUST_FIT_NO_FINAL)
        return int(np.sum(status != cf.CFUST_OK))

    def sequential():
        bad = 0
        for c in ctxs:
            try:
                cf.cfust_estep(c)
                cf.cfust_mstep(c)
            except cf.CfustError:
                bad += 1
        return bad

    def timed(fn, nsteps, clocked):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        n0 = sum(cf.cfust_launch_count(c) for c in ctxs)
        clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0"))) if clocked else None
        if clocks:
            clocks.start()
        per, failed = [], 0
        for _ in range(nsteps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            failed += fn()
            torch.cuda.synchronize()
            per.append((time.perf_counter() - t0) * 1e3)
        clk = clocks.stop() if clocks else None
        launches = sum(cf.cfust_launch_count(c) for c in ctxs) - n0
        return float(np.mean(per)), clk, launches, failed

    ms_b, clk, launches, failed_b = timed(batched, steps, with_clocks)
    ms_s, _, _, _ = timed(sequential, max(1, steps // 2), False)
    out = {"workload": "batch", "fits": len(ctxs), "problems": args.nfits, "starts": args.starts,
           "pairs_per_iteration": pairs, "p=q": "uniform 2..8", "g": "uniform 2..6",
           "n": "log-uniform 1e3..1e5", "n_total": int(sum(f["n"] for f in B["fits"])),
           "qmc": f"{qmc['npoints']}x{qmc['nshifts']}",
           "form": "single-pass moments, " + PRECISION_NOTE["fp32"],
           "step": "one EM iteration of every fit (cfust_fit_batch, max_iter 1, no final density pass)",
           "timing": "host clock around the synchronous batch call, device synchronised on both sides",
           "chosen": {"form": "batched: one device-controlled CUDA graph per fit, all fits concurrent",
                      "value": pairs / (ms_b / 1e3), "unit": UNIT, "ms_per_step": ms_b,
                      "gpu_launches": int(launches / steps), "failed_fits": failed_b // steps},
           "plain": {"form": "cfust_estep + cfust_mstep fit by fit on one stream",
                     "value": pairs / (ms_s / 1e3), "unit": UNIT, "ms_per_step": ms_s},
           "speedup_of_chosen": ms_s / ms_b,
           "autotune": {"contexts_tuned": tuned, "seconds": t_tune,
                        "note": "one cfust_autotune run per record dimension q, on its largest fit; "
                                "every other fit of that q takes its choice"}}
    return out, clk


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    nsample = args.ref_sample or REF_SAMPLE.get(w["name"], 200)
    chosen = FORMS[w["name"]][0]
    per = []
    for i in range(args.warmup + args.steps):
        b = cpu_baseline(w, nsample, chosen["moments"] if w["q"] >= 3 else 0)
        if i >= args.warmup:
            per.append(b["ms_per_step"])
    ms = float(np.mean(per))
    value = nsample * w["g"] / (ms / 1e3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": w["name"], "n": w["n"], "p": w["p"], "q": w["q"], "g": w["g"],
                       "qmc": f"{w['qmc']['npoints']}x{w['qmc']['nshifts']}",
                       "form": ("single-pass moments" if chosen["moments"] and w["q"] >= 3
                                else "moment recursion"),
                       "precision": "fp64 throughout (the CPU oracle)",
                       "parallelism": f"{cores} host threads (OpenMP over observations)",
                       "sample_n": nsample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"first {nsample} observations per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", default="wide_p16")
    ap.add_argument("--n", type=int, default=None, help="override the workload size")
    ap.add_argument("--sub", default="flow_p4,learned_p6,batch",
                    help="comma-separated workloads measured as sub-objects ('' for none)")
    ap.add_argument("--sub-steps", type=int, default=3)
    ap.add_argument("--sub-warmup", type=int, default=3)
    ap.add_argument("--ref-sample", type=int, default=None)
    ap.add_argument("--cpu-sample", type=int, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fit-check", action="store_true")
    ap.add_argument("--rates-seconds", type=float, default=1.5)
    ap.add_argument("--nfits", type=int, default=64, help="batch workload: problems")
    ap.add_argument("--starts", type=int, default=4, help="batch workload: starts per problem")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    subs = [s for s in args.sub.split(",") if s] if world == 1 else []

    if args.workload == "batch":
        if args.impl == "reference":
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the batch workload has no "
                                  "oracle leg; time the oracle on a single-fit workload"}))
            return
    from paper_1606_02054_gb300 import synth

    w = None
    if args.workload != "batch":
        w = synth.make_workload(args.workload, n=args.n)
        w["name"] = args.workload
    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return

    # CPU leg first (in-process OpenMP threads; no fork after CUDA initialisation): the
    # timed oracle baseline and the oracle fits every form's error is measured against
    cpu, refs, sub_w, sub_refs = None, None, {}, {}
    if rank == 0 and w is not None:
        chosen = FORMS[w["name"]][0]
        if not args.no_cpu_baseline:
            cpu = cpu_baseline(w, args.cpu_sample or CPU_SAMPLE.get(w["name"], 200),
                               chosen["moments"] if w["q"] >= 3 else 0)
        if not args.no_fit_check:
            refs = oracle_fits(w, FORMS[w["name"]], *FIT_SAMPLE[w["name"]])
        for s in subs:
            if s == "batch":
                continue
            ws = synth.make_workload(s)
            ws["name"] = s
            sub_w[s] = ws
            if not args.no_fit_check:
                sub_refs[s] = oracle_fits(ws, FORMS[s], *FIT_SAMPLE[s])

    import torch

    torch.cuda.set_device(local)
    shard = None
    if world > 1:
        from paper_1606_02054_gb300 import shard as shard_mod

        shard = shard_mod.TorchGroup.from_env("nccl", local)

    from paper_1606_02054_gb300 import build

    build.build()
    import paper_1606_02054_gb300 as cf

    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    rates = cf.cfust_measure_rates(local, args.rates_seconds)

    if w is None:  # the batch workload alone
        b, clk = run_batch(args, cf, torch, stream, flush, with_clocks=True)
        if rank == 0:
            line = {"metric": METRIC, "value": b["chosen"]["value"] * world, "unit": UNIT, "n_gpus": world,
                    "steps": args.steps, "warmup": args.warmup, "ms_per_step": b["chosen"]["ms_per_step"],
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                    "data": "synthetic", "config": {**{k: v for k, v in b.items() if k not in ("chosen", "plain")},
                                                     "l2": "flushed (256 MB write) before every timed step",
                                                     "parallelism": f"replicas x{world}"},
                    "gpu_launches": b["chosen"]["gpu_launches"], "clocks": clk,
                    "plain_gpu": b["plain"], "speedup_of_chosen": b["speedup_of_chosen"], "rates": rates}
            print(json.dumps(line), flush=True)
        return

    main_out, runs, w, y_dev = run_workload(cf, torch, w["name"], args, stream, flush, args.steps,
                                            args.warmup, True, refs, FIT_SAMPLE[w["name"]], rates,
                                            shard=shard, w=w)
    chosen_form = FORMS[w["name"]][0]
    run = runs["chosen"]
    ms = run["ms"]
    pairs = w["n"] * w["g"]
    value = pairs / (ms / 1e3)  # every rank's rows together: the whole problem

    # end to end through the C ABI with host buffers: each step copies the observations
    # and the parameters in, runs the EM iteration, and copies the parameters out
    e2e = None
    if not args.no_e2e and shard is None:
        p, q, g = w["p"], w["q"], w["g"]
        ctx2 = cf.cfust_create(p, q, g, w["n"], _opts(cf, w, chosen_form, stream=stream.cuda_stream))
        y_host = torch.from_numpy(_y_store(w)).pin_memory()
        params = {k: np.array(v, dtype=float) for k, v in w["init"].items()}
        pbytes = 8 * (g + g * p + g * p * p + g * p * q + g)

        def e2e_step(params):
            cf.cfust_set_data(ctx2, y_host)
            cf.cfust_set_params(ctx2, params)
            cf.cfust_estep(ctx2)
            cf.cfust_mstep(ctx2)
            return cf.cfust_get_params(ctx2)

        for _ in range(max(1, args.warmup)):
            params = e2e_step(params)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            params = e2e_step(params)
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        e2e = {"value": pairs / (e2e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(y_host.numel() * y_host.element_size() + pbytes),
               "d2h_bytes_per_step": int(pbytes + 8 + 4 + 4 * g), "ms_per_step": e2e_ms}
        del ctx2

    sub = {}
    for s in subs:
        torch.cuda.synchronize()
        if s == "batch":
            sub[s], _ = run_batch(args, cf, torch, stream, flush, steps=args.sub_steps, warmup=args.sub_warmup)
        else:
            sub[s], _, _, _ = run_workload(cf, torch, s, args, stream, flush, args.sub_steps, args.sub_warmup,
                                           False, sub_refs.get(s), FIT_SAMPLE[s], rates, w=sub_w.get(s),
                                           plain_steps=SUB_PLAIN_STEPS.get(s), plain_warmup=SUB_PLAIN_STEPS.get(s))
        torch.cuda.empty_cache()

    if rank == 0:
        ch = main_out["chosen"]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
                "vs_baseline": None,
                "dtype": "f64" if chosen_form["precision"] == "fp64" else "f32", "data": "synthetic",
                "config": {"workload": w["name"], "n": w["n"], "p": w["p"], "q": w["q"], "g": w["g"],
                           "qmc": main_out["qmc"], "form": ch["form"],
                           "y_storage": "fp32" if w["name"] in Y32_WORKLOADS else "fp64",
                           "l2": "flushed (256 MB write) before every timed step; inputs > L2",
                           "parallelism": (f"rows sharded over {world} ranks, one all-gather of the "
                                           f"segment statistics per iteration" if world > 1 else "1 GPU")},
                "em_iter_per_s": 1e3 / ms, "step_ms_spread": ch["step_ms_spread"],
                "estep_obs_comp_per_s": ch["estep_obs_comp_per_s"],
                "loglik_last": ch["loglik_last"],
                "gpu_launches": ch["gpu_launches"],
                "kernel_ms_per_step": ch["kernel_ms_per_step"],
                "roofline": ch["roofline"], "clocks": run["clk"], "e2e": e2e, "cpu_baseline": cpu,
                "loglik_err": ch.get("loglik_err"),
                "plain_gpu": main_out["plain"], "speedup_of_chosen": main_out["speedup_of_chosen"],
                "rates": rates, "sub": sub}
        print(json.dumps(line), flush=True)
    if shard is not None:
        shard.close()


if __name__ == "__main__":
    main()
