"""Benchmark of the FM-CFUST EM hot path on GB300 (one JSON line on stdout).

A step is one EM iteration (E-step over every observation-component pair with
the tau-weighted sufficient statistics, then the M-step) over the whole
synthetic workload `flow_p4`: p = q = g = 4 (the HSCT flow-cytometry shape),
n = 200,000 observations drawn from the latent hierarchy of eq (6), T_4 and
T_3 by the randomised lattice (1024 points x 8 shifts).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64|mixed]
  python bench.py --workload wide_p16 --precision mixed   (p = 16, q = 2, g = 8, n = 2e6)
  python bench.py --workload batch [--nfits 64 --starts 4] (concurrent graph-driven fits)
  python bench.py --impl reference ...   (the FP64 CPU oracle, bounded sample)

value: observation-component pairs per second of whole EM iterations, summed
over ranks (each rank runs its own replica: weak scaling).  Inputs are
resident in HBM; L2 (129 MB) is flushed before every timed step.
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
# Executed thread-instructions per unit of work of the FP32 integrators
# (smsp__inst_executed.sum x smsp__thread_inst_executed_per_inst_executed.ratio
# / units) from the ncu captures summarised in profiles/lattice_fp32_flow_p4.md,
# profiles/moments_fp32_flow_p4.md and profiles/t2_mixed_wide_p16.md.  Lattice
# kernels count per lattice point (records x N x M; the same kernels run in the
# fp32 and mixed forms), the T_2 quadrature per record (its node count depends
# on the precision form, so the key names it).
INSTR_PER_UNIT = {("lattice", 4): 188.8, ("moments", 4): 219.5, ("t2", 2, "mixed"): 14128.0}
# DRAM bytes per integral record in the same captures (dram__bytes_read.sum +
# dram__bytes_write.sum of the launch / its records: 16,000 records of each
# lattice kind at flow_p4 n = 4,000; 320,000 T_2 records at wide_p16 n = 20,000);
# the records dominate, so traffic scales with the record count.
INTEG_TRAFFIC_BYTES_PER_RECORD = {("lattice", 4): 797440 / 16000, ("moments", 4): 1091072 / 16000,
                                  ("t2", 2, "mixed"): 11594752 / 320000}


def _unit_key(kind, k, precision):
    if precision == "fp64":
        return None
    return (kind, k, precision) if kind == "t2" else (kind, k)


PRECISION_NOTE = {
    "fp64": "fp64 throughout",
    "fp32": "fp32 lattice/quadrature integrals; fp64 whitening, densities, tau, loglik, "
            "statistics, M-step",
    "mixed": "fp32 whitening, integrals and compensated statistics; fp64 factorisations, "
             "tau, loglik, M-step, nu",
}
SM_COUNT = 152
LANES_PER_SM = 128  # 4 sub-partitions x 32 lanes, one instruction per lane per clock


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


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


def _opts(cf, w, precision, profile=0, stream=None, moments=1):
    q = w["qmc"]
    return cf.cfust_default_opts(precision=precision, qmc_points=q["npoints"],
                                 qmc_shifts=q["nshifts"], qmc_korobov_a=q["korobov_a"],
                                 seed=q["seed"], profile=profile,
                                 cuda_stream=stream, moments=moments)


def cpu_baseline(w, nsample, steps=1, moments=1):
    """The FP64 oracle, as it stands, on `nsample` observations of the workload
    (same moment reading as the timed GPU form)."""
    import oracle

    sub = w["y"][:nsample]
    spec = oracle.qmc(**dict(w["qmc"], moments=moments))
    cores = os.cpu_count() or 1
    params = {k: np.array(v, dtype=float) for k, v in w["init"].items()}
    t0 = time.perf_counter()
    ll0 = None
    for _ in range(steps):
        e = oracle.estep(sub, params, spec, nthreads=cores)
        ll0 = e["loglik"] if ll0 is None else ll0
        params, _ = oracle.mstep(sub, e, params)
    dt = (time.perf_counter() - t0) / steps
    return {"value": nsample * w["g"] / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {nsample} of {w['n']} observations of {w['name']}, "
                      f"E-step + M-step in FP64 on {cores} host threads, {steps} step(s)",
            "ms_per_step": dt * 1e3, "loglik_at_start": ll0}


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    nsample = args.ref_sample
    per = []
    for i in range(args.warmup + args.steps):
        b = cpu_baseline(w, nsample, 1, 1 if args.moments == "single-pass" else 0)
        if i >= args.warmup:
            per.append(b["ms_per_step"])
    ms = float(np.mean(per))
    value = nsample * w["g"] / (ms / 1e3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": w["name"], "n": w["n"], "p": w["p"], "q": w["q"], "g": w["g"],
                       "qmc": f"{w['qmc']['npoints']}x{w['qmc']['nshifts']}",
                       "form": ("single-pass moments" if args.moments == "single-pass" and w["q"] >= 3
                                else "moment recursion"),
                       "precision": "fp64 throughout (the CPU oracle)",
                       "parallelism": f"{cores} host threads (OpenMP over observations)",
                       "sample_n": nsample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"first {nsample} observations per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(args, rank, world):
    """Batched fits (p = q uniform on 2..8, g on 2..6, n log-uniform on 1e3..1e5): every
    fit's EM loop is one device-controlled CUDA graph and all fits run concurrently
    (cfust_fit_batch).  One step = one EM iteration of every fit; value = sum over fits
    of n*g per second.  The same iteration run fit by fit through cfust_estep /
    cfust_mstep is timed beside it."""
    import torch

    from paper_1606_02054_gb300 import build, synth

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build.build()
    import paper_1606_02054_gb300 as cf

    prec = {"fp32": cf.CFUST_PREC_FP32, "fp64": cf.CFUST_PREC_FP64,
            "mixed": cf.CFUST_PREC_MIXED}[args.precision]
    moments = 1 if args.moments == "single-pass" else 0
    B = synth.make_batch(nfits=args.nfits, starts=args.starts)
    qmc = B["qmc"]
    ctxs, pairs = [], 0
    for f in B["fits"]:
        for st in f["starts"]:
            o = cf.cfust_default_opts(precision=prec, qmc_points=qmc["npoints"],
                                      qmc_shifts=qmc["nshifts"], qmc_korobov_a=qmc["korobov_a"],
                                      seed=qmc["seed"], moments=moments)
            c = cf.cfust_create(f["p"], f["q"], f["g"], f["n"], o)
            cf.cfust_set_data(c, f["y"])
            cf.cfust_set_params(c, st)
            ctxs.append(c)
            pairs += f["n"] * f["g"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

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

    def timed(fn, steps, with_clocks):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        n0 = sum(cf.cfust_launch_count(c) for c in ctxs)
        clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0"))) if with_clocks else None
        if clocks:
            clocks.start()
        per, failed = [], 0
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            failed += fn()
            torch.cuda.synchronize()
            per.append((time.perf_counter() - t0) * 1e3)
        clk = clocks.stop() if clocks else None
        launches = sum(cf.cfust_launch_count(c) for c in ctxs) - n0
        return float(np.mean(per)), clk, launches, failed

    ms_b, clk, launches, failed_b = timed(batched, args.steps, True)
    ms_s, _, launches_s, failed_s = timed(sequential, max(1, args.steps // 2), False)
    if rank != 0:
        return
    shapes = sorted({(f["p"], f["g"]) for f in B["fits"]})
    line = {"metric": METRIC, "value": pairs * world / (ms_b / 1e3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": "batch", "fits": len(ctxs), "problems": args.nfits,
                       "starts": args.starts, "pairs_per_iteration": pairs,
                       "p=q": "uniform 2..8",
                       "g": "uniform 2..6", "n": "log-uniform 1e3..1e5",
                       "n_total": int(sum(f["n"] for f in B["fits"])),
                       "qmc": f"{qmc['npoints']}x{qmc['nshifts']}",
                       "form": "single-pass moments" if moments else "moment recursion",
                       "precision": PRECISION_NOTE[args.precision],
                       "step": "one EM iteration of every fit (cfust_fit_batch, max_iter 1, "
                               "no final density pass)",
                       "timing": "host clock around the synchronous batch call, device "
                                 "synchronised on both sides",
                       "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": f"replicas x{world}"},
            "gpu_launches": int(launches / args.steps), "failed_fits": failed_b // args.steps,
            "clocks": clk,
            "sequential": {"form": "cfust_estep + cfust_mstep fit by fit on one stream",
                           "value": pairs * world / (ms_s / 1e3), "unit": UNIT,
                           "ms_per_step": ms_s,
                           "speedup_of_batched": ms_s / ms_b},
            "distinct_shapes_pg": len(shapes)}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", default="flow_p4")
    ap.add_argument("--n", type=int, default=None, help="override the workload size")
    ap.add_argument("--precision", choices=["fp32", "fp64", "mixed"], default="fp32")
    ap.add_argument("--moments", choices=["single-pass", "recursion"], default="single-pass",
                    help="truncated-t moments of the timed form (the plain recursion is "
                         "also timed when single-pass is chosen)")
    ap.add_argument("--ref-sample", type=int, default=160)
    ap.add_argument("--cpu-sample", type=int, default=240)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nfits", type=int, default=64, help="batch workload: problems")
    ap.add_argument("--starts", type=int, default=4, help="batch workload: starts per problem")
    ap.add_argument("--surrogate", action="store_true",
                    help="learned surrogate form (single-pass moments, q >= 3): train at the start "
                         "values (untimed), then time E-steps through the network")
    ap.add_argument("--surrogate-refresh", type=int, default=5,
                    help="surrogate form: every R-th step is a lattice E-step that also fine-tunes "
                         "the network on its records (timed); 0: never")
    ap.add_argument("--surrogate-refresh-epochs", type=int, default=4)
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.workload == "batch":
        if args.impl == "gpu":
            run_batch(args, rank, world)
        elif rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the batch workload has no "
                              "oracle leg; time the oracle on a single-fit workload"}))
        return

    from paper_1606_02054_gb300 import synth

    w = synth.make_workload(args.workload, n=args.n)
    w["name"] = args.workload

    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return

    import torch

    # CPU baseline first (in-process OpenMP threads; no fork after CUDA init)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.cpu_sample, 1, 1 if args.moments == "single-pass" else 0)

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1606_02054_gb300 import build

    build.build()
    import paper_1606_02054_gb300 as cf

    prec = {"fp32": cf.CFUST_PREC_FP32, "fp64": cf.CFUST_PREC_FP64,
            "mixed": cf.CFUST_PREC_MIXED}[args.precision]
    stream = torch.cuda.current_stream()
    # the wide workload stores its observations in FP32
    y_dtype = torch.float32 if w["name"] == "wide_p16" else torch.float64
    y_dev = torch.tensor(w["y"], dtype=y_dtype, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    pairs = w["n"] * w["g"]

    def measure(moments, with_clocks, surrogate=False):
        """warm-up, then `steps` timed EM iterations (CUDA events per step, L2
        flushed before each); returns timings and the library's kernel profile."""
        ctx = cf.cfust_create(w["p"], w["q"], w["g"], w["n"],
                              _opts(cf, w, prec, profile=1, stream=stream.cuda_stream,
                                    moments=moments))
        cf.cfust_set_data(ctx, y_dev)
        cf.cfust_set_params(ctx, w["init"])
        sur = None
        if surrogate:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ll_lat, losses = cf.cfust_surrogate_train(ctx)
            torch.cuda.synchronize()
            t_train = time.perf_counter() - t0
            ll_sur = cf.cfust_loglik(ctx)  # the density pass through the network, same Psi
            o = cf.cfust_surrogate_default_opts()
            sur = {"train_s": t_train, "epochs": o.epochs, "batch": o.batch,
                   "samples_per_epoch": o.samples_per_epoch, "loss_first": float(losses[0]),
                   "loss_last": float(losses[-1]), "loglik_lattice_at_start": ll_lat,
                   "loglik_surrogate_at_start": ll_sur,
                   "loglik_rel_err_at_start": abs(ll_sur - ll_lat) / abs(ll_lat)}

        count = [0]
        ft = cf.cfust_surrogate_default_opts(epochs=args.surrogate_refresh_epochs) if surrogate else None

        def step():
            R = args.surrogate_refresh
            if surrogate and R > 0 and count[0] > 0 and count[0] % R == 0:
                L, _ = cf.cfust_surrogate_train(ctx, ft)  # a lattice E-step, then fine-tuning
            else:
                L = cf.cfust_estep(ctx)
            cf.cfust_mstep(ctx)
            count[0] += 1
            return L

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        cf.cfust_profile(ctx, reset=True)
        n0 = cf.cfust_launch_count(ctx)
        clocks = Clocks(local) if with_clocks else None
        if clocks:
            clocks.start()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        total_ms, lls = 0.0, []
        for _ in range(args.steps):
            flush.fill_(1.0)  # evict L2 before each timed step
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lls.append(step())
            e1.record(stream)
            e1.synchronize()
            total_ms += e0.elapsed_time(e1)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clk = clocks.stop() if clocks else None
        launches = cf.cfust_launch_count(ctx) - n0
        prof = cf.cfust_profile(ctx)
        ms = total_ms / args.steps
        if dist:
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        estep_ms = sum(v[0] for k, v in prof.items() if k != "mstep") / args.steps
        if sur is not None:
            recs, fb = cf.cfust_surrogate_info(ctx)
            sur["fallback_fraction_last_surrogate_step"] = fb / max(recs, 1)
            sur["refresh_every"] = args.surrogate_refresh
            sur["refresh_epochs"] = args.surrogate_refresh_epochs
            cf.cfust_surrogate_use(ctx, 0)
        # l at the final parameters by the lattice density pass (the same yardstick for every form)
        ll_final = cf.cfust_loglik(ctx) if args.surrogate else None
        return dict(ll_final=ll_final, ms=ms, prof=prof, launches=launches, ll=lls[-1], clk=clk, estep_ms=estep_ms, sur=sur)

    chosen_moments = 1 if args.moments == "single-pass" else 0
    if args.surrogate and not (chosen_moments == 1 and w["q"] >= 3):
        raise SystemExit("--surrogate needs single-pass moments and q >= 3")
    main_run = measure(chosen_moments, True, surrogate=args.surrogate)
    plain_run = measure(0, False) if chosen_moments == 1 and w["q"] >= 3 and not args.surrogate else None
    lattice_run = measure(chosen_moments, False) if args.surrogate else None
    ms, prof, clk = main_run["ms"], main_run["prof"], main_run["clk"]
    launches = main_run["launches"]
    value = pairs * world / (ms / 1e3)

    # dominant kernel class and its roofline
    cls = {"level0_Tq": (w["q"], 1 if chosen_moments and w["q"] >= 3 else 2),
           "level1_Tq-1": (w["q"] - 1, w["q"]),
           "level2_Tq-2": (w["q"] - 2, w["q"] * (w["q"] - 1)),
           "moments_Tq": (w["q"], 1)}
    lat_classes = [k for k in cls if prof[k][1] > 0 and cls[k][0] >= 2]
    dom = max(lat_classes, key=lambda k: prof[k][0])
    dom_ms_per_launch = prof[dom][0] / prof[dom][1]
    kdim, mult = cls[dom]
    kind = "moments" if dom == "moments_Tq" else ("t2" if kdim == 2 else "lattice")
    records = pairs * mult
    units = records * (w["qmc"]["npoints"] * w["qmc"]["nshifts"] if kind != "t2" else 1)
    unit_name = "record" if kind == "t2" else "lattice point"
    f_sm = (clk.get("sm_mhz") or _peaks().get("sm_max_mhz", 2070.0)) * 1e6
    key = _unit_key(kind, kdim, args.precision)
    ipu = INSTR_PER_UNIT.get(key) if key else None
    secs = dom_ms_per_launch / 1e3
    if args.surrogate and prof["surrogate"][1] > 0:
        # the network's inference kernel: one launch per record set (n g records), a dense
        # BF16 contraction; algorithmic FLOPs of the used widths (nin -> 256 -> 256 -> 256 -> nout)
        q = w["q"]
        nin, nout = q + q * (q - 1) // 2 + 1, 1 + q + q * (q + 1) // 2
        flops_rec = 2 * (nin * 256 + 2 * 256 * 256 + 256 * nout)
        ms_l = prof["surrogate"][0] / prof["surrogate"][1]
        achieved = flops_rec * pairs / (ms_l / 1e3) / 1e12
        peak = _peaks().get("bf16_tflops")
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if peak else None, "traffic": None,
                "kernel": "mlp_infer_kernel", "flops_per_record": flops_rec, "records_per_launch": pairs,
                "ms_per_launch": ms_l,
                "peak_basis": "MEASURED_PEAKS.json bf16_tflops (burst, cuBLAS 8192^3) of measured",
                "note": "mma.sync m16n8k16 BF16 (legacy tensor path), weights staged per layer in shared memory"}
    elif ipu:
        achieved = ipu * units / secs / 1e12
        peak = SM_COUNT * LANES_PER_SM * f_sm / 1e12
        tb = INTEG_TRAFFIC_BYTES_PER_RECORD.get(key)
        roof = {"bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "Tinst/s", "frac": achieved / peak,
                "traffic": tb * records if tb else None,
                "kernel": dom, "k": kdim, "units_per_launch": units, "unit_of_work": unit_name,
                "inst_per_unit": ipu, "g_units_per_s": units / secs / 1e9,
                "ms_per_launch": dom_ms_per_launch,
                "peak_basis": "152 SMs x 128 lanes x 1 thread-instruction/clock at the sampled "
                              "median SM clock (issue-slot ceiling)"}
    else:
        roof = {"bound": "alu", "achieved": units / secs / 1e9, "peak": None,
                "unit": f"G{unit_name.split()[-1]}s/s", "frac": None, "traffic": None,
                "kernel": dom, "k": kdim, "units_per_launch": units, "unit_of_work": unit_name,
                "ms_per_launch": dom_ms_per_launch,
                "note": "no instruction count measured for this kernel and precision"}

    # the stated loglik error: the GPU's E-step l on the CPU baseline's sample (same
    # observations, starting values and lattice) against the oracle's
    ll_check = None
    if cpu is not None and cpu.get("loglik_at_start") is not None:
        ns = args.cpu_sample
        cchk = cf.cfust_create(w["p"], w["q"], w["g"], ns, _opts(cf, w, prec, moments=chosen_moments))
        cf.cfust_set_data(cchk, np.ascontiguousarray(w["y"][:ns]))
        cf.cfust_set_params(cchk, w["init"])
        lg = cf.cfust_estep(cchk)
        lo = cpu["loglik_at_start"]
        ll_check = {"rel_err": abs(lg - lo) / abs(lo), "gpu": lg, "oracle": lo,
                    "sample": f"first {ns} observations at the starting values, same lattice"}

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        p, q, g = w["p"], w["q"], w["g"]
        ctx2 = cf.cfust_create(p, q, g, w["n"], _opts(cf, w, prec, stream=stream.cuda_stream,
                                                      moments=chosen_moments))
        # pinned host copy in the workload's storage type (FP32 for the wide workload)
        y_host = torch.from_numpy(np.ascontiguousarray(
            w["y"], dtype=np.float32 if w["name"] == "wide_p16" else np.float64)).pin_memory()
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
        if dist:
            t = torch.tensor([e2e_ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_ms = float(t.item())
        e2e = {"value": pairs * world / (e2e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(y_host.numel() * y_host.element_size() + pbytes),
               "d2h_bytes_per_step": int(pbytes + 8 + 4 + 4 * g), "ms_per_step": e2e_ms}

    if rank == 0:
        form = ("single-pass moments" if chosen_moments and w["q"] >= 3 else "moment recursion")
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
                "config": {"workload": w["name"], "n": w["n"], "p": w["p"], "q": w["q"],
                           "g": w["g"], "qmc": f"{w['qmc']['npoints']}x{w['qmc']['nshifts']}",
                           "form": form,
                           "precision": PRECISION_NOTE[args.precision],
                           "l2": "flushed (256 MB write) before every timed step",
                           "parallelism": f"replicas x{world}"},
                "em_iter_per_s": 1e3 / ms,
                "estep_obs_comp_per_s": pairs * world / (main_run["estep_ms"] / 1e3),
                "loglik_last": main_run["ll"],
                "gpu_launches": int(launches),
                "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
                "roofline": roof, "clocks": clk, "e2e": e2e, "cpu_baseline": cpu,
                "loglik_check": ll_check}
        if main_run["sur"] is not None:
            line["config"]["form"] = ("learned surrogate (BF16 MLP, lattice fallback; every "
                                      f"{args.surrogate_refresh}th step a lattice E-step that fine-tunes it) "
                                      "+ single-pass moments")
            line["surrogate"] = main_run["sur"]
            line["gpu_launches_note"] = ("E- and M-step kernels; the refresh steps' training kernels "
                                         "(GEMMs, Adam) are not counted")
            line["surrogate"]["loglik_final_by_lattice"] = main_run["ll_final"]
            line["surrogate"]["loglik_final_lattice_form"] = lattice_run["ll_final"]
            line["surrogate"]["loglik_final_rel_diff"] = (abs(main_run["ll_final"] - lattice_run["ll_final"])
                                                          / abs(lattice_run["ll_final"]))
            line["lattice_gpu"] = {
                "form": "single-pass moments, lattice only", "value": pairs * world / (lattice_run["ms"] / 1e3),
                "unit": UNIT, "ms_per_step": lattice_run["ms"],
                "estep_obs_comp_per_s": pairs * world / (lattice_run["estep_ms"] / 1e3),
                "kernel_ms_per_step": {k: v[0] / args.steps for k, v in lattice_run["prof"].items()}}
        if plain_run:
            line["plain_gpu"] = {
                "form": "moment recursion (T_q, T_{q-1}, T_{q-2} records)",
                "value": pairs * world / (plain_run["ms"] / 1e3), "unit": UNIT,
                "ms_per_step": plain_run["ms"], "em_iter_per_s": 1e3 / plain_run["ms"],
                "estep_obs_comp_per_s": pairs * world / (plain_run["estep_ms"] / 1e3),
                "loglik_last": plain_run["ll"], "gpu_launches": int(plain_run["launches"]),
                "kernel_ms_per_step": {k: v[0] / args.steps for k, v in plain_run["prof"].items()}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
