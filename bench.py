#!/usr/bin/env python
"""Benchmark of the unbinned-likelihood hot path on GB300.

Workload (default): the 3D product model -- 10,000,000 events over (m, dE, t), signal
Gauss x Gauss x Exp plus background Argus x Poly2 x Exp, 12 free parameters, 128^3 midpoint
grid normalisation.  One step is one pass of the whole hot path: parameter upload, grid
normalisation, per-event evaluation, log, accumulation, adjoint gradient and the final
reduction, through goo_nll_grad with FP32 per-event arithmetic and compensated accumulation.
The FP64 plain form (goo_nll in float64) is timed beside it.

Prints ONE JSON line on rank 0.  With --impl reference it times the FP64 CPU oracle on
the host cores instead (bounded samples of the same workload).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_EVENTS = 10_000_000
GRID = 128
METRIC = "NLL evals/s (events/s) FP64 plain vs FP32+grad; toy fits/s, p50/p99 latency"
UNIT = "events/s"
BYTES_PER_EVENT_F32 = 12   # three float32 columns
BYTES_PER_EVENT_F64 = 24
# Counters of one launch of each timed kernel from one ncu capture (the profiles/ file named
# in "profile"): DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) and, for the FP64
# kernels, the FP64 pipe's active fraction (sm__pipe_fp64_cycles_active).  A record is used
# only while the kernel's sources still hash to the captured value; bytes scale with events.
_SOP_SRC = ['paper_1710_08826_gb300/csrc/tree.cu', 'paper_1710_08826_gb300/csrc/sop_kernels.cuh', 'paper_1710_08826_gb300/csrc/jit.cu', 'paper_1710_08826_gb300/csrc/common.cuh', 'paper_1710_08826_gb300/csrc/model.cuh']
_COH_SRC = ['paper_1710_08826_gb300/csrc/dalitz.cu', 'paper_1710_08826_gb300/csrc/dalitz.cuh', 'paper_1710_08826_gb300/csrc/common.cuh', 'paper_1710_08826_gb300/csrc/model.cuh']
_TD4_SRC = ['paper_1710_08826_gb300/csrc/td4.cu', 'paper_1710_08826_gb300/csrc/dalitz.cuh', 'paper_1710_08826_gb300/csrc/common.cuh', 'paper_1710_08826_gb300/csrc/model.cuh', 'paper_1710_08826_gb300/csrc/timeterms.cuh']
_TD3_SRC = _COH_SRC + ['paper_1710_08826_gb300/csrc/timeterms.cuh']
# warp-instruction issue peak of a GB300: 152 SMs x 4 schedulers x 2.07 GHz (one warp
# instruction per scheduler per cycle)
ISSUE_PEAK = 152 * 4 * 2.07e9

NCU_RECORDS = {
    "sop_nll_grad_f32": {"bytes": 127_851_008, "events": 10_000_000, "duration_ns": 40864, "warp_inst": 21_770_696, "issue_active": 0.5403,
        "sources": _SOP_SRC, "sha256": "510948a29bee9a77654bc84a7a3df5014e9aba8eb1fb4f7f3c6495b38be33291",
        "profile": "profiles/sop_event2_kernel_f32_c2_10M.md"},
    "sop_nll_f64": {"bytes": 243_686_912, "events": 10_000_000, "duration_ns": 2504160, "fp64_pipe": 0.8625, "fp64_ops": {"dfma": 649_995_818, "dadd": 340_076_105, "dmul": 259_998_770},
        "sources": _SOP_SRC, "sha256": "510948a29bee9a77654bc84a7a3df5014e9aba8eb1fb4f7f3c6495b38be33291",
        "profile": "profiles/sop_event_kernel_f64_c2_10M.md"},
    "coh_nll_grad_f32": {"bytes": 323_078_912, "events": 5_000_000, "duration_ns": 62912, "warp_inst": 30_962_164, "issue_active": 0.4583,
        "sources": _COH_SRC, "sha256": "e6dd74780f809bce3110cf47365aa77f11795ed20f00040bf6bdb22689ec5c10",
        "profile": "profiles/coh_nll_staged_kernel_f32_c3_5M.md"},
    "coh_nll_f64": {"bytes": 643_060_224, "events": 5_000_000, "duration_ns": 773056, "fp64_pipe": 0.8699, "fp64_ops": {"dfma": 165_155_649, "dadd": 135_077_825, "dmul": 105_000_000},
        "sources": _COH_SRC, "sha256": "e6dd74780f809bce3110cf47365aa77f11795ed20f00040bf6bdb22689ec5c10",
        "profile": "profiles/coh_nll_kernel_f64_c3_5M.md"},
    "coh_ls_mc_f32": {"bytes": 8_068_608, "events": 1_000_000, "duration_ns": 91424, "warp_inst": 65_097_718, "issue_active": 0.6327,
        "sources": _COH_SRC, "sha256": "e6dd74780f809bce3110cf47365aa77f11795ed20f00040bf6bdb22689ec5c10",
        "profile": "profiles/coh_ls_kernel_f32_c3_floating_5M.md"},
    "coh_ls_grad_f32": {"bytes": 40_095_744, "events": 5_000_000, "duration_ns": 423008, "warp_inst": 313_878_490, "issue_active": 0.6404,
        "sources": _COH_SRC, "sha256": "e6dd74780f809bce3110cf47365aa77f11795ed20f00040bf6bdb22689ec5c10",
        "profile": "profiles/coh_ls_kernel_f32_c3_floating_5M.md"},
    "td3_nll_grad_f32": {"bytes": 523_792_384, "events": 2_000_000, "duration_ns": 123872, "warp_inst": 57_684_324, "issue_active": 0.4858,
        "sources": _TD3_SRC, "sha256": "6ed9dd3bdcc23857eee61afd5ccf6fea65229ed5889dce989198cfbc3c23a7cc",
        "profile": "profiles/td3_nll_kernel_td3_2M.md"},
    "td3_nll_f64": {"bytes": 979_099_392, "events": 2_000_000, "duration_ns": 1546976, "fp64_pipe": 0.8508, "fp64_ops": {"dfma": 365_298_265, "dadd": 152_012_483, "dmul": 204_519_536},
        "sources": _TD3_SRC, "sha256": "6ed9dd3bdcc23857eee61afd5ccf6fea65229ed5889dce989198cfbc3c23a7cc",
        "profile": "profiles/td3_nll_kernel_td3_2M.md"},
    "td4_nll_grad_f32": {"bytes": 170_933_248, "events": 2_000_000, "duration_ns": 65632, "warp_inst": 40_895_064, "issue_active": 0.6042,
        "sources": _TD4_SRC, "sha256": "898395f56ed8fefb846f9ef3fb08867f16fcc8eb6ff15e61bc5de84b41a27fd9",
        "profile": "profiles/td4_nll_f32_kernel_c4_2M.md"},
    "td4_nll_f64": {"bytes": 339_106_816, "events": 2_000_000, "duration_ns": 1312992, "fp64_pipe": 0.8540, "fp64_ops": {"dfma": 325_287_209, "dadd": 112_011_018, "dmul": 164_442_328},
        "sources": _TD4_SRC, "sha256": "898395f56ed8fefb846f9ef3fb08867f16fcc8eb6ff15e61bc5de84b41a27fd9",
        "profile": "profiles/td4_nll_f64_kernel_c4_2M.md"},
}


def sources_sha256(paths):
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def ncu_record(kernel, n_events):
    """The kernel's ncu counters scaled to n_events, or None when absent or stale."""
    rec = NCU_RECORDS.get(kernel)
    if rec is None or sources_sha256(rec["sources"]) != rec["sha256"]:
        return None
    out = {"traffic": rec["bytes"] * n_events / rec["events"], "profile": rec["profile"]}
    if "fp64_pipe" in rec:
        out["fp64_pipe_active"] = rec["fp64_pipe"]
    if "warp_inst" in rec:
        out["warp_inst"] = rec["warp_inst"] * n_events / rec["events"]
        out["issue_active"] = rec["issue_active"]
    return out


def fp64_roofline(kernel, n_events, kernel_ms, fma64_per_s):
    """Counted FP64 work of one launch (ncu's thread-level DFMA, DADD and DMUL counts, scaled
    to n_events) over the launch's duration, against the measured FP64 FMA peak: FLOP/s with
    an FMA as two operations.  None without a current ncu record of the counts."""
    rec = NCU_RECORDS.get(kernel)
    if rec is None or "fp64_ops" not in rec or sources_sha256(rec["sources"]) != rec["sha256"]:
        return None
    ops = rec["fp64_ops"]
    scale = n_events / rec["events"]
    flops = (2.0 * ops["dfma"] + ops["dadd"] + ops["dmul"]) * scale
    insts = (ops["dfma"] + ops["dadd"] + ops["dmul"]) * scale
    achieved = flops / (kernel_ms * 1e-3)
    peak = 2.0 * fma64_per_s
    # a DADD or DMUL takes an FP64 issue slot as a DFMA does but counts one operation: the
    # instruction rate against the FMA rate says how full the pipe's arithmetic slots are
    return {"bound": "fp64", "flops_per_launch": flops, "achieved_flops": achieved, "peak_flops": peak,
            "flops_frac": achieved / peak, "fp64_inst_frac": insts / (kernel_ms * 1e-3) / fma64_per_s,
            "fp64_pipe_active": rec.get("fp64_pipe"),
            "counts_per_launch": {k: v * scale for k, v in ops.items()},
            "peak_source": "goo_peak_fma (fma.rn.f64 chains on every SM), measured in this run",
            "profile": rec["profile"]}


def idle_gpu_wait(cycles=200_000):
    """Keeps the current stream busy for about 0.1 ms without touching memory, so that a
    synchronous evaluation issued meanwhile starts right after its start event (tight event
    brackets) while L2 keeps its contents clean.  Used where the inputs exceed L2 and no flush
    is needed."""
    import torch
    torch.cuda._sleep(cycles)


def ncu_traffic(kernel, n_events):
    rec = ncu_record(kernel, n_events)
    return None if rec is None else rec["traffic"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--events", type=int, default=N_EVENTS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=1_000_000)
    ap.add_argument("--ref-sample", type=int, default=250_000)
    ap.add_argument("--no-extra", action="store_true", help="skip the Dalitz and serving measurements")
    ap.add_argument("--toys", type=int, default=4096)
    ap.add_argument("--rate", type=float, default=1000.0, help="Poisson arrival rate of the second serving run")
    ap.add_argument("--profile", action="store_true", help="short fixed launch sequence for ncu captures")
    ap.add_argument("--profile-workload", default="c2", choices=["c2", "c3", "c3f", "c4", "c5", "td3"])
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


# ---------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on the host cores, on a bounded sample
# ---------------------------------------------------------------------------------------
def oracle_rate(cols, n_sample, min_seconds=10.0, max_evals=20):
    import torch

    import synth
    from oracle import model as om
    spec = synth.c2_spec(bins=GRID)
    sample = {k: v[:n_sample] for k, v in cols.items()}
    m = om.TreeModel(spec)
    theta = synth.param_values(spec)
    m.nll_grad(sample, theta)  # warm
    t0 = time.perf_counter()
    evals = 0
    while evals < max_evals:
        m.nll_grad(sample, theta)
        evals += 1
        if time.perf_counter() - t0 >= min_seconds:
            break
    dt = (time.perf_counter() - t0) / evals
    return {"value": n_sample / dt, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"first {n_sample:,} of {len(cols['m']):,} events of the 3D workload, FP64 NLL + autograd "
                      f"gradient incl. the {GRID}^3 grid normalisation, {evals} evaluations, "
                      f"{dt * 1e3:.0f} ms each"}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo) and its logical core count."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                name = ln.split(":", 1)[1].strip()
                if ln.startswith("Model name"):
                    break
    except (OSError, subprocess.SubprocessError):
        pass
    if name is None:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    name = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            name = "unknown"
    return {"model": name, "logical_cores": os.cpu_count()}


def _time_calls(fn, min_seconds, max_calls):
    fn()  # warm
    t0 = time.perf_counter()
    calls = 0
    while calls < max_calls:
        fn()
        calls += 1
        if time.perf_counter() - t0 >= min_seconds:
            break
    return (time.perf_counter() - t0) / calls, calls


def oracle_baselines(min_seconds=1.5, with_fits=True):
    """The FP64 oracle, as it stands, on bounded samples of every workload, on this process's
    threads: events/s of one NLL + gradient evaluation per configuration and, with_fits,
    oracle fits of toys of the served study drawn from three strata of its event-count
    distribution."""
    import numpy as np
    import torch

    import synth
    from oracle import dalitz as od
    from oracle import fit as ofit
    from oracle import model as om
    from oracle import td3 as ot3
    from oracle import td4 as ot
    from oracle import toys as otoys
    out = {}

    def entry(n_events, fn, sample, min_s=min_seconds, max_calls=20):
        dt, calls = _time_calls(fn, min_s, max_calls)
        return {"value": n_events / dt, "unit": UNIT, "s_per_eval": dt, "evals": calls, "sample": sample}

    spec = synth.c1_spec()
    cols = synth.gen_c1()
    m1 = om.TreeModel(spec)
    th1 = synth.param_values(spec)
    out["c1_1d"] = entry(len(cols["x"]), lambda: m1.nll_grad(cols, th1),
                         "all 100,000 events; FP64 NLL + autograd gradient, analytic normalisation")
    spec = synth.c2_spec(bins=GRID)
    n2 = 250_000
    cols = synth.gen_c2(n=n2, seed=1710002)
    m2 = om.TreeModel(spec)
    th2 = synth.param_values(spec)
    out["c2_3d"] = entry(n2, lambda: m2.nll_grad(cols, th2),
                         f"{n2:,} events of the 3D recipe; FP64 NLL + autograd gradient incl. the {GRID}^3 grid")
    spec = synth.c3_spec()
    k = synth.DALITZ_MASSES
    n3, nmc3 = 200_000, 40_000
    d3 = synth.dalitz_candidates(n3, 1710003, k["M"], k["m1"], k["m2"], k["m3"])
    mc3 = synth.dalitz_candidates(nmc3, 1710013, k["M"], k["m1"], k["m2"], k["m3"])
    m3 = od.DalitzModel(spec)
    th3 = synth.param_values(spec)
    out["c3_dalitz"] = entry(n3, lambda: m3.nll_grad(d3, mc3, th3),
                             f"{n3:,} phase-space events + {nmc3:,} MC points (the workload's 5:1 ratio); FP64 "
                             "amplitudes, NLL and autograd gradient recomputed per evaluation")
    spec, d4, mc4 = c4_inputs(100_000, 150_000)
    m4 = ot.TD4Model(spec)
    th4 = np.array(synth.param_values(spec))
    a4, mca4 = m4.amplitudes(d4), m4.amplitudes(mc4)
    out["c4_td4"] = entry(100_000, lambda: m4.nll_grad(d4, mca4, th4, a=a4),
                          "100,000 events, amplitudes of the events and of 150,000 MC points computed once (as the "
                          "GPU path caches them); FP64 rate, NLL and analytic gradient")
    spec, dt3, mct3 = td3_inputs(100_000, 50_000)
    mt3 = ot3.TD3Model(spec)
    tht3 = np.array(synth.param_values(spec))
    at3, gt3 = mt3.amplitudes(dt3, tht3), mt3.grams(mct3, tht3)
    out["td3_dalitz"] = entry(100_000, lambda: mt3.nll_grad(dt3, mct3, tht3, amps=at3, grams=gt3),
                              "100,000 events, amplitude caches and Gram matrices (50,000 MC points) computed once; "
                              "FP64 rate, NLL and analytic gradient")
    if not with_fits:
        return out
    # served study: oracle fits of toys from three strata of the log-uniform sizes
    spec = synth.c3_spec()
    theta = np.array(synth.param_values(spec))
    free = np.array([not p[2] for p in spec["params"]])
    steps = np.array([p[3] if p[3] > 0 else 1.0 for p in spec["params"]])
    mc = synth.dalitz_candidates(50_000, 1710013, k["M"], k["m1"], k["m2"], k["m3"])
    env = otoys.envelope(spec, theta)
    sizes = synth.toy_sizes(4096)
    fits = []
    for target in (2_400, 13_000, 75_000):   # geometric middles of [1e3, 5.6e3), [5.6e3, 3.2e4), [3.2e4, 1.8e5)
        i = int(np.argmin(np.abs(sizes - target)))
        a, b, _ = otoys.generate_toy(spec, theta, env, 1710100 + i, int(sizes[i]))
        toy = {"s12": a.astype(np.float64), "s13": b.astype(np.float64)}
        t0 = time.perf_counter()
        ofit.fit(lambda t: m3.nll_grad(toy, mc, t), theta, free, steps)
        fits.append({"toy": i, "events": int(sizes[i]), "fit_s": time.perf_counter() - t0})
    # mean fit time over the study's sizes from t = a + b N through the three measured fits
    N = np.array([f["events"] for f in fits], float)
    T = np.array([f["fit_s"] for f in fits])
    b, a = np.polyfit(N, T, 1)
    mean_t = float(np.mean(a + b * sizes))
    out["c5_serving"] = {"value": 1.0 / mean_t, "unit": "fits/s", "fits": fits,
                         "sample": "one toy from each of three strata of the 4096 event counts (geometric middles "
                                   "2.4k, 13k, 75k), generated by the oracle's counter-based generator, fitted by the "
                                   "oracle (scipy BFGS + Newton polish, autograd gradient) with a 50,000-point MC; "
                                   "fits/s = 1 / mean over the 4096 sizes of a + b N fitted to the three fit times"}
    return out


def oracle_baselines_subprocess(threads, with_fits, min_seconds, timeout=900):
    """oracle_baselines() in a fresh interpreter with `threads` threads for torch, OpenMP and
    BLAS (0: the host's default), so that the single-thread figure uses one core."""
    env = dict(os.environ)
    if threads:
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[v] = str(threads)
    code = ("import json, sys, torch; sys.path.insert(0, %r); import bench; "
            "%s print(json.dumps({'threads': torch.get_num_threads(), "
            "'configs': bench.oracle_baselines(min_seconds=%r, with_fits=%r)}))"
            % (ROOT, "torch.set_num_threads(%d);" % threads if threads else "", min_seconds, with_fits))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=timeout)
    if r.returncode != 0:
        return {"error": (r.stderr or r.stdout)[-500:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    import torch

    import synth
    from oracle import model as om
    cols = synth.gen_c2(n=args.events, seed=1710002)
    n_sample = min(args.ref_sample, args.events)
    spec = synth.c2_spec(bins=GRID)
    sample = {k: v[:n_sample] for k, v in cols.items()}
    m = om.TreeModel(spec)
    theta = synth.param_values(spec)
    for _ in range(args.warmup):
        m.nll_grad(sample, theta)
    t_all = time.perf_counter()
    for _ in range(args.steps):
        m.nll_grad(sample, theta)
    elapsed = time.perf_counter() - t_all
    value = n_sample * args.steps / elapsed
    base = {"value": value, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"{args.steps} steps, each one FP64 NLL + autograd gradient (incl. the {GRID}^3 grid "
                      f"normalisation) of the first {n_sample:,} events"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"c2_3d: {args.events:,} events (m, dE, t), 12 params, {GRID}^3 grid",
                       "events_per_step": n_sample},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------------------
# our path
# ---------------------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    import synth
    from paper_1710_08826_gb300 import build
    build()
    from paper_1710_08826_gb300 import dist as gdist
    from paper_1710_08826_gb300 import goo

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    spec = synth.c2_spec(bins=GRID)
    n = args.events
    cols = synth.gen_c2(n=n, seed=1710002 + rank)      # each rank holds its own shard (weak scaling)
    stream = torch.cuda.Stream()                       # the library and torch share this stream
    torch.cuda.set_stream(stream)
    ctx = goo.Context(local_rank, stream=stream.cuda_stream)
    ds = goo.Dataset.from_spec(ctx, spec, cols, dtype="f64")
    model = goo.Model(ctx, spec)
    theta = np.array(synth.param_values(spec))
    P = len(theta)

    def step(precision, grad=True):
        # one shard record per rank; N > 1: all-gather and the ordered, compensated combine
        out = model.nll_partial(ds, 0, ds.n, theta, precision, want_grad=grad)
        if pg is not None:
            nll, g, _ = gdist.combine(gdist.allgather_records(out, device="cuda"), P)
            return nll, g
        return out[0] + out[1], out[3:]

    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def timed(precision, grad, steps, warmup):
        # the step time is taken without the library's per-kernel events (they would sit
        # between the normalisation and event kernels and serialise them); a second pass of
        # the same steps with per-kernel events gives each kernel's launch duration
        for _ in range(warmup):
            step(precision, grad)
        # then back-to-back steps for at least 0.25 s, so that the GPU leaves its idle clocks
        # (the kernel compilation on the first call leaves it idle for seconds)
        t_end = time.perf_counter() + 0.25
        while time.perf_counter() < t_end:
            step(precision, grad)
        barrier()
        launches0 = ctx.launches

        def run(n):
            # the interpreter's garbage collector stays off while steps are timed (its pauses
            # are host jitter, not work of the step)
            import gc
            gc.disable()
            try:
                return run_steps(n)
            finally:
                gc.enable()

        def run_steps(n):
            ms = []
            for _ in range(n):
                flush.zero_()                       # L2 flush between timed steps (not timed)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step(precision, grad)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            return ms

        ms = run(steps)
        barrier()
        launches = ctx.launches - launches0
        ctx.kernel_times(reset=True)
        ctx.timing(True)
        run(max(3, min(steps, 10)))
        barrier()
        ctx.timing(False)
        kt = ctx.kernel_times(reset=True)
        total = sum(ms)
        if pg is not None:
            t = torch.tensor([total], dtype=torch.float64, device="cuda")
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            total = float(t.item())
        return total, ms, kt, launches

    with ClockSampler(local_rank) as clocks:
        total_mix, ms_mix, kt_mix, launches = timed("f32", True, args.steps, args.warmup)
        steps64 = max(3, args.steps // 5)
        total_64, ms_64, kt_64, _ = timed("f64", False, steps64, min(args.warmup, 3))
    clk = clocks.summary()
    # the arithmetic rooflines' denominators, measured on this GPU now (goo_peak_fma)
    fma_peaks = {k: max(ctx.peak_fma(k)[0] for _ in range(2)) for k in ("f64", "f32", "f32x2")}

    # parity spot check of this very configuration against the FP64 path
    nll32 = step("f32", True)[0]
    nll64 = step("f64", False)[0]

    # ---- end-to-end through the public API: pinned host columns -> device -> NLL+grad -> host
    host_cols = {k: torch.from_numpy(np.asarray(v, dtype=np.float32)).pin_memory()
                 for k, v in synth.round_to_f32(cols, spec).items()}
    lo = [o[1] for o in spec["observables"]]
    hi = [o[2] for o in spec["observables"]]
    names = [o[0] for o in spec["observables"]]

    # Three forms of the user's step, each timed over the same number of steps: a dataset
    # created and freed every step; one dataset refilled every step through the copy engine
    # (goo_dataset_update, GOO_COPY); and refilled by the ingest kernel reading the pinned
    # host columns itself (GOO_COPY_MAPPED).  Every form moves the step's columns host ->
    # device and reads the NLL and gradient back.
    cols_np = [host_cols[k].numpy() for k in names]
    cols_pin = [host_cols[k] for k in names]
    ds_stream = goo.Dataset(ctx, cols_np, lo, hi, dtype="f32")

    def e2e_fresh():
        d = goo.Dataset(ctx, cols_np, lo, hi, dtype="f32")
        out = model.nll_grad(d, theta, "f32")
        d.close()
        return out

    def e2e_update():
        ds_stream.update(cols_np)
        return model.nll_grad(ds_stream, theta, "f32")

    def e2e_mapped():
        ds_stream.update(cols_pin, mapped=True)
        return model.nll_grad(ds_stream, theta, "f32")

    def e2e_streamed(chunks):
        return lambda: model.nll_grad_streamed(ds_stream, cols_pin, theta, n_chunks=chunks)

    # the columns stay in pinned host memory; every evaluation reads them over the host link
    ds_host = goo.Dataset(ctx, cols_pin, lo, hi, dtype="f32", borrow_host=True)

    def e2e_borrow_host():
        return model.nll_grad(ds_host, theta, "f32")

    e2e_steps = max(3, args.steps // 5)

    def e2e_time(fn):
        for _ in range(2):
            fn()
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            fn()
        barrier()
        sec = time.perf_counter() - t0
        if pg is not None:
            t = torch.tensor([sec], dtype=torch.float64, device="cuda")
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            sec = float(t.item())
        return sec

    e2e_forms = {
        "borrow_host": (e2e_time(e2e_borrow_host), "GOO_BORROW_HOST dataset: the event kernel reads the pinned float32 "
                                                   "host columns over the host link itself (no copy, no ingest pass; "
                                                   "range-checked in the kernel) + goo_nll_grad"),
        "streamed_8": (e2e_time(e2e_streamed(8)), "goo_nll_grad_streamed, 8 chunks: the copy engine moves chunk c + 1 "
                                                  "from the pinned float32 host columns while chunk c is range-checked "
                                                  "and evaluated"),
        "streamed_16": (e2e_time(e2e_streamed(16)), "goo_nll_grad_streamed, 16 chunks"),
        "update_mapped": (e2e_time(e2e_mapped), "goo_dataset_update (GOO_COPY_MAPPED: the ingest kernel reads the "
                                                "pinned float32 host columns) + goo_nll_grad"),
        "update_copy": (e2e_time(e2e_update), "goo_dataset_update (GOO_COPY: copy engine from pinned float32 host "
                                              "columns) + goo_nll_grad"),
        "fresh_upload": (e2e_time(e2e_fresh), "goo_dataset_upload from pinned float32 host columns + goo_nll_grad + "
                                              "goo_dataset_free"),
    }
    ds_stream.close()
    ds_host.close()
    # the host link's copy bandwidth for the step's bytes (pinned host -> device, copy engine):
    # the floor of any end-to-end form
    link_src = torch.empty(n * BYTES_PER_EVENT_F32, dtype=torch.uint8).pin_memory()
    link_dst = torch.empty_like(link_src, device="cuda")
    for _ in range(2):
        link_dst.copy_(link_src, non_blocking=True)
    ls0 = torch.cuda.Event(enable_timing=True)
    ls1 = torch.cuda.Event(enable_timing=True)
    ls0.record(stream)
    for _ in range(5):
        link_dst.copy_(link_src, non_blocking=True)
    ls1.record(stream)
    ls1.synchronize()
    link_ms = ls0.elapsed_time(ls1) / 5
    host_link = {"h2d_gbs": link_src.numel() / (link_ms * 1e-3) / 1e9, "bytes": int(link_src.numel()),
                 "floor_ms_per_step": link_ms,
                 "what": "pinned host -> device copy of the step's column bytes (copy engine), 5 copies timed"}
    del link_src, link_dst
    e2e_best = min(e2e_forms, key=lambda k: e2e_forms[k][0])
    e2e_s = e2e_forms[e2e_best][0]

    # ---- roofline of the dominant kernel of the FP32+grad step
    name, (cnt, kms) = max(kt_mix.items(), key=lambda kv: kv[1][1])
    per_launch_s = kms / cnt * 1e-3
    peak, peak_kind = measured_peaks()
    if name.startswith("sop_nll"):
        alg_bytes = n * BYTES_PER_EVENT_F32
    else:
        alg_bytes = 0
    achieved = alg_bytes / per_launch_s / 1e9
    # the kernel is bound by instruction issue (see "issue" below); achieved and frac are its
    # algorithmic bytes against the measured HBM copy bandwidth
    roofline = {"bound": "issue", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": ncu_traffic(name, n), "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                "launch_ms": per_launch_s * 1e3,
                "algorithmic_bytes_per_launch": alg_bytes,
                "kernel_share": {k: round(v[1] / max(sum(x[1] for x in kt_mix.values()), 1e-12), 4)
                                 for k, v in kt_mix.items()}}
    rec = ncu_record(name, n)
    if rec is not None and "warp_inst" in rec:
        # the binding resource: instruction issue (one warp instruction per scheduler per
        # cycle at the maximum SM clock); the warp-instruction count is ncu's for this kernel
        roofline["issue"] = {"warp_inst_per_launch": rec["warp_inst"],
                             "achieved_frac_of_issue_peak": rec["warp_inst"] / per_launch_s / ISSUE_PEAK,
                             "ncu_issue_active": rec["issue_active"], "peak_warp_inst_per_s": ISSUE_PEAK}

    value = n * world * args.steps / (total_mix * 1e-3)
    e2e_value = n * world * e2e_steps / e2e_s
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_mix / args.steps,
        "ms_per_step_p50": float(np.median(ms_mix)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"c2_3d: {n:,} events/GPU over (m, dE, t), signal Gauss*Gauss*Exp + background "
                               f"Argus*Poly2*Exp, 12 free params, {GRID}^3 grid normalisation, NLL + adjoint gradient",
                   "events_per_gpu": n, "params": P, "grid": [GRID] * 3,
                   "precision": "FP32 per-event, compensated FP32 / double-float accumulation, FP64 final combine",
                   "l2": "flushed between timed steps (256 MB write, not timed)",
                   "parallelism": f"dp{world} (events sharded, partials all-reduced)" if world > 1 else "single GPU"},
        "nll_evals_per_s": args.steps / (total_mix * 1e-3),
        "fp64_plain": {"events_per_s": n * world * steps64 / (total_64 * 1e-3),
                       "evals_per_s": steps64 / (total_64 * 1e-3), "ms_per_eval": total_64 / steps64,
                       "what": "goo_nll in float64 (FP64 per-event arithmetic and grid), no gradient",
                       "kernels_ms": {k: v[1] / v[0] for k, v in kt_64.items()},
                       "roofline": fp64_roofline("sop_nll_f64", n, kt_64["sop_nll_f64"][1] / kt_64["sop_nll_f64"][0],
                                                 fma_peaks["f64"]) if "sop_nll_f64" in kt_64 else None,
                       "ncu": ncu_record("sop_nll_f64", n)},
        "fma_peaks": {"fma_per_s": fma_peaks, "flops_per_s": {k: 2 * v for k, v in fma_peaks.items()},
                      "what": "goo_peak_fma: num_sms x 4 blocks of 256 threads, 8 independent FMA chains each"},
        "parity_this_run": {"nll_f32": nll32, "nll_f64": nll64, "rel": abs(nll32 - nll64) / abs(nll64)},
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n * BYTES_PER_EVENT_F32 + 8 * P,
                "d2h_bytes_per_step": 8 * (2 + P), "ms_per_step": e2e_s / e2e_steps * 1e3,
                "what": e2e_forms[e2e_best][1],
                "forms_ms_per_step": {k: v[0] / e2e_steps * 1e3 for k, v in e2e_forms.items()},
                "host_link": host_link},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_extra:
        # the fit of this configuration: every parameter free but the Argus endpoint m0 (the
        # likelihood is not differentiable where m0 crosses an event), from shifted values
        free = np.ones(P, bool)
        free[[p[0] for p in spec["params"]].index("m0")] = False
        start = theta.copy()
        start[[0, 2]] += np.array([2e-4, 2e-3])
        start[[1, 3, 4, 6, 7, 8, 9, 10, 11]] *= 1.03
        scale = np.array([p[3] for p in spec["params"]])
        r32, r32u, r64 = [], [], []
        line["c2_fit"] = {"f32": fit_timed(model, ds, start, free, scale, "f32", keep=r32),
                          "f32_without_fp64_refinement": fit_timed(model, ds, start, free, scale, "f32", keep=r32u,
                                                                   refine=False),
                          "f64": fit_timed(model, ds, start, free, scale, "f64", keep=r64)}
        # the FP32 fits' distance from the FP64 fit of the same 10M events, in FP64 errors
        for key, r in (("f32", r32), ("f32_without_fp64_refinement", r32u)):
            line["c2_fit"][key]["max_abs_diff_sigma_vs_f64"] = float(np.max(np.abs(r[0] - r64[0])[free] / r64[1][free]))
        line["c1_1d"] = c1_measure(goo, ctx, stream, max(20, args.steps))
        line["c3_dalitz"] = c3_measure(goo, ctx, stream, max(5, args.steps // 2), fma64=fma_peaks["f64"])
        line["c4_td4"] = c4_measure(goo, ctx, stream, max(5, args.steps // 2), fma64=fma_peaks["f64"])
        line["td3_dalitz"] = td3_measure(goo, ctx, stream, max(5, args.steps // 2), fma64=fma_peaks["f64"])
        line["c5_serving"] = c5_study(goo, ctx, n_toys=args.toys)
        line["c5_serving_poisson"] = c5_study(goo, ctx, n_toys=max(64, args.toys // 4), rate=args.rate, plain_sample=0)
        # a sweep of arrival rates below and above the served throughput
        line["c5_rate_sweep"] = [
            {k: v for k, v in c5_study(goo, ctx, n_toys=max(64, args.toys // 8), rate=r, plain_sample=0).items()
             if k in ("toys", "arrival", "fits_per_s", "latency_p50_s", "latency_p99_s", "converged")}
            for r in (250.0, 4000.0, 16000.0)]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_rate(cols, min(args.cpu_sample, n))
        # the oracle beside every configuration: all host cores (with oracle fits of served
        # toys) and one thread, each in its own interpreter
        allc = oracle_baselines_subprocess(0, with_fits=True, min_seconds=1.5)
        one = oracle_baselines_subprocess(1, with_fits=False, min_seconds=1.0)
        host = cpu_model()
        line["oracle_baselines"] = {"host": host, "all_cores": allc, "single_thread": one}
        for key, cfg in (allc.get("configs") or {}).items():
            if key in line and isinstance(line[key], dict):
                base = {"all_cores": dict(cfg, cores=allc.get("threads"), kind="oracle")}
                if key in (one.get("configs") or {}):
                    base["single_thread"] = dict(one["configs"][key], cores=1, kind="oracle")
                base["host"] = host
                line[key]["cpu_baseline"] = base
    if rank == 0:
        print(json.dumps(line))
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------------------
# three-body amplitude workload (5M events, 1M-point MC normalisation)
# ---------------------------------------------------------------------------------------
def fit_timed(model, ds, start, free, steps, precision="f32", gradient="adjoint", keep=None, refine=True):
    """One goo_fit from `start` (errors from the Hessian): wall time and the minimiser's
    counts.  The model has been evaluated before, so no kernel is compiled inside the timed
    fit."""
    t0 = time.perf_counter()
    th, err, info = model.fit(ds, start, free, steps, precision=precision, gradient=gradient, refine=refine)
    wall = time.perf_counter() - t0
    if keep is not None:
        keep.extend([th, err])
    return {"wall_s": wall, "precision": precision, "gradient": gradient,
            "fp64_refinement": bool(refine and precision == "f32" and gradient == "adjoint"), "status": int(info["status"]),
            "edm": info["edm"],
            "iterations": int(info["iterations"]), "nll_evals": int(info["nll_evals"]),
            "grad_evals": int(info["grad_evals"]), "free_params": int(sum(bool(f) for f in free))}


def c1_measure(goo, ctx, stream, steps):
    """C1 (100,000 events in 1D): launch-bound evaluations and the fit wall time."""
    import numpy as np
    import torch

    import synth
    spec = synth.c1_spec()
    cols = synth.gen_c1()
    ds = goo.Dataset.from_spec(ctx, spec, cols)
    model = goo.Model(ctx, spec)
    theta = np.array(synth.param_values(spec))
    n = len(cols["x"])
    out = {"workload": f"c1_1d: {n:,} events on [0, 10], 0.3 Gauss + 0.7 Exp, 4 free parameters, analytic "
                       "normalisation (launch-bound: the data is L2-resident)"}
    for prec, grad in (("f32", True), ("f64", False)):
        for _ in range(3):
            model.nll_grad(ds, theta, prec) if grad else model.nll(ds, theta, prec)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            model.nll_grad(ds, theta, prec) if grad else model.nll(ds, theta, prec)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        out["f32_grad" if grad else "f64_plain"] = {"evals_per_s": steps / (ms * 1e-3), "us_per_eval": ms / steps * 1e3,
                                                    "events_per_s": n * steps / (ms * 1e-3)}
    free = np.ones(len(theta), bool)
    scale = np.array([p[3] for p in spec["params"]])
    out["fit_f32"] = fit_timed(model, ds, theta * 1.05, free, scale, "f32")
    out["fit_f64"] = fit_timed(model, ds, theta * 1.05, free, scale, "f64")
    # the configuration's own form: FP64 with the minimiser's numerical (central-difference)
    # gradient
    out["fit_f64_numerical_gradient"] = fit_timed(model, ds, theta * 1.05, free, scale, "f64", "fd")
    return out


def c3_measure(goo, ctx, stream, steps, n_events=5_000_000, n_mc=1_000_000, fma64=None):
    import numpy as np
    import torch

    import synth
    spec = synth.c3_spec(n_mc=n_mc)
    kin = synth.DALITZ_MASSES
    mc = synth.round_to_f32(synth.dalitz_candidates(n_mc, 1710013, kin["M"], kin["m1"], kin["m2"], kin["m3"]), spec)
    mcds = goo.Dataset.from_spec(ctx, spec, mc)
    model = goo.Model(ctx, spec, mc=mcds)
    theta = np.array(synth.param_values(spec))
    t0 = time.perf_counter()
    a, b = goo.toy_generate(model, theta, None, 1710003, n_events)   # accept-reject on the device
    gen_s = time.perf_counter() - t0
    ds = goo.Dataset.from_spec(ctx, spec, {"s12": a.astype(np.float64), "s13": b.astype(np.float64)})
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    out = {"workload": f"c3_dalitz: {n_events:,} events generated on the device from the 8-resonance model, "
                       f"{n_mc:,}-point phase-space MC, 16 free coefficients",
           "generation_s": gen_s,
           "l2": "inputs larger than L2 (320 MB amplitude cache per evaluation), no flush"}
    for prec, grad, k in (("f32", True, steps), ("f64", False, max(3, steps // 5))):
        for _ in range(3):
            model.nll_grad(ds, theta, prec) if grad else model.nll(ds, theta, prec)
        torch.cuda.synchronize()
        ctx.kernel_times(reset=True)
        ctx.timing(True)
        ms = 0.0
        for _ in range(k):
            idle_gpu_wait()  # inputs larger than L2: no flush; the GPU busy while the call is issued
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            model.nll_grad(ds, theta, prec) if grad else model.nll(ds, theta, prec)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        ctx.timing(False)
        kt = ctx.kernel_times(reset=True)
        name, (cnt, kms) = max(kt.items(), key=lambda kv: kv[1][1])
        bytes_per_event = 64 if prec == "f32" else 128
        per = kms / cnt
        out["f32_grad" if grad else "f64_plain"] = {
            "evals_per_s": k / (ms * 1e-3), "events_per_s": n_events * k / (ms * 1e-3), "ms_per_eval": ms / k,
            "kernel": name, "kernel_ms": per,
            "hbm_frac": n_events * bytes_per_event / (per * 1e-3) / 1e9 / measured_peaks()[0],
            "bound": "hbm" if grad else "fp64", "ncu": ncu_record(name, n_events),
            "roofline": None if grad or fma64 is None else fp64_roofline(name, n_events, per, fma64),
            "what": ("goo_nll_grad, FP32 amplitude cache (64 B/event), adjoint gradient" if grad
                     else "goo_nll, FP64 amplitude cache (128 B/event)")}
    free = np.array([not p[2] for p in spec["params"]])
    scale = np.array([p[3] if p[3] > 0 else 1.0 for p in spec["params"]])
    start = theta.copy()
    start[free] *= 1.05
    out["fit_f32"] = fit_timed(model, ds, start, free, scale)
    out["floating_lineshapes"] = c3_floating_measure(goo, ctx, stream, model, ds, theta, flush, steps, n_events, n_mc)
    return out


def c3_floating_measure(goo, ctx, stream, model, ds, theta, flush, steps, n_events, n_mc):
    """The same events with the resonance masses and widths free: every evaluation runs an MC
    pass and an event pass that evaluate all amplitudes and their lineshape derivatives."""
    import numpy as np
    import torch

    model.set_lineshapes("floating")
    out = {"workload": f"c3_dalitz floating lineshapes: {n_events:,} events + {n_mc:,} MC points per evaluation, "
                       "8 resonances recomputed with d/dm0 and d/dGamma0, 32 parameters (16 coefficients, "
                       "8 masses, 8 widths)"}
    for prec, grad, k in (("f32", True, steps), ("f64", False, max(3, steps // 5))):
        for _ in range(3):
            model.nll_grad(ds, theta, prec) if grad else model.nll(ds, theta, prec)
        torch.cuda.synchronize()
        ctx.kernel_times(reset=True)
        ctx.timing(True)
        ms = 0.0
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            model.nll_grad(ds, theta, prec) if grad else model.nll(ds, theta, prec)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        ctx.timing(False)
        kt = ctx.kernel_times(reset=True)
        kernels = {name: kms / cnt for name, (cnt, kms) in kt.items()}
        name = max(kernels, key=kernels.get)
        rec = ncu_record(name, n_events)
        entry = {"evals_per_s": k / (ms * 1e-3), "events_per_s": n_events * k / (ms * 1e-3), "ms_per_eval": ms / k,
                 "kernels_ms": kernels, "kernel": name, "bound": "alu (FP32 issue)" if grad else "fp64",
                 "ncu": rec,
                 "what": ("goo_nll_grad, FP32 amplitudes and lineshape derivatives per event and MC point, "
                          "adjoint gradient over all 32 parameters" if grad
                          else "goo_nll, FP64 amplitudes per event and MC point")}
        if rec and rec.get("warp_inst") and grad:
            # issue roofline: warp instructions per launch / duration / (SMs x 4 schedulers x clock)
            entry["issue_frac"] = rec["warp_inst"] / (kernels[name] * 1e-3) / ISSUE_PEAK
        out["f32_grad" if grad else "f64_plain"] = entry
    n32, g32 = model.nll_grad(ds, theta, "f32")
    n64 = model.nll(ds, theta, "f64")
    out["parity_this_run"] = {"nll_f32": n32, "nll_f64": n64, "rel": abs(n32 - n64) / abs(n64)}
    model.set_lineshapes("cached")
    return out


# ---------------------------------------------------------------------------------------
# time-dependent four-body workload (2M events, 3M-point MC normalisation)
# ---------------------------------------------------------------------------------------
def c4_inputs(n_events, n_mc, seed=1710004):
    """Four-body phase-space events with decay times Exp(tau) smeared by N(0, sigma_t).

    The events follow phase space and the lifetime, not the amplitude model: the per-event
    work and the bytes read do not depend on where the events fall.
    """
    import numpy as np

    import synth
    spec = synth.c4_spec(n_mc=n_mc)
    kin = dict(synth.TD4_MASSES)
    tau, sig = synth.TD4_TIME["tau"], synth.TD4_TIME["sigma_t"]
    tlo, thi = spec["observables"][5][1:]
    data = synth.gen_c4_candidates(n_events, seed, kin, 1.0 / tau)
    data["t"] = np.clip(synth.smear_times(data.pop("t_true"), sig, seed + 1), tlo, thi)
    mc = synth.four_body_phase_space(n_mc, 1710014, **kin)
    mc["t"] = np.zeros(n_mc)
    return spec, synth.round_to_f32(data, spec), synth.round_to_f32(mc, spec)


def c4_measure(goo, ctx, stream, steps, n_events=2_000_000, n_mc=3_000_000, fma64=None):
    import numpy as np
    import torch

    import synth
    spec, data, mc = c4_inputs(n_events, n_mc)
    mcds = goo.Dataset.from_spec(ctx, spec, mc)
    model = goo.Model(ctx, spec, mc=mcds)
    ds = goo.Dataset.from_spec(ctx, spec, data)
    theta = np.array(synth.param_values(spec))
    out = {"workload": f"c4_td4: {n_events:,} four-body events (phase space, t = Exp(0.41 ps) + N(0, 0.05 ps)), "
                       f"{n_mc:,}-point phase-space MC, 10 amplitudes, 24 free parameters (20 coefficients, x, y, "
                       "tau, sigma_t)",
           "l2": "inputs larger than L2 (168 MB of amplitude planes and times per evaluation), no flush"}
    nll = {}
    for prec, grad, k in (("f32", True, steps), ("f64", False, max(3, steps // 5))):
        for _ in range(3):
            model.nll_grad(ds, theta, prec) if grad else model.nll(ds, theta, prec)
        torch.cuda.synchronize()
        ms = 0.0
        for _ in range(k):
            idle_gpu_wait()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            v = model.nll_grad(ds, theta, prec)[0] if grad else model.nll(ds, theta, prec)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        nll[prec] = v
        ctx.kernel_times(reset=True)
        ctx.timing(True)
        for _ in range(3):
            idle_gpu_wait()
            model.nll_grad(ds, theta, prec) if grad else model.nll(ds, theta, prec)
        ctx.timing(False)
        kt = ctx.kernel_times(reset=True)
        name, (cnt, kms) = max(kt.items(), key=lambda kv: kv[1][1])
        bytes_per_event = 84 if prec == "f32" else 168   # amplitude planes + the time column
        per = kms / cnt
        out["f32_grad" if grad else "f64_plain"] = {
            "evals_per_s": k / (ms * 1e-3), "events_per_s": n_events * k / (ms * 1e-3), "ms_per_eval": ms / k,
            "kernel": name, "kernel_ms": per,
            "hbm_frac": n_events * bytes_per_event / (per * 1e-3) / 1e9 / measured_peaks()[0],
            "bound": "hbm" if grad else "fp64", "ncu": ncu_record(name, n_events),
            "roofline": None if grad or fma64 is None else fp64_roofline(name, n_events, per, fma64),
            "what": ("goo_nll_grad, FP32 amplitude cache (80 B/event) + time, adjoint gradient" if grad
                     else "goo_nll, FP64 amplitude cache (160 B/event) + time")}
    out["parity_this_run"] = {"nll_f32": nll["f32"], "nll_f64": nll["f64"],
                              "rel": abs(nll["f32"] - nll["f64"]) / abs(nll["f64"])}
    # no fit is timed here: these events are phase-space points, not drawn from the model
    # (the fit parity tests use events generated from it)
    return out


def td3_inputs(n_events, n_mc, seed=1710016):
    """Uniform three-body phase-space events (pi0 pi+ pi- masses) with decay times Exp(tau)
    smeared by N(0, sigma_t); the per-event work does not depend on where the events fall."""
    import numpy as np

    import synth
    spec = synth.td3_spec(n_mc=n_mc)
    k = synth.TD3_MASSES
    tau, sig = synth.TD4_TIME["tau"], synth.TD4_TIME["sigma_t"]
    data = synth.dalitz_candidates(n_events, seed, k["M"], k["m1"], k["m2"], k["m3"])
    rng = np.random.default_rng(seed + 1)
    data["t"] = np.clip(rng.exponential(tau, n_events) + rng.normal(0.0, sig, n_events), *spec["observables"][2][1:])
    mc = synth.dalitz_candidates(n_mc, 1710015, k["M"], k["m1"], k["m2"], k["m3"])
    mc["t"] = np.zeros(n_mc)
    return spec, synth.round_to_f32(data, spec), synth.round_to_f32(mc, spec)


def td3_measure(goo, ctx, stream, steps, n_events=2_000_000, n_mc=1_000_000, fma64=None):
    import numpy as np
    import torch

    import synth
    spec, data, mc = td3_inputs(n_events, n_mc)
    mcds = goo.Dataset.from_spec(ctx, spec, mc)
    model = goo.Model(ctx, spec, mc=mcds)
    ds = goo.Dataset.from_spec(ctx, spec, data)
    theta = np.array(synth.param_values(spec))
    out = {"workload": f"td3_dalitz: {n_events:,} pi0 pi+ pi- phase-space events (t = Exp(0.41 ps) + N(0, 0.05 ps)), "
                       f"{n_mc:,}-point MC, 15 resonances + NR at the event and the exchanged point, 36 parameters "
                       "(30 free coefficients, x, y, tau, sigma_t)",
           "l2": "inputs larger than L2 (520 MB of amplitude planes and times per evaluation), no flush"}
    nll = {}
    for prec, grad, k in (("f32", True, steps), ("f64", False, max(3, steps // 5))):
        for _ in range(3):
            model.nll_grad(ds, theta, prec) if grad else model.nll(ds, theta, prec)
        torch.cuda.synchronize()
        ms = 0.0
        for _ in range(k):
            idle_gpu_wait()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            v = model.nll_grad(ds, theta, prec)[0] if grad else model.nll(ds, theta, prec)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        nll[prec] = v
        ctx.kernel_times(reset=True)
        ctx.timing(True)
        for _ in range(3):
            idle_gpu_wait()
            model.nll_grad(ds, theta, prec) if grad else model.nll(ds, theta, prec)
        ctx.timing(False)
        kt = ctx.kernel_times(reset=True)
        name, (cnt, kms) = max(kt.items(), key=lambda kv: kv[1][1])
        # two caches of 15 amplitudes (8 float4 / 15 double2 planes each) and the time column
        bytes_per_event = 2 * 8 * 16 + 4 if prec == "f32" else 2 * 15 * 16 + 8
        per = kms / cnt
        out["f32_grad" if grad else "f64_plain"] = {
            "evals_per_s": k / (ms * 1e-3), "events_per_s": n_events * k / (ms * 1e-3), "ms_per_eval": ms / k,
            "kernel": name, "kernel_ms": per,
            "hbm_frac": n_events * bytes_per_event / (per * 1e-3) / 1e9 / measured_peaks()[0],
            "bound": "issue" if grad else "fp64", "ncu": ncu_record(name, n_events),
            "roofline": None if grad or fma64 is None else fp64_roofline(name, n_events, per, fma64),
            "what": ("goo_nll_grad, FP32 amplitude caches (2 x 128 B/event) + time, adjoint gradient" if grad
                     else "goo_nll, FP64 amplitude caches (2 x 240 B/event) + time")}
    out["parity_this_run"] = {"nll_f32": nll["f32"], "nll_f64": nll["f64"],
                              "rel": abs(nll["f32"] - nll["f64"]) / abs(nll["f64"])}
    return out


# ---------------------------------------------------------------------------------------
# served toy-MC study
# ---------------------------------------------------------------------------------------
def c5_study(goo, ctx, n_toys=4096, rate=None, plain_sample=8, n_mc=1_000_000, seed0=1710100):
    import numpy as np

    import synth
    spec = synth.c3_spec(n_mc=n_mc)
    kin = synth.DALITZ_MASSES
    mc = synth.round_to_f32(synth.dalitz_candidates(n_mc, 1710013, kin["M"], kin["m1"], kin["m2"], kin["m3"]), spec)
    mcds = goo.Dataset.from_spec(ctx, spec, mc)
    model = goo.Model(ctx, spec, mc=mcds)
    theta = np.array(synth.param_values(spec))
    free = np.array([not p[2] for p in spec["params"]])
    steps = np.array([p[3] if p[3] > 0 else 1.0 for p in spec["params"]])
    sizes = synth.toy_sizes(n_toys)
    rng = np.random.default_rng(1710098)
    arrivals = np.zeros(n_toys) if rate is None else np.cumsum(rng.exponential(1.0 / rate, n_toys))
    server = goo.Server(model, theta)
    submitted, pending = {}, {}
    finish = np.full(n_toys, np.nan)
    results = {}
    t0 = time.perf_counter()
    nxt = 0
    last_done = 0
    rounds = 0
    while True:
        now = time.perf_counter() - t0
        while nxt < n_toys and arrivals[nxt] <= now:
            tk = server.submit(int(sizes[nxt]), seed0 + nxt)
            submitted[nxt] = tk
            pending[tk] = nxt
            nxt += 1
        q, a, d = server.step()
        rounds += 1
        if d != last_done:
            now = time.perf_counter() - t0
            for tk in server.finished():
                i = pending.pop(tk)
                finish[i] = now
                results[i] = server.result(tk)
            last_done = d
        if nxt == n_toys and q == 0 and a == 0:
            break
        if nxt < n_toys and q == 0 and a == 0:
            time.sleep(max(0.0, min(arrivals[nxt] - (time.perf_counter() - t0), 0.01)))
    wall = time.perf_counter() - t0
    lat = finish - arrivals
    stats = server.stats()
    statuses = np.array([results[i][2]["status"] for i in range(n_toys)])
    out = {"toys": n_toys, "events_total": int(sizes.sum()), "arrival": "all at once" if rate is None
           else f"Poisson, {rate:g} fits/s", "wall_s": wall, "fits_per_s": n_toys / wall,
           "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
           "rounds": int(stats["rounds"]), "generation_s": stats["gen_ms"] / 1e3,
           "generator_acceptance": stats["accepted"] / max(stats["candidates"], 1.0),
           "envelope_violations": int(stats["envelope_violations"]), "converged": int((statuses == 0).sum())}
    # the fits that ended without EDM < tolerance: status 1 iteration limit, 2 line search found
    # no decrease, 3 final Hessian not positive definite
    out["not_converged"] = [{"toy": int(i), "events": int(sizes[i]), "status": int(results[i][2]["status"]),
                             "edm": float(results[i][2]["edm"]), "iterations": int(results[i][2]["iterations"]),
                             "nll": float(results[i][2]["nll"])}
                            for i in range(n_toys) if results[i][2]["status"] != 0][:16]
    if plain_sample:
        # the plain form: per-fit serial FP64 with the finite-difference gradient, same toys,
        # on a sample stratified over the log-uniform event counts (the toys at the quantiles
        # (2q + 1) / (2 plain_sample) of the sizes), so that its mean fit time stands for the
        # whole study's
        order = np.argsort(sizes, kind="stable")
        sample = [int(order[(2 * q + 1) * n_toys // (2 * plain_sample)]) for q in range(plain_sample)]
        t_plain = 0.0
        worst = 0.0
        for i in sample:
            a, b = goo.toy_generate(model, theta, None, seed0 + i, int(sizes[i]))  # the server's toys
            ds = goo.Dataset.from_spec(ctx, spec, {"s12": a.astype(np.float64), "s13": b.astype(np.float64)})
            model.nll(ds, theta, "f64")   # builds the FP64 amplitude cache outside the timing
            tp = time.perf_counter()
            th, err, info = model.fit(ds, theta, free, steps, precision="f64", gradient="fd")
            t_plain += time.perf_counter() - tp
            idx = np.flatnonzero(free)
            worst = max(worst, float(np.max(np.abs(results[i][0][idx] - th[idx]) / err[idx])))
        out["plain_fp64_fd"] = {"fits_per_s": len(sample) / t_plain,
                                "sample": f"{len(sample)} toys at the quantiles (2q+1)/{2 * len(sample)} of the event "
                                          f"counts ({', '.join(str(int(sizes[i])) for i in sample)} events), goo_fit "
                                          "FP64 + central-difference gradient",
                                "max_abs_diff_sigma_vs_served": worst}
        out["speedup_vs_plain"] = out["fits_per_s"] / out["plain_fp64_fd"]["fits_per_s"]
    return out


def run_profile(args):
    """Short fixed launch sequences for ncu captures.

    c2: 4 FP32+grad evaluations (one event kernel each: the kernel specialised for the model
        at run time, normalising the grid itself), then one FP64 evaluation (grid kernel, then
        the scalar event kernel), 10M events.
    c3: amplitude caches and Gram (first call), then 4 FP32+grad and 1 FP64 coherent
        evaluations on 5M events generated on the device.
    c3f: the same events with floating lineshapes: 4 FP32+grad evaluations (an MC pass and an
        event pass each), then 1 FP64 evaluation.
    c4: amplitude caches and Gram (first call), then 4 FP32+grad and 1 FP64 time-dependent
        four-body evaluations on 2M events.
    td3: amplitude caches and Gram matrices (first call), then 4 FP32+grad and 1 FP64
        time-dependent three-body evaluations on 2M events.
    c5: a served study of 64 toys (generation passes, then rounds of batched evaluation and
        minimiser updates).
    """
    import numpy as np

    import synth
    from paper_1710_08826_gb300 import build
    build()
    from paper_1710_08826_gb300 import goo
    ctx = goo.Context(0)
    w = args.profile_workload
    if w in ("c4", "td3"):
        spec, data, mc = c4_inputs(2_000_000, 3_000_000) if w == "c4" else td3_inputs(2_000_000, 1_000_000)
        mcds = goo.Dataset.from_spec(ctx, spec, mc)
        model = goo.Model(ctx, spec, mc=mcds)
        ds = goo.Dataset.from_spec(ctx, spec, data)
        theta = np.array(synth.param_values(spec))
        out = [model.nll_grad(ds, theta, "f32")[0] for _ in range(4)]
        out.append(model.nll(ds, theta, "f64"))
    elif w == "c2":
        spec = synth.c2_spec(bins=GRID)
        cols = synth.gen_c2(n=args.events, seed=1710002)
        ds = goo.Dataset.from_spec(ctx, spec, cols, dtype="f64")
        model = goo.Model(ctx, spec)
        theta = np.array(synth.param_values(spec))
        out = [model.nll_grad(ds, theta, "f32")[0] for _ in range(4)]
        out.append(model.nll(ds, theta, "f64"))
    else:
        spec = synth.c3_spec()
        kin = synth.DALITZ_MASSES
        mc = synth.round_to_f32(synth.dalitz_candidates(1_000_000, 1710013, kin["M"], kin["m1"], kin["m2"], kin["m3"]),
                                spec)
        mcds = goo.Dataset.from_spec(ctx, spec, mc)
        model = goo.Model(ctx, spec, mc=mcds)
        theta = np.array(synth.param_values(spec))
        if w in ("c3", "c3f"):
            a, b = goo.toy_generate(model, theta, None, 1710003, 5_000_000)
            ds = goo.Dataset.from_spec(ctx, spec, {"s12": a.astype(np.float64), "s13": b.astype(np.float64)})
            if w == "c3f":
                model.set_lineshapes("floating")
            out = [model.nll_grad(ds, theta, "f32")[0] for _ in range(4)]
            out.append(model.nll(ds, theta, "f64"))
        else:
            server = goo.Server(model, theta)
            sizes = synth.toy_sizes(64)
            for i, n in enumerate(sizes):
                server.submit(int(n), 1710100 + i)
            rounds = 0
            while True:
                q, a_, d = server.step()
                rounds += 1
                if q == 0 and a_ == 0:
                    break
            out = [rounds, d]
    print(json.dumps({"profile": w, "result": out, "launches": ctx.launches}))
    return 0


def main():
    args = parse()
    if args.profile:
        return run_profile(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
