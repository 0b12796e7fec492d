"""Throughput of the limited-1PN N-body step on B300: 1PN pair interactions/s.

One step = one kick-drift-kick leapfrog step through the C ABI (pn_step):
kick/drift, prologue, pass 1, pass 2, epilogue, hole reduction -- the whole
hot path -- over the full synthetic workload.  An interaction is one ordered
pair of bodies (i, j), i != j, in one acceleration evaluation, so a step of
N bodies counts N (N - 1).

Usage:
    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--precision mixed|fp64] [--impl reference]

Default workload: 131072 bodies (hole of mass 0.76 + Plummer stars, 1% on
e = 0.9 orbits about the hole), c = 30, eps = 5e-5, dt = 1/8192, mixed
precision, 200 steps.  Prints ONE JSON line on rank 0.

--impl reference times the FP64 CPU oracle (the checker of this library, as
it stands) on the host cores, each step a bounded sample of the same
evaluation (a fixed number of star rows and hole rows of the O(N^2) work),
scaled to interactions/s.

With --gpus N > 1 (launched by torch.distributed.run) every rank runs an
independent replica of the workload on its own GPU (the path has no
cross-GPU exchange in this build): value = all ranks' interactions / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1PN pair interactions/s at N=16k/128k, mixed vs FP64 on B300 at <=1e-5 rel err"
FLOPS_PASS1 = 29   # hand count of the mixed pass-1 pair body (FMA = 2, rsqrt = 1)
FLOPS_PASS2 = 67   # hand count of the mixed pass-2 pair body
FLOPS_FUSED = 77   # hand count of the scalar fused pair body (pass 1 + pass 2 sharing x, r, rsqrt)
FLOPS_F64_FUSED = 71   # hand count of the fused double-precision pair body (rsqrt counted as 1)
FLOPS_PACKED = 73  # hand count of the packed fused pair body, law-of-cosines form (r_near > 0):
                   # 46 FP32-pipe operations, 26 of them FMA, + 1 rsqrt
OPS_PACKED = 46    # FP32-pipe operations per pair of that body (FMA, add and mul count 1 each)
FLOPS_PACKED_FAR = 67  # the same body on far units of the spatial order (x_ij from the high
                       # parts: 6 adds fewer)
OPS_PACKED_FAR = 40
FLOPS_JERK = 199   # hand count of the FP32 dual-number pair body of the jerk (mixed contexts,
                   # sources beyond r_near, the law-of-cosines hole term; nearer sources 207;
                   # the FP64 contexts' body, D form and the Wr sum: 213)
FLOPS_ENERGY = 44  # hand count of the FP64 energy pair body (Eq. 7-8 sums; FMA = 2, the
                   # rsqrt seed 1, its Newton step 5)
OPS_ENERGY_DS = 355  # FP32-pipe operations per pair of the double-single energy body (mixed
                     # contexts; ncu's FMA-pipe instruction count gives the same)
                   # (dual add 2, dual multiply 4, scalar x dual 2, rsqrt + its derivative 6)
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="plummer128k_ecc")
    ap.add_argument("--bodies", type=int, default=None,
                    help="override the workload's body count (smaller profiling cases)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--pair-kernel", default="fused", choices=["fused", "two_pass"])
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-16k", action="store_true")
    ap.add_argument("--steps-16k", type=int, default=1000)
    ap.add_argument("--batched-steps", type=int, default=500)
    ap.add_argument("--no-jerk", action="store_true")
    ap.add_argument("--no-energy", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=1000)
    ap.add_argument("--no-adjoint-fd", action="store_true",
                    help="skip the FP64 central-difference check of the adjoint")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the per-workload accuracy report against the oracle")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


# ------------------------------------------------------------- clocks --

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
              "clocks.mem")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # the raw samples: $PN_BENCH_CLOCKS_DIR (default: the system temp dir)
        d = os.environ.get("PN_BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"pn_bench_clocks_gpu{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        sm, smax, mem, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
            if len(parts) > 8:
                try:
                    mem.append(float(parts[8]))
                except ValueError:
                    pass
        if not sm:
            return None
        load = [s for s in sm if s > 0.5 * max(sm)]
        out = {"sm_mhz": float(np.median(load)), "sm_max_mhz": float(max(smax)),
               "reasons": sorted(reasons), "samples": len(sm)}
        if mem:
            out["mem_mhz"] = float(np.median(mem))
        return out


# ---------------------------------------------------------- CPU oracle --

def oracle_rate(x, v, m, w, star_rows: int, hole_rows: int, seed: int = 0):
    """Time the oracle on `star_rows` star targets (each a full sum over all
    bodies) plus `hole_rows` rows of the hole's O(N^2) double sum, and scale
    to interactions/s of a full evaluation (N - 1 of each kind of row)."""
    import oracle
    n = w.n
    rng = np.random.default_rng(seed)
    stars = rng.choice(np.arange(1, n), size=min(star_rows, n - 1), replace=False)
    js = rng.choice(np.arange(1, n), size=min(hole_rows, n - 1), replace=False)
    t0 = time.perf_counter()
    oracle.accel_rows(x, v, m, stars, G=w.G, c=w.c, eps=w.eps)
    t1 = time.perf_counter()
    oracle.bh_rows(x, v, m, js, G=w.G, eps=w.eps)
    t2 = time.perf_counter()
    per_eval = (n - 1) * ((t1 - t0) / len(stars) + (t2 - t1) / len(js))
    return n * (n - 1) / per_eval, t2 - t0, oracle.threads()


def oracle_extra(x, v, m, w, one_core_rows: int = 256):
    """The oracle on one host core (a smaller row sample of the same
    evaluation), and whole evaluations of the 1k and 16k workloads on all
    cores, in interactions/s: N(N - 1) over the time of one full oracle.accel
    call, the hole's double sum included."""
    import oracle
    from paper_1801_07986_b300.inputs import WORKLOADS
    cores = oracle.threads()
    out = {}
    try:
        oracle.set_threads(1)
        r1, secs1, _ = oracle_rate(x, v, m, w, one_core_rows, one_core_rows, seed=7)
        out["one_core"] = {"value": r1, "cores": 1,
                           "sample": f"{one_core_rows} star rows + {one_core_rows} hole "
                                     f"double-sum rows of the N={w.n} evaluation ({secs1:.1f} s)"}
    finally:
        oracle.set_threads(cores)
    full = {}
    for name in ("plummer1k_fp64", "plummer16k"):
        wk = WORKLOADS[name]
        xk, vk, mk = wk.state()
        t0 = time.perf_counter()
        oracle.accel(xk, vk, mk, G=wk.G, c=wk.c, eps=wk.eps)
        t = time.perf_counter() - t0
        full[name] = {"n_bodies": wk.n, "value": wk.n * (wk.n - 1) / t, "seconds": t}
    out["full_evaluations"] = full
    return out


def run_reference(args, w):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    x, v, m = w.state()
    steps = args.steps if args.steps is not None else 20
    # each step a bounded sample of the evaluation: `rows` star rows and
    # `rows` rows of the hole's double sum (each row a full O(N) sum), so the
    # K + W steps end within a few minutes on the host cores
    rows = max(16, min(w.n - 1, 1024))
    for _ in range(args.warmup):
        oracle_rate(x, v, m, w, rows, rows, seed=1)
    rates, secs = [], 0.0
    for k in range(steps):
        r, t, cores = oracle_rate(x, v, m, w, rows, rows, seed=100 + k)
        rates.append(r)
        secs += t
    value = len(rates) / sum(1.0 / r for r in rates)
    sample = (f"each step: {rows} star rows + {rows} hole double-sum rows of the N={w.n} "
              f"evaluation ({1e3 * secs / steps:.0f} ms, the line's ms_per_step), scaled to "
              f"interactions/s by (N-1)/rows; a whole evaluation would take "
              f"{w.n * (w.n - 1) / value:.0f} s")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "interactions/s",
        "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / steps,
        "interactions_per_step": 2.0 * rows * (w.n - 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(w, "fp64", args),
        "cpu_baseline": {"value": value, "unit": "interactions/s", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "interactions/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def config_of(w, precision, args):
    return {"workload": w.name, "n_bodies": w.n, "m_bh": w.m_bh, "c": w.c, "eps": w.eps,
            "dt": w.dt, "precision": precision, "ecc_frac": w.ecc_frac,
            "parallelism": "replicas" if args.gpus > 1 else "single",
            "l2": "256 MiB buffer written between timed steps"}


# ---------------------------------------------------------------- GPU --

# Source region of each measured kernel (from its first line to the next
# section marker), so that a committed ncu traffic figure stays valid only
# while that kernel's own source is unchanged.
_FUSED_REGION = ("// The pair terms, shared by the two-pass and the fused kernels.",
                 "// Sums, for every star slot, the stream-K segments that cover its target")
_KERNEL_REGIONS = {"fused_mixed": _FUSED_REGION, "fused_packed": _FUSED_REGION}


def _code_only(text: str) -> str:
    """Source text without // comments and blank lines, so that a committed
    measurement stays tied to the code it measured, not to its comments."""
    out = []
    for line in text.splitlines():
        code = line.split("//", 1)[0].rstrip()
        if code:
            out.append(code)
    return "\n".join(out)


def kernel_source_hash(tag: str | None = None):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1801_07986_b300", "csrc")
    if tag in _KERNEL_REGIONS:
        text = open(os.path.join(csrc, "pn_kernels.cu")).read()
        a, b = _KERNEL_REGIONS[tag]
        i0 = text.find(a)
        i1 = text.find(b, i0)
        if i0 >= 0 and i1 > i0:
            region = _code_only(text[i0:i1])
            h.update(region.encode())
            # the header's compile-time tunables that the region names
            hdr = open(os.path.join(csrc, "pn_internal.h")).read().splitlines()
            used = []
            for l in hdr:
                m = re.match(r"constexpr\s+[\w:<>\s]+?\b(\w+)\s*=", l)
                if m and re.search(rf"\b{m.group(1)}\b", region):
                    used.append(l)
            h.update(_code_only("\n".join(used)).encode())
            return h.hexdigest()[:16]
    for f in ("pn_kernels.cu", "pn_internal.h"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_tag: str, inst: str = ""):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source and on the instantiation `inst` that runs
    (else None)."""
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None
    src = kernel_source_hash(kernel_tag)
    for f in sorted(os.listdir(d)):
        if not f.endswith(".md"):
            continue
        txt = open(os.path.join(d, f)).read()
        m1 = re.search(rf"traffic_bytes_per_launch\[{re.escape(kernel_tag + inst)}\]:\s*([0-9.eE+]+)",
                       txt)
        m2 = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
        if m1 and m2 and m2.group(1) == src:
            return float(m1.group(1))
    return None


def run_native(args, w):
    import torch
    from paper_1801_07986_b300 import pn

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    steps = args.steps if args.steps is not None else w.steps
    x, v, m = w.state()
    X = torch.tensor(x, device=dev)
    V = torch.tensor(v, device=dev)
    M = torch.tensor(m, device=dev)
    A = torch.empty_like(X)
    stream = torch.cuda.current_stream(dev)
    ctx = pn.pn_init(w.n, G=w.G, c=w.c, eps=w.eps, precision=args.precision, device=local,
                     stream=stream, pair_kernel=args.pair_kernel)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    pn.pn_accel(ctx, X, V, M, A)
    for _ in range(args.warmup):
        pn.pn_step(ctx, X, V, M, A, w.dt, 1)
    pn.pn_sync(ctx)

    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    # the state the timed steps start from (the end-to-end run repeats them)
    start_state = None if args.no_e2e else (X.cpu().numpy(), V.cpu().numpy(), A.cpu().numpy())
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    pn.pn_set_timing(ctx, True)
    launches0 = pn.pn_launch_count(ctx)
    with ClockSampler(local) as clk:
        for k in range(steps):
            flush.zero_()
            ev0[k].record(stream)
            pn.pn_step(ctx, X, V, M, A, w.dt, 1)
            ev1[k].record(stream)
        torch.cuda.synchronize(dev)
    pn.pn_sync(ctx)
    launches = pn.pn_launch_count(ctx) - launches0
    kms, klaunch = pn.pn_get_timing(ctx)
    far_units, all_units = pn.pn_get_pair_stats(ctx)
    pn.pn_set_timing(ctx, False)
    ms = float(sum(a.elapsed_time(b) for a, b in zip(ev0, ev1)))
    if world > 1:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
        torch.distributed.barrier()
    inter = float(w.n) * (w.n - 1) * steps * world
    value = inter / (ms * 1e-3)
    launch = pn.pn_get_launch(ctx)
    variant = pn.pn_get_variant(ctx)
    if variant["targets_per_thread"]:
        launch.update({k: variant[k] for k in ("unroll", "form", "stages")})

    # roofline of the dominant pair kernel (plain FP32 ALU bound)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    sms = launch["sms"]
    peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    k_dom = int(np.argmax(kms[:2]))
    per_launch_ms = kms[k_dom] / max(1, klaunch[k_dom])
    pairs = float(w.n - 1) * (w.n - 2)
    fused = args.precision == "mixed" and args.pair_kernel == "fused"
    f64_fused = args.precision == "fp64" and args.pair_kernel == "fused"
    packed = fused and bool(launch.get("packed"))
    # share of the pairs the spatially ordered packed kernel took through its
    # far-unit body (device counters; 0 without the spatial order)
    far_frac = far_units / all_units if packed and all_units else 0.0
    fpp = (FLOPS_PACKED - far_frac * (FLOPS_PACKED - FLOPS_PACKED_FAR) if packed else FLOPS_FUSED) \
        if fused else (FLOPS_F64_FUSED if f64_fused else (FLOPS_PASS2 if k_dom == 1 else FLOPS_PASS1))
    flops = fpp * pairs
    achieved = flops / (per_launch_ms * 1e-3) / 1e12
    clocks = clk.summary()
    inst = ""
    if fused:
        tag = "fused_packed" if launch.get("packed") else "fused_mixed"
        # the instantiation the traffic was captured on
        # (k_fused_packed<NP, UNROLL, FORM, TILE, ST>, NP = targets / 2; the scalar
        # k_fused_mixed<P, UNROLL>)
        if launch.get("packed"):
            inst = "<{},{},{},{},{}>".format(variant["targets_per_thread"] // 2, variant["unroll"],
                                             variant["form"], variant["tile"], variant["stages"])
        else:
            inst = "<{},{}>".format(variant["targets_per_thread"], variant["unroll"])
    elif f64_fused:
        tag = "fused_f64"
    else:
        tag = f"pass{k_dom + 1}_{args.precision}"
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": profiled_traffic(tag, inst), "kernel": tag + inst,
            "flops_per_pair": fpp,
            "launch_ms": per_launch_ms,
            "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz "
                          "(sm_max_mhz of MEASURED_PEAKS.json)",
            "kernel_ms_share": {"pass1": kms[0] / ms, "pass2_or_fused": kms[1] / ms,
                                "near": kms[2] / ms}}
    if clocks and clocks.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = achieved / (peak * clocks["sm_mhz"] / sm_max)
    if packed:
        # the FP32 pipe's own limit: operations issued per pair against its
        # lane-operation rate (an FMA is one operation and two flops)
        opp = OPS_PACKED - far_frac * (OPS_PACKED - OPS_PACKED_FAR)
        ops = opp * pairs / (per_launch_ms * 1e-3)
        roof["far_unit_fraction"] = far_frac
        roof["fp32_pipe_ops_per_pair"] = opp
        roof["fp32_pipe_frac"] = ops / (sms * FP32_LANES_PER_SM * sm_max * 1e6)
    try:
        meas = pn.pn_measure_peaks(local, stream)
        roof["fp32_fma_microbench_tflops"] = meas["fp32_fma_tflops"]
        roof["frac_of_fma_microbench"] = achieved / meas["fp32_fma_tflops"]
        roof["fp64_fma_microbench_tflops"] = meas["fp64_fma_tflops"]
        roof["fp32x2_fma_microbench_tflops"] = meas["fp32x2_fma_tflops"]
        if args.precision == "fp64":
            # the double-precision path is bound by the FP64 pipe: its peak
            # is the measured FP64 FMA rate (no nominal FP64 figure is given)
            roof["peak"] = meas["fp64_fma_tflops"]
            roof["frac"] = achieved / roof["peak"]
            roof["peak_basis"] = "FP64 FMA-chain microbenchmark on this device (pn_measure_peaks)"
            roof.pop("frac_at_sampled_clock", None)
    except Exception as e:  # reported, not required
        roof["fp32_fma_microbench_error"] = str(e)[:200]
    roof["flops_per_interaction"] = fpp if (fused or f64_fused) else FLOPS_PASS1 + FLOPS_PASS2

    line = {
        "metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": ms / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "mixed" else "f64",
        "data": "synthetic", "config": config_of(w, args.precision, args),
        "roofline": roof, "gpu_launches": launches, "clocks": clocks,
        "launch_shape": launch,
    }

    # end to end through the host-array entry point, copies inside the timing:
    # the first e2e_steps of the timed run again, from the same state, so that
    # they compare with the device-timed ms of those steps
    if not args.no_e2e:
        e2e_steps = max(3, min(steps, 50))
        dev_ms = float(sum(a.elapsed_time(b) for a, b in zip(ev0[:e2e_steps], ev1[:e2e_steps])))
        pin = lambda a: torch.tensor(a).pin_memory().numpy()
        xh, vh, mh = pin(x), pin(v), pin(m)
        ah = pin(A.cpu().numpy())
        pn.pn_step_host(ctx, xh, vh, mh, ah, w.dt, 1)     # warm-up of the host path
        xh[:], vh[:], ah[:] = start_state
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for _ in range(e2e_steps):
            flush.zero_()
            e0.record(stream)
            pn.pn_step_host(ctx, xh, vh, mh, ah, w.dt, 1)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        if world > 1:       # whole job: every rank's steps over the slowest rank's time
            t = torch.tensor([tot, dev_ms], device=dev, dtype=torch.float64)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            tot, dev_ms = float(t[0].item()), float(t[1].item())
        line["e2e"] = {"value": float(w.n) * (w.n - 1) * e2e_steps * world / (tot * 1e-3),
                       "unit": "interactions/s", "h2d_bytes_per_step": 80 * w.n,
                       "d2h_bytes_per_step": 72 * w.n, "steps": e2e_steps,
                       "device_value_same_steps": float(w.n) * (w.n - 1) * e2e_steps * world
                       / (dev_ms * 1e-3),
                       "steps_note": "the first steps of the timed run, again from its start state"}

    # the same workload on the FP64 path (a few steps) for the mixed/FP64 ratio
    if args.precision == "mixed" and not args.no_fp64_compare:
        c64 = pn.pn_init(w.n, G=w.G, c=w.c, eps=w.eps, precision="fp64", device=local,
                         stream=stream)
        X2, V2, A2 = X.clone(), V.clone(), A.clone()
        pn.pn_step(c64, X2, V2, M, A2, w.dt, 1)
        pn.pn_sync(c64)
        nst = 3 if w.n > 50000 else 20
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pn.pn_step(c64, X2, V2, M, A2, w.dt, nst)
        e1.record(stream)
        e1.synchronize()
        r64 = float(w.n) * (w.n - 1) * nst / (e0.elapsed_time(e1) * 1e-3)
        line["fp64_path"] = {"value": r64, "unit": "interactions/s", "steps": nst,
                             "mixed_over_fp64": value / world / r64}
        c64.close()

    if not args.no_16k and world == 1 and w.name != "plummer16k":
        try:
            line["plummer16k"] = run_16k(local, stream, args.warmup, args.steps_16k)
        except Exception as e:  # reported, not required
            line["plummer16k"] = {"error": str(e)[:300]}

    if not args.no_batched and world == 1:
        try:
            line["batched"] = run_batched(local, stream, args.batched_steps, args.warmup)
        except Exception as e:  # reported, not required
            line["batched"] = {"error": str(e)[:300]}

    if not args.no_jerk and world == 1:
        try:
            line["jerk"] = run_jerk(local, stream, args.warmup)
        except Exception as e:  # reported, not required
            line["jerk"] = {"error": str(e)[:300]}

    if not args.no_energy and world == 1:
        try:
            line["energy"] = run_energy(local, stream)
        except Exception as e:  # reported, not required
            line["energy"] = {"error": str(e)[:300]}

    if not args.no_adjoint and world == 1:
        try:
            line["adjoint"] = run_adjoint(local, stream, args.adjoint_steps,
                                          fd=not args.no_adjoint_fd)
        except Exception as e:  # reported, not required
            line["adjoint"] = {"error": str(e)[:300]}

    if rank == 0 and world == 1 and not args.no_accuracy:
        try:
            line["accuracy"] = run_accuracy(local, stream)
        except Exception as e:  # reported, not required
            line["accuracy"] = {"error": str(e)[:300]}

    if rank == 0 and not args.no_cpu_baseline:
        try:
            rows = max(64, min(w.n - 1, 16384))
            r, secs, cores = oracle_rate(x, v, m, w, rows, rows)
            line["cpu_baseline"] = {
                "value": r, "unit": "interactions/s", "cores": cores, "kind": "oracle",
                "sample": f"{rows} star rows + {rows} hole double-sum rows of the N={w.n} "
                          f"evaluation ({secs:.1f} s), scaled by (N-1)/{rows}"}
            line["cpu_baseline"].update(oracle_extra(x, v, m, w))
        except Exception as e:  # the baseline is reported, not required
            line["cpu_baseline"] = {"value": None, "error": str(e)[:200]}
    ctx.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def run_16k(local, stream, warmup, steps, fp64_steps=10):
    """The 16k Plummer workload (M = 0.05, c = 50, eps = 1e-4, dt = 1/2048):
    `steps` KDK steps in mixed precision and `fp64_steps` in FP64, timed with
    CUDA events on the launching stream (inputs are L2-resident at this size:
    1.3 MB of records); the mixed run's relative energy change (Eq. 7, FP64)
    over its steps.  The mixed steps run as pn_step_graph replays of a
    100-step CUDA graph (the first 100, which capture it, untimed) and, for
    comparison, as one eager pn_step call; the FP64 steps as one pn_step."""
    import torch
    from paper_1801_07986_b300 import pn
    from paper_1801_07986_b300.inputs import WORKLOADS
    w = WORKLOADS["plummer16k"]
    x, v, m = w.state()
    dev = torch.device(f"cuda:{local}")
    out = {"workload": "plummer16k", "n_bodies": w.n, "unit": "interactions/s",
           "l2": "inputs L2-resident (each run's steps timed together)"}
    graph_steps = 100
    for key, prec, nst, graph in (("mixed", "mixed", steps, steps > graph_steps),
                                  ("mixed_eager", "mixed", steps, False),
                                  ("fp64", "fp64", fp64_steps, False)):
        X, V, M = (torch.tensor(a, device=dev) for a in (x, v, m))
        A = torch.empty_like(X)
        ctx = pn.pn_init(w.n, G=w.G, c=w.c, eps=w.eps, precision=prec, device=local,
                         stream=stream)
        pn.pn_accel(ctx, X, V, M, A)
        for _ in range(max(1, warmup)):
            pn.pn_step(ctx, X, V, M, A, w.dt, 1)
        E0 = pn.pn_energy(ctx, X, V, M)["E"]
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        timed = nst
        if graph:
            pn.pn_step_graph(ctx, X, V, M, A, w.dt, graph_steps)     # capture + first run
            timed = (nst - graph_steps) // graph_steps * graph_steps
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(timed // graph_steps):
                pn.pn_step_graph(ctx, X, V, M, A, w.dt, graph_steps)
            e1.record(stream)
        else:
            e0.record(stream)
            pn.pn_step(ctx, X, V, M, A, w.dt, nst)
            e1.record(stream)
        e1.synchronize()
        pn.pn_sync(ctx)
        ms = e0.elapsed_time(e1)
        E1 = pn.pn_energy(ctx, X, V, M)["E"]
        ctx.close()
        out[key] = {"value": float(w.n) * (w.n - 1) * timed / (ms * 1e-3),
                     "steps": graph_steps + timed if graph else nst, "timed_steps": timed,
                     "ms_per_step": ms / timed, "dE_over_E": (E1 - E0) / abs(E0),
                     "launch": "pn_step_graph replays" if graph else "one pn_step call"}
    out["value"] = out["mixed"]["value"]
    out["mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    out["note"] = ("dE_over_E is the integrator's on this workload: between steps 100 and 200 "
                   "a star passes the unsoftened hole closer than one step resolves and leaves "
                   "at |v| ~ 37, in FP64 and mixed alike")
    return out


def run_batched(local, stream, steps, warmup):
    """The batched workload: 64 Plummer clusters, N log-uniform in [512, 32768],
    hole mass U[0.01, 0.2], c U[20, 200]; the fused kernel's shape from the
    autotuner; `steps` KDK steps captured in one CUDA graph and timed as one
    launch (CUDA events on the launching stream)."""
    import torch
    from paper_1801_07986_b300 import pn
    from paper_1801_07986_b300.inputs import batched_workloads
    ws = batched_workloads()
    xs, vs, ms = zip(*(w.state() for w in ws))
    off = np.concatenate([[0], np.cumsum([w.n for w in ws])])
    dev = torch.device(f"cuda:{local}")
    X = torch.tensor(np.concatenate(xs), device=dev)
    V = torch.tensor(np.concatenate(vs), device=dev)
    M = torch.tensor(np.concatenate(ms), device=dev)
    A = torch.empty_like(X)
    ctx = pn.pn_init_batched(off, c=[w.c for w in ws], eps=[w.eps for w in ws],
                             precision="mixed", device=local, stream=stream)
    tuned = pn.pn_tune(ctx, X, V, M, A)
    pn.pn_accel(ctx, X, V, M, A)
    dt = ws[0].dt
    for _ in range(max(1, warmup)):
        pn.pn_step(ctx, X, V, M, A, dt, 1)
    t0 = time.perf_counter()
    pn.pn_step_graph(ctx, X, V, M, A, dt, steps)        # capture + first replay
    pn.pn_sync(ctx)
    capture_s = time.perf_counter() - t0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = pn.pn_launch_count(ctx)
    e0.record(stream)
    pn.pn_step_graph(ctx, X, V, M, A, dt, steps)        # replay, timed
    e1.record(stream)
    launches = pn.pn_launch_count(ctx) - l0
    e1.synchronize()
    pn.pn_sync(ctx)
    ms_tot = e0.elapsed_time(e1)
    inter = float(sum(w.n * (w.n - 1) for w in ws)) * steps
    ctx.close()
    return {"workload": "batched64", "clusters": len(ws), "bodies": int(off[-1]),
            "n_min": int(min(w.n for w in ws)), "n_max": int(max(w.n for w in ws)),
            "steps": steps, "value": inter / (ms_tot * 1e-3), "unit": "interactions/s",
            "ms_per_step": ms_tot / steps, "graph": "all steps in one CUDA graph launch",
            "graph_capture_and_first_run_s": capture_s, "autotuned": tuned,
            "gpu_launches": launches}


def run_jerk(local, stream, warmup, reps=5):
    """The jerk (Appendix A) and the Hermite integrator on the 16k Plummer
    workload in a mixed-precision context: pn_jerk (A, then the dual-number
    jerk pass with single-precision pair sums) timed with CUDA events, and a
    Hermite step (two A + two jerk evaluations) from calls of 2 and 10
    steps."""
    import torch
    from paper_1801_07986_b300 import pn
    from paper_1801_07986_b300.inputs import WORKLOADS
    w = WORKLOADS["plummer16k"]
    x, v, m = w.state()
    dev = torch.device(f"cuda:{local}")
    X, V, M = (torch.tensor(a, device=dev) for a in (x, v, m))
    A, J = torch.empty_like(X), torch.empty_like(X)
    ctx = pn.pn_init(w.n, G=w.G, c=w.c, eps=w.eps, precision="mixed", integrator="hermite",
                     device=local, stream=stream)
    for _ in range(max(1, warmup)):
        pn.pn_jerk(ctx, X, V, M, A, J)
    pn.pn_sync(ctx)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        pn.pn_jerk(ctx, X, V, M, A, J)
    e1.record(stream)
    e1.synchronize()
    ms_jerk = e0.elapsed_time(e1) / reps
    pn.pn_step(ctx, X, V, M, A, w.dt, 1)
    pn.pn_sync(ctx)
    # a call of k Hermite steps costs k steps (two A + two jerk evaluations
    # each) plus the call's own jerk at the entry state and A at the end:
    # calls of 2 and 10 steps separate the two
    call_ms = {}
    for k in (2, 10):
        e0.record(stream)
        pn.pn_step(ctx, X, V, M, A, w.dt, k)
        e1.record(stream)
        e1.synchronize()
        pn.pn_sync(ctx)
        call_ms[k] = e0.elapsed_time(e1)
    ms_step = (call_ms[10] - call_ms[2]) / 8
    ms_call_fixed = call_ms[2] - 2 * ms_step
    ctx.close()
    pairs = float(w.n - 1) * (w.n - 2)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    peak = 148 * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = FLOPS_JERK * pairs / (ms_jerk * 1e-3) / 1e12
    both = (FLOPS_JERK + FLOPS_PACKED) * pairs / (ms_jerk * 1e-3) / 1e12
    return {"workload": "plummer16k", "n_bodies": w.n,
            "value": float(w.n) * (w.n - 1) / (ms_jerk * 1e-3), "unit": "interactions/s",
            "what": "pn_jerk in a mixed context: A + dual-number jerk (FP32 pair sums), "
                    "per evaluation",
            "ms_per_jerk": ms_jerk, "hermite_ms_per_step": ms_step,
            "hermite_ms_per_call_fixed": ms_call_fixed,
            "hermite_note": "per step from calls of 2 and 10 steps; the fixed part is each "
                            "call's jerk at the entry state and its final A",
            "roofline": {"bound": "alu", "achieved": both, "peak": peak, "unit": "TFLOP/s",
                         "frac": both / peak,
                         "peak_basis": f"148 SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                                       f"{sm_max:.0f} MHz",
                         "flops_per_pair": FLOPS_JERK + FLOPS_PACKED,
                         "note": "whole pn_jerk call timed: its whole work, the A evaluation "
                                 "it returns (packed pair body) and the dual jerk body",
                         "achieved_jerk_only": achieved, "frac_jerk_only": achieved / peak,
                         "flops_per_pair_jerk_only": FLOPS_JERK,
                         "note_jerk_only": "the same call time against the dual jerk body's "
                                           "flops alone"}}


def run_energy(local, stream, reps=5):
    """Eq. 7-8 (pn_energy) on the 16k Plummer workload: whole calls timed
    with CUDA events (the prologue, the pair kernel, the per-star and
    per-cluster sums and the 8-double copy back).  A mixed context takes the
    pair sums in double-single arithmetic on the FP32 pipe (roofline: its
    lane-operation rate); beside it an FP64 context's FP64 pair sums
    (roofline: the measured FP64 FMA rate)."""
    import torch
    from paper_1801_07986_b300 import pn
    from paper_1801_07986_b300.inputs import WORKLOADS
    w = WORKLOADS["plummer16k"]
    x, v, m = w.state()
    dev = torch.device(f"cuda:{local}")
    X, V, M = (torch.tensor(a, device=dev) for a in (x, v, m))

    def timed(precision):
        ctx = pn.pn_init(w.n, G=w.G, c=w.c, eps=w.eps, precision=precision, device=local,
                         stream=stream)
        first = pn.pn_energy(ctx, X, V, M)
        pn.pn_sync(ctx)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            pn.pn_energy(ctx, X, V, M)
        e1.record(stream)
        e1.synchronize()
        ctx.close()
        return e0.elapsed_time(e1) / reps, first["E"]

    ms, E = timed("mixed")
    ms64, E64 = timed("fp64")
    pairs = float(w.n - 1) * (w.n - 2)
    meas = pn.pn_measure_peaks(local, stream)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    lane_peak = meas["sms"] * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12      # Tops/s
    achieved = OPS_ENERGY_DS * pairs / (ms * 1e-3) / 1e12
    achieved64 = FLOPS_ENERGY * pairs / (ms64 * 1e-3) / 1e12
    return {"workload": "plummer16k", "n_bodies": w.n, "ms_per_call": ms,
            "value": float(w.n) * (w.n - 1) / (ms * 1e-3), "unit": "interactions/s",
            "what": "pn_energy (Eq. 7 energy, Eq. 8 momentum) in a mixed context: "
                    "double-single pair sums on the FP32 pipe, whole call",
            "E": E, "E_rel_vs_fp64_context": abs(E - E64) / abs(E64),
            "roofline": {"bound": "alu", "pipe": "fp32", "achieved": achieved,
                         "peak": lane_peak, "unit": "Tops/s", "frac": achieved / lane_peak,
                         "peak_basis": f"{meas['sms']} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                                       f"{sm_max:.0f} MHz (operations, an FMA counted once)",
                         "ops_per_pair": OPS_ENERGY_DS,
                         "note": "whole call timed; the pair kernel's operations only"},
            "fp64_context": {"ms_per_call": ms64,
                             "value": float(w.n) * (w.n - 1) / (ms64 * 1e-3),
                             "roofline": {"bound": "alu", "pipe": "fp64", "achieved": achieved64,
                                          "peak": meas["fp64_fma_tflops"], "unit": "TFLOP/s",
                                          "frac": achieved64 / meas["fp64_fma_tflops"],
                                          "peak_basis": "FP64 FMA-chain microbenchmark on this "
                                                        "device (pn_measure_peaks)",
                                          "flops_per_pair": FLOPS_ENERGY}}}


def run_adjoint(local, stream, nsteps, fd=True):
    """The adjoint workload: N = 8192 Plummer cluster (M = 0.1, c = 50,
    dt = 1/2048), loss = sum over the 16 stars nearest the hole at t = 0 of
    |x(T)|^2 after nsteps KDK steps (mixed-precision forward, single-
    precision pair sums in the reverse sweeps), gradient with respect to M,
    c, x0 and v0 through pn_step_vjp with sqrt(T) checkpoints, timed with
    CUDA events.  With `fd`: the same gradient on the FP64 path, both against
    FP64 central differences (adjoint_fd_check), and the mixed gradient
    against the FP64 one over every component."""
    from paper_1801_07986_b300.inputs import WORKLOADS
    w = WORKLOADS["plummer8k_adjoint"]
    state = w.state()
    x = state[0]
    near = np.argsort(np.linalg.norm(x[1:] - x[0], axis=1))[:16] + 1
    xb, vb, gM, gc, s_grad, s_fwd, s_x0 = adjoint_gradient(local, stream, w, state, near,
                                                           nsteps, "mixed", from_x0=True)
    pairs = float(w.n) * (w.n - 1) * nsteps
    out = {"workload": "plummer8k_adjoint", "n_bodies": w.n, "steps": nsteps,
           "checkpoint": "every ceil(sqrt(steps)) steps",
           "loss": "sum over the 16 stars nearest the hole at t=0 of |x(T)|^2",
           "value": pairs / s_grad, "unit": "interactions/s",
           "what": "trajectory steps differentiated per second x N(N-1)",
           "gradient_s": s_grad, "forward_s": s_fwd, "gradient_over_forward": s_grad / s_fwd,
           "gradient_note": "forward = pn_accel + pn_step_save (the steps keeping the "
                            "checkpoints); gradient = pn_step_vjp_saved (re-runs each segment "
                            "once, then the reverse); gradient_from_x0_s = pn_step_vjp, which "
                            "runs the forward itself first (same result, checked bitwise)",
           "gradient_from_x0_s": s_x0,
           "dL_dM": gM, "dL_dc": gc, "grad_x0_norm": float(np.linalg.norm(xb)),
           "grad_v0_norm": float(np.linalg.norm(vb))}
    if fd:
        try:
            x6, v6, gM6, gc6, s6, _, _ = adjoint_gradient(local, stream, w, state, near,
                                                          nsteps, "fp64")
            out["fp64_gradient_s"] = s6
            out["mixed_vs_fp64_adjoint"] = {
                "x0_rel_norm": float(np.linalg.norm(xb - x6) / np.linalg.norm(x6)),
                "v0_rel_norm": float(np.linalg.norm(vb - v6) / np.linalg.norm(v6)),
                "M_rel": abs(gM - gM6) / abs(gM6), "c_rel": abs(gc - gc6) / abs(gc6)}
            out["fd_check"] = adjoint_fd_check(
                local, stream, nsteps, {"mixed": (xb, vb, gM, gc), "fp64": (x6, v6, gM6, gc6)},
                near)
        except Exception as e:  # reported, not required
            out["fd_check"] = {"error": str(e)[:300]}
    return out


# ----------------------------------------------------------- accuracy --

def _rel(a, b):
    """Per-body relative error |a - b| / |b| (rows of n x 3 arrays)."""
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


def _stats(err):
    err = np.asarray(err, dtype=np.float64)
    return {"median": float(np.median(err)), "max": float(np.max(err)), "bodies": int(err.size)}


def _divergence(x, v, xr, vr):
    """Trajectory divergence of (x, v) from the reference (xr, vr): the largest
    position and velocity differences, relative to the largest reference
    coordinate."""
    return {"x": float(np.abs(x - xr).max() / np.abs(xr).max()),
            "v": float(np.abs(v - vr).max() / np.abs(vr).max())}


class _GpuRun:
    """One workload stepped through pn_step; accel() is A on the current state
    (a separate buffer, so the carried acceleration is untouched)."""

    def __init__(self, w, precision, local, stream, state=None):
        import torch
        from paper_1801_07986_b300 import pn
        self.pn, self.w = pn, w
        x, v, m = w.state() if state is None else state
        self.m = m
        dev = torch.device(f"cuda:{local}")
        self.ctx = pn.pn_init(w.n, G=w.G, c=w.c, eps=w.eps, precision=precision, device=local,
                              stream=stream)
        self.X, self.V, self.M = (torch.tensor(a, device=dev) for a in (x, v, m))
        self.A = torch.empty_like(self.X)
        self.B = torch.empty_like(self.X)
        pn.pn_accel(self.ctx, self.X, self.V, self.M, self.A)

    def step(self, k):
        self.pn.pn_step(self.ctx, self.X, self.V, self.M, self.A, self.w.dt, k)

    def state(self):
        self.pn.pn_sync(self.ctx)
        return self.X.cpu().numpy(), self.V.cpu().numpy()

    def accel(self):
        self.pn.pn_accel(self.ctx, self.X, self.V, self.M, self.B)
        self.pn.pn_sync(self.ctx)
        return self.B.cpu().numpy()

    def energy(self):
        return self.pn.pn_energy(self.ctx, self.X, self.V, self.M)["E"]

    def close(self):
        self.ctx.close()


def accuracy_c1(local, stream, oracle_traj):
    """1k FP64 workload, as configured (100 steps): the same-state force error
    against the oracle at every step (every body), the divergence of the
    final state from the oracle's own 100 steps, and the energy change."""
    import oracle
    from paper_1801_07986_b300.inputs import WORKLOADS
    w = WORKLOADS["plummer1k_fp64"]
    r = _GpuRun(w, "fp64", local, stream)
    worst, per_step = 0.0, []
    E0 = r.energy()
    for s in range(w.steps + 1):
        if s:
            r.step(1)
        x, v = r.state()
        err = _rel(r.accel(), oracle.accel(x, v, r.m, G=w.G, c=w.c, eps=w.eps))
        per_step.append(float(err.max()))
        worst = max(worst, float(err.max()))
    E1 = r.energy()
    r.close()
    xo, vo = oracle_traj.result()
    return {"precision": "fp64", "steps": w.steps, "bodies_checked_per_step": w.n,
            "force_err_max_all_steps": worst,
            "force_err_median_of_step_max": float(np.median(per_step)),
            "divergence_vs_oracle_trajectory": _divergence(x, v, xo, vo),
            "dE_over_E": (E1 - E0) / abs(E0), "tolerance": 1e-12}


def accuracy_c2(local, stream, oracle_prefix, prefix_steps, rows=256):
    """16k workload, 1000 steps in mixed precision and in FP64: the same-state
    force error at steps 0, 100, ..., 1000 (sampled stars; the hole at the
    first and last check), the energy change, the divergence of both runs
    from the oracle's own trajectory over its first `prefix_steps` steps, and
    the divergence of the mixed run from the FP64 run every 100 steps."""
    import oracle
    from paper_1801_07986_b300.inputs import WORKLOADS
    w = WORKLOADS["plummer16k"]
    out = {"steps": w.steps, "rows_per_check": rows, "hole_checked_at": [0, w.steps]}
    traj = {}
    for prec in ("mixed", "fp64"):
        r = _GpuRun(w, prec, local, stream)
        rng = np.random.default_rng(16)
        checks, states = [], {}
        E0 = r.energy()
        s = 0
        marks = sorted(set([0, prefix_steps] + list(range(100, w.steps + 1, 100))))
        for target in marks:
            if target > s:
                r.step(target - s)
                s = target
            x, v = r.state()
            states[s] = (x, v)
            if s % 100:
                continue
            idx = list(rng.choice(np.arange(1, w.n), rows, replace=False))
            if s in (0, w.steps):
                idx = [0] + idx
            err = _rel(r.accel()[idx], oracle.accel_rows(x, v, r.m, idx, G=w.G, c=w.c,
                                                         eps=w.eps))
            checks.append({"step": s, **_stats(err)})
        E1 = r.energy()
        r.close()
        traj[prec] = states
        out[prec] = {"same_state_force_err": checks,
                     "force_err_median_max_over_checks": max(c["median"] for c in checks),
                     "force_err_max_over_checks": max(c["max"] for c in checks),
                     "dE_over_E": (E1 - E0) / abs(E0)}
    xo, vo = oracle_prefix.result()
    for prec in ("mixed", "fp64"):
        x, v = traj[prec][prefix_steps]
        out[prec]["divergence_vs_oracle_trajectory"] = {"steps": prefix_steps,
                                                        **_divergence(x, v, xo, vo)}
    out["mixed_vs_fp64_divergence"] = [
        {"step": s, **_divergence(*traj["mixed"][s], *traj["fp64"][s])}
        for s in range(100, w.steps + 1, 100)]
    out["tolerance"] = {"fp64": 1e-12, "mixed_median": 2e-7, "mixed_max": 1e-5}
    return out


def accuracy_c3(local, stream, prefix_steps=3, rows_ecc=64, rows_plummer=192):
    """128k eccentric workload, 200 mixed steps: the same-state force error at
    steps 0, 50, ..., 200 on sampled stars of both populations (the hole's
    O(N^2) double sum is left out: a full oracle evaluation of it takes
    minutes on the host), and the divergence of the mixed run from the FP64
    run over the first `prefix_steps` steps (its trajectories are outside
    the 1PN regime and chaotic, so only same-state parity is a gate)."""
    import oracle
    from paper_1801_07986_b300.inputs import WORKLOADS
    w = WORKLOADS["plummer128k_ecc"]
    n_ecc = int(round(w.ecc_frac * (w.n - 1)))
    r = _GpuRun(w, "mixed", local, stream)
    rng = np.random.default_rng(128)
    checks, s, pref = [], 0, None
    for target in sorted(set([prefix_steps] + list(range(0, w.steps + 1, 50)))):
        if target > s:
            r.step(target - s)
            s = target
        x, v = r.state()
        if s == prefix_steps:
            pref = (x, v)
        if s % 50:
            continue
        idx = np.concatenate([rng.choice(np.arange(1, n_ecc + 1), rows_ecc, replace=False),
                              rng.choice(np.arange(n_ecc + 1, w.n), rows_plummer, replace=False)])
        got = r.accel()[idx]
        want = oracle.accel_rows(x, v, r.m, idx, G=w.G, c=w.c, eps=w.eps)
        err = _rel(got, want)
        checks.append({"step": s, **_stats(err), "eccentric": _stats(err[:rows_ecc])})
    r.close()
    f = _GpuRun(w, "fp64", local, stream)
    f.step(prefix_steps)
    xf, vf = f.state()
    f.close()
    return {"steps": w.steps, "rows_per_check": rows_ecc + rows_plummer,
            "same_state_force_err": checks,
            "force_err_median_max_over_checks": max(c["median"] for c in checks),
            "force_err_max_over_checks": max(c["max"] for c in checks),
            "divergence_vs_fp64_gpu": {"steps": prefix_steps, **_divergence(*pref, xf, vf)},
            "tolerance": {"mixed_median": 2e-7, "mixed_max": 1e-5}}


def run_accuracy(local, stream, prefix_16k=10):
    """Every configured workload's accuracy against the FP64 oracle, as
    configured (not timed).  The oracle's own trajectories (1k: 100 steps;
    16k: the first `prefix_16k` steps) run on the host cores in a thread
    while the GPU runs."""
    import concurrent.futures as cf
    import oracle
    from paper_1801_07986_b300.inputs import WORKLOADS
    w1, w2 = WORKLOADS["plummer1k_fp64"], WORKLOADS["plummer16k"]

    def own(w, nst):
        x, v, m = w.state()
        a = oracle.accel(x, v, m, G=w.G, c=w.c, eps=w.eps)
        xo, vo, _ = oracle.step(x, v, m, a, w.dt, nst, G=w.G, c=w.c, eps=w.eps)
        return xo, vo

    out = {}
    with cf.ThreadPoolExecutor(max_workers=1) as ex:
        f1 = ex.submit(own, w1, w1.steps)
        f2 = ex.submit(own, w2, prefix_16k)
        for key, fn in (("plummer1k_fp64", lambda: accuracy_c1(local, stream, f1)),
                        ("plummer16k", lambda: accuracy_c2(local, stream, f2, prefix_16k)),
                        ("plummer128k_ecc", lambda: accuracy_c3(local, stream))):
            try:
                out[key] = fn()
            except Exception as e:  # reported, not required
                out[key] = {"error": str(e)[:300]}
    return out


# Central-difference steps of the adjoint check: absolute in the hole mass,
# the initial positions and the initial velocities; relative in c, whose
# gradient is five orders smaller than dL/dM on the adjoint workload, so
# its difference takes a larger step to stay above the FP64 rounding of the
# perturbed runs.
ADJ_FD_H = 1e-8
ADJ_FD_H_C = 1e-6
# Components of dL/dx0 and dL/dv0 below ADJ_FD_SMALL_G take the larger step
# ADJ_FD_H_SMALL: the rounding noise of a difference is about the same
# absolute size for every parameter (3e-3 at h = 1e-8 over 1000 steps of the
# adjoint workload), so a small component needs a larger step to rise above
# it.
ADJ_FD_SMALL_G = 1e3
ADJ_FD_H_SMALL = 1e-6


def adjoint_gradient(local, stream, w, state, near, nsteps, precision, from_x0=False):
    """Gradient of the adjoint workload's loss (sum over the stars `near` of
    |x(T)|^2 after nsteps KDK steps) with sqrt(T) checkpoints: the forward
    keeps its checkpoints (pn_step_save), the backward starts from them
    (pn_step_vjp_saved).  Returns (xbar0, vbar0, dL/dM, dL/dc, backward
    seconds, forward seconds, and with from_x0 the seconds of pn_step_vjp,
    which runs the forward again itself, else None), CUDA-event timed on the
    launching stream."""
    import torch
    from paper_1801_07986_b300 import pn
    x, v, m = state
    dev = torch.device(f"cuda:{local}")
    X0, V0, M = (torch.tensor(a, device=dev) for a in (x, v, m))
    ctx = pn.pn_init(w.n, G=w.G, c=w.c, eps=w.eps, precision=precision, device=local,
                     stream=stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    XB, VB = torch.empty_like(X0), torch.empty_like(X0)
    # warm-up: allocations of both halves
    X, V, A = X0.clone(), V0.clone(), torch.empty_like(X0)
    pn.pn_accel(ctx, X, V, M, A)
    ck = pn.pn_step_save(ctx, X, V, M, A, w.dt, 2)
    pn.pn_step_vjp_saved(ctx, ck, M, w.dt, 2, X, V, XB, VB)
    del ck
    X, V = X0.clone(), V0.clone()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    pn.pn_accel(ctx, X, V, M, A)
    ckpt = pn.pn_step_save(ctx, X, V, M, A, w.dt, nsteps)
    e1.record(stream)
    e1.synchronize()
    ms_fwd = e0.elapsed_time(e1)
    xbT = torch.zeros_like(X)
    xbT[near] = 2.0 * X[near]
    vbT = torch.zeros_like(X)
    e0.record(stream)
    scal = pn.pn_step_vjp_saved(ctx, ckpt, M, w.dt, nsteps, xbT, vbT, XB, VB)
    e1.record(stream)
    e1.synchronize()
    ms_grad = e0.elapsed_time(e1)
    s_x0 = None
    if from_x0:
        XB2, VB2 = torch.empty_like(X0), torch.empty_like(X0)
        e0.record(stream)
        scal2 = pn.pn_step_vjp(ctx, X0, V0, M, w.dt, nsteps, xbT, vbT, XB2, VB2)
        e1.record(stream)
        e1.synchronize()
        s_x0 = e0.elapsed_time(e1) * 1e-3
        if not (torch.equal(XB, XB2) and torch.equal(VB, VB2) and np.array_equal(scal, scal2)):
            raise RuntimeError("pn_step_vjp and pn_step_vjp_saved differ")
    ctx.close()
    return (XB.cpu().numpy(), VB.cpu().numpy(), float(scal[0, 0]),
            float(-2.0 * scal[0, 1] / w.c ** 3), ms_grad * 1e-3, ms_fwd * 1e-3, s_x0)


def adjoint_fd_check(local, stream, nsteps, grads, near, h=ADJ_FD_H):
    """Gradients of the adjoint workload's loss against FP64 central
    differences.  `grads` maps a name ("mixed", "fp64") to (xbar0, vbar0,
    dL/dM, dL/dc) from pn_step_vjp; the first entry picks the components.
    Checked: dL/dM, dL/dc, and four components each of dL/dx0 and dL/dv0 --
    the two largest of tagged stars (the 16 nearest the hole) and the two
    largest of the untagged stars: a difference over a chaotic 1000-step run
    carries the two perturbed runs' FP64 rounding grown by the dynamics
    (about 3e-3 absolute at h = 1e-8 on this workload), so only components
    well above that are resolved to 1e-6.  Every perturbed trajectory is one cluster of a single
    batched FP64 context (all of them advance in the same launches); dL/dM
    is also differenced at 2h, whose gap to the h difference bounds the
    difference's truncation error.  With two gradient sets each checked
    component also gets their mutual difference."""
    import torch
    from paper_1801_07986_b300 import pn
    from paper_1801_07986_b300.inputs import WORKLOADS
    w = WORKLOADS["plummer8k_adjoint"]
    x, v, m = w.state()
    names = list(grads)
    xb = grads[names[0]][0]
    vb = grads[names[0]][1]
    tagged = set(int(j) for j in near)
    untag = np.array([j for j in range(1, w.n) if j not in tagged])
    tag = np.array(sorted(tagged))
    params = [("M", 0, 0, h), ("M", 0, 0, 2 * h), ("c", 0, 0, ADJ_FD_H_C)]
    for name, g in (("x0", xb), ("v0", vb)):
        for rows in (tag, untag):
            flat = np.abs(g[rows]).ravel()
            for q in np.argsort(flat)[::-1][:2]:
                hq = h if flat[q] >= ADJ_FD_SMALL_G else ADJ_FD_H_SMALL
                params.append((name, int(rows[q // 3]), int(q % 3), hq))
    xs, vs, ms, cs = [], [], [], []
    for name, j, k, hh in params:
        for sgn in (1.0, -1.0):
            xx, vv, mm, cc = x.copy(), v.copy(), m.copy(), w.c
            if name == "M":
                mm[0] += sgn * hh
            elif name == "c":
                cc = w.c * (1.0 + sgn * hh)
            elif name == "x0":
                xx[j, k] += sgn * hh
            else:
                vv[j, k] += sgn * hh
            xs.append(xx), vs.append(vv), ms.append(mm), cs.append(cc)
    nc = len(xs)
    off = np.arange(nc + 1) * w.n
    dev = torch.device(f"cuda:{local}")
    X = torch.tensor(np.concatenate(xs), device=dev)
    V = torch.tensor(np.concatenate(vs), device=dev)
    M = torch.tensor(np.concatenate(ms), device=dev)
    A = torch.empty_like(X)
    ctx = pn.pn_init_batched(off, G=w.G, c=cs, eps=w.eps, precision="fp64", device=local,
                             stream=stream)
    t0 = time.perf_counter()
    pn.pn_accel(ctx, X, V, M, A)
    pn.pn_step(ctx, X, V, M, A, w.dt, nsteps)
    pn.pn_sync(ctx)
    secs = time.perf_counter() - t0
    ctx.close()
    xT = X.cpu().numpy().reshape(nc, w.n, 3)
    L = (xT[:, near, :] ** 2).sum(axis=(1, 2))

    def value(gs, name, j, k):
        if name == "M":
            return gs[2]
        if name == "c":
            return gs[3]
        return (gs[0] if name == "x0" else gs[1])[j, k]

    checks, fdM = [], {}
    for q, (name, j, k, hh) in enumerate(params):
        fd = (L[2 * q] - L[2 * q + 1]) / (2 * hh * (w.c if name == "c" else 1.0))
        if name == "M":
            fdM[hh] = fd
            if hh != h:
                continue
        row = {"param": name if name in ("M", "c") else f"{name}[{j},{k}]",
               "tagged": j in tagged, "h": hh, "central_difference": float(fd)}
        for nm in names:
            g = value(grads[nm], name, j, k)
            row[nm] = float(g)
            row[f"rel_err_{nm}"] = float(abs(g - fd) / abs(fd))
        if len(names) > 1:
            g0, g1 = value(grads[names[0]], name, j, k), value(grads[names[1]], name, j, k)
            row[f"rel_{names[0]}_vs_{names[1]}"] = float(abs(g0 - g1) / abs(g1))
        checks.append(row)
    out = {"steps": nsteps, "h": h, "h_c": ADJ_FD_H_C,
           "h_note": "absolute in M, x0 and v0; relative in c",
           "fd_path": "fp64 (batched context, one cluster per perturbed trajectory)",
           "fd_seconds": secs, "checks": checks,
           "fd_dL_dM_h_vs_2h_rel": float(abs(fdM[h] - fdM[2 * h]) / abs(fdM[h]))}
    for nm in names:
        out[f"max_rel_err_{nm}"] = max(c[f"rel_err_{nm}"] for c in checks)
    if len(names) > 1:
        key = f"rel_{names[0]}_vs_{names[1]}"
        out[f"max_{key}"] = max(c[key] for c in checks)
    return out


def main():
    args = parse()
    from paper_1801_07986_b300.inputs import WORKLOADS
    w = WORKLOADS[args.workload]
    if args.bodies:
        import dataclasses
        w = dataclasses.replace(w, n=args.bodies, name=f"{w.name}@n={args.bodies}")
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_native(args, w)


if __name__ == "__main__":
    main()
