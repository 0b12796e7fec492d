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
FLOPS_PACKED = 72  # hand count of the packed fused pair body, law-of-cosines form (r_near > 0)
OPS_PACKED = 46    # FP32-pipe operations per pair of that body (FMA, add and mul count 1 each)
FLOPS_PACKED_FAR = 66  # the same body on far units of the spatial order (x_ij from the high parts)
OPS_PACKED_FAR = 40
FLOPS_JERK = 213   # hand count of the dual-number pair body of the jerk
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
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=1000)
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
    rows = 16
    for _ in range(args.warmup):
        oracle_rate(x, v, m, w, rows, rows, seed=1)
    rates, secs = [], 0.0
    for k in range(steps):
        r, t, cores = oracle_rate(x, v, m, w, rows, rows, seed=100 + k)
        rates.append(r)
        secs += t
    value = len(rates) / sum(1.0 / r for r in rates)
    sample = (f"each step: {rows} star rows + {rows} hole double-sum rows of the N={w.n} "
              f"evaluation, scaled by (N-1)/rows")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "interactions/s",
        "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * w.n * (w.n - 1) / value, "higher_is_better": True,
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


def profiled_traffic(kernel_tag: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None
    src = kernel_source_hash(kernel_tag)
    for f in sorted(os.listdir(d)):
        if not f.endswith(".md"):
            continue
        txt = open(os.path.join(d, f)).read()
        m1 = re.search(rf"traffic_bytes_per_launch\[{kernel_tag}\]:\s*([0-9.eE+]+)", txt)
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
    if fused:
        tag = "fused_packed" if launch.get("packed") else "fused_mixed"
    elif f64_fused:
        tag = "fused_f64"
    else:
        tag = f"pass{k_dom + 1}_{args.precision}"
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": profiled_traffic(tag), "kernel": tag,
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
        line["e2e"] = {"value": float(w.n) * (w.n - 1) * e2e_steps / (tot * 1e-3),
                       "unit": "interactions/s", "h2d_bytes_per_step": 80 * w.n,
                       "d2h_bytes_per_step": 72 * w.n, "steps": e2e_steps,
                       "device_value_same_steps": float(w.n) * (w.n - 1) * e2e_steps
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

    if not args.no_adjoint and world == 1:
        try:
            line["adjoint"] = run_adjoint(local, stream, args.adjoint_steps)
        except Exception as e:  # reported, not required
            line["adjoint"] = {"error": str(e)[:300]}

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
    Hermite step (two A + two jerk evaluations)."""
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
    e0.record(stream)
    pn.pn_step(ctx, X, V, M, A, w.dt, 2)
    e1.record(stream)
    e1.synchronize()
    pn.pn_sync(ctx)
    ms_step = e0.elapsed_time(e1) / 2
    ctx.close()
    pairs = float(w.n - 1) * (w.n - 2)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2032.0))
    peak = 148 * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = FLOPS_JERK * pairs / (ms_jerk * 1e-3) / 1e12
    return {"workload": "plummer16k", "n_bodies": w.n,
            "value": float(w.n) * (w.n - 1) / (ms_jerk * 1e-3), "unit": "interactions/s",
            "what": "pn_jerk in a mixed context: A + dual-number jerk (FP32 pair sums), "
                    "per evaluation",
            "ms_per_jerk": ms_jerk, "hermite_ms_per_step": ms_step,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "peak_basis": f"148 SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                                       f"{sm_max:.0f} MHz",
                         "flops_per_pair": FLOPS_JERK,
                         "note": "whole pn_jerk call timed (A + the dual pair kernel)"}}


def run_adjoint(local, stream, nsteps):
    """The adjoint workload: N = 8192 Plummer cluster (M = 0.1, c = 50,
    dt = 1/2048), loss = sum over the 16 stars nearest the hole at t = 0 of
    |x(T)|^2 after nsteps KDK steps (mixed-precision forward, FP64
    derivatives), gradient with respect to M, c, x0 and v0 through
    pn_step_vjp with sqrt(T) checkpoints; timed with CUDA events."""
    import torch
    from paper_1801_07986_b300 import pn
    from paper_1801_07986_b300.inputs import WORKLOADS
    w = WORKLOADS["plummer8k_adjoint"]
    x, v, m = w.state()
    near = np.argsort(np.linalg.norm(x[1:] - x[0], axis=1))[:16] + 1
    dev = torch.device(f"cuda:{local}")
    X0, V0, M = (torch.tensor(a, device=dev) for a in (x, v, m))
    ctx = pn.pn_init(w.n, G=w.G, c=w.c, eps=w.eps, precision="mixed", device=local,
                     stream=stream)
    X, V = X0.clone(), V0.clone()
    A = torch.empty_like(X)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    pn.pn_accel(ctx, X, V, M, A)
    pn.pn_step(ctx, X, V, M, A, w.dt, nsteps)
    e1.record(stream)
    e1.synchronize()
    ms_fwd = e0.elapsed_time(e1)
    xbT = torch.zeros_like(X)
    xbT[near] = 2.0 * X[near]
    vbT = torch.zeros_like(X)
    XB, VB = torch.empty_like(X), torch.empty_like(X)
    pn.pn_step_vjp(ctx, X0, V0, M, w.dt, 2, xbT, vbT, XB, VB)       # allocations, warm-up
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e0.record(stream)
    scal = pn.pn_step_vjp(ctx, X0, V0, M, w.dt, nsteps, xbT, vbT, XB, VB)
    e1.record(stream)
    e1.synchronize()
    wall = time.perf_counter() - t0
    ms_grad = e0.elapsed_time(e1)
    ctx.close()
    pairs = float(w.n) * (w.n - 1) * nsteps
    return {"workload": "plummer8k_adjoint", "n_bodies": w.n, "steps": nsteps,
            "checkpoint": "every ceil(sqrt(steps)) steps",
            "loss": "sum over the 16 stars nearest the hole at t=0 of |x(T)|^2",
            "value": pairs / (ms_grad * 1e-3), "unit": "interactions/s",
            "what": "trajectory steps differentiated per second x N(N-1)",
            "gradient_s": ms_grad * 1e-3, "gradient_wall_s": wall,
            "forward_s": ms_fwd * 1e-3, "gradient_over_forward": ms_grad / ms_fwd,
            "dL_dM": float(scal[0, 0]), "dL_dc": float(-2.0 * scal[0, 1] / w.c ** 3),
            "grad_x0_norm": float(torch.linalg.norm(XB)), "grad_v0_norm": float(torch.linalg.norm(VB))}


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
