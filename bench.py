#!/usr/bin/env python3
"""Benchmark of the GB300 ADS wildfire time step.

Default workload (one "step" = one Peaceman-Rachford time step of every scenario): the batched
ensemble of 256 scenarios of 256 x 256 elements of quadratic B-splines (258 x 258 = 66,564
DOFs each, 17.04 M in all), each with a seeded mean wind (direction U[0, 2 pi), speed U[0, 3])
and ignition point, sharing one seeded fuel field; FP32 bulk with FP64 1-D factorisations; one
batch handle stepped by the launch form and shapes the autotuner picks (one persistent launch
per step over every slot, or one launch per pass).  The state (five fields per slot, ~380 MB)
is larger than the L2 cache, so no flush is needed between steps.  Each rank of a multi-GPU run
steps its own contiguous share of the scenarios (independent problems, no collective).

The same JSON line carries, as extra keys, the single-instance FP64 path on the 1024^2 domain
(value, ms/step, error against the FP64 oracle on the same steps) and the served request
stream (Poisson arrivals at 0.8 x the measured capacity; p50/p99 latency, aggregate
DOF-steps/s).  --workload c2 / c3 / c5 print those configurations as lines of their own;
--impl reference times the FP64 CPU oracle on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import platform
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ADS DOF-steps/s & HBM roofline frac, FP32 vs FP64 @ rel-L2; serving p50/p99"
UNIT = "DOF-steps/s"
L2_FLUSH_BYTES = 256 << 20
T_AMB = 300.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), sm_max_mhz=float(d.get("sm_max_mhz", 2070.0)), src="measured")
    except Exception:
        return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, src="fallback")


def alu_peak(wf, fp64: bool, sm_count: int, mhz: float):
    """FMA rate of this GPU (TFLOP/s), measured by the library's probe; the derivation if it fails."""
    try:
        v = wf.wf_measure_fma_peak(wf.WF_FP64 if fp64 else wf.WF_FP32)
        return v, ("measured: FMA chains on every SM (wf_measure_fma_peak), "
                   + ("FP64" if fp64 else "FP32, faster of scalar and packed-pair FMAs"))
    except Exception:
        if fp64:
            return 1.25, "nominal FP64 rate (probe failed)"
        return sm_count * 128 * 2 * mhz * 1e6 / 1e12, "derived from SM count and clock (probe failed)"


def algorithmic_costs(p: int, fused_x2: bool = False) -> dict:
    """Algorithmic bytes and flops per DOF of each kernel class of a PR step (FP32 values).

    Flops count fused multiply-adds (2 flops each) of the sum-factorised method, once per DOF:
    the quadrature interpolates T, dT/dx (x) and T, dT/dx, dT/dy (y) from p+1 coefficients,
    2q(p+1) + 3q^2(p+1); the fuel q(p+1) + q^2(p+1); tests them against the basis functions at
    the same cost (the mirror); 6 per Gauss point for the point source; and forms R with two
    Kronecker products, 4W + 1 (W = 2p+1: an x and a y band each, plus the scaled F).  A line
    solve is 4p + 1 per value (p forward, p + 1 backward, 2p spike), + 1 where an increment base
    is added.  Bytes: each field read or written once by its pass.
    """
    q = nb = p + 1
    W = 2 * p + 1
    interp = 2 * q * nb + 3 * q * q * nb
    fuel = q * nb + q * q * nb
    quad = interp + fuel + (interp + fuel) + 6 * q * q + (4 * W + 1)
    line = 4 * p + 1
    mv = 4 * W + 1
    c = {
        "rhs_quadrature_1": dict(bytes=20, flops=2 * quad),          # read T, phi; write F, Phi, R
        "xsolve_1": dict(bytes=16, flops=2 * 2 * line),               # R and Phi in and out
        "ysolve_1": dict(bytes=24, flops=2 * 2 * (line + 1)),         # R, Phi, bases T, phi in; T, phi out
        "matvec_2": dict(bytes=12, flops=2 * mv),                     # T*, F in; R out
        "xsolve_2": (dict(bytes=12, flops=2 * (mv + line)) if fused_x2 else dict(bytes=8, flops=2 * line)),
        "ysolve_2": dict(bytes=12, flops=2 * (line + 1)),             # R, base T* in; T out
    }
    step_flops = c["rhs_quadrature_1"]["flops"] + c["xsolve_1"]["flops"] + c["ysolve_1"]["flops"] + \
        2 * mv + 2 * line + c["ysolve_2"]["flops"]
    # one persistent launch is one whole step: the method's minimum bytes (each pass reads and
    # writes its fields once, the quadrature's R and Phi consumed by the first x pass: 56 B)
    c["step_persistent"] = dict(bytes=56, flops=step_flops)
    return c


def min_step_bytes(scheme: str) -> int:
    """Least HBM bytes per DOF of one step (FP32): fields read and written once per pass.

    PR: x1 reads T, phi and writes its two results and F (20); y1 reads and writes two
    fields (16); x2 reads T*, F and writes its result (12); y2 reads and writes one (8).
    Strang-CN: 16 + 16 (substep 1) + 8 (y substep) + 12 + 8 (substep 3).
    Explicit: x reads T, phi and writes two results (16); y reads them and the bases T, phi
    and writes two fields (24).
    """
    return {"pr": 56, "strang": 60, "explicit": 40}[scheme]


def roofline(kernel: str, ms: float, dofs: int, costs: dict, es: int, hbm_gbs: float, hbm_src: str,
             alu: float, alu_src: str, traffic=None) -> dict:
    """Achieved rate of one kernel against its bound: min(HBM x AI, ALU peak) decides which."""
    c = costs.get(kernel, dict(bytes=0, flops=0))
    b = c["bytes"] * (es / 4) * dofs
    fl = c["flops"] * dofs
    ai = fl / max(b, 1)
    balance = alu * 1e12 / (hbm_gbs * 1e9)
    if ai > balance:
        ach = fl / (ms * 1e-3) / 1e12
        r = {"bound": "alu", "achieved": ach, "peak": alu, "unit": "TFLOP/s", "frac": ach / alu,
             "peak_source": alu_src + " (of measured)"}
    else:
        ach = b / (ms * 1e-3) / 1e9
        r = {"bound": "hbm", "achieved": ach, "peak": hbm_gbs, "unit": "GB/s", "frac": ach / hbm_gbs,
             "peak_source": f"{hbm_src} copy bandwidth (of {hbm_src})"}
    r.update({"kernel": kernel, "ms_per_launch": ms, "algorithmic_bytes_per_launch": b,
              "algorithmic_flops_per_launch": fl, "arithmetic_intensity": ai, "traffic": traffic,
              "hbm_frac_of_algorithmic_bytes": b / (ms * 1e-3) / 1e9 / hbm_gbs,
              "alu_frac_of_algorithmic_flops": fl / (ms * 1e-3) / 1e12 / alu})
    return r


def scheme_of(args) -> str:
    return "strang" if args.strang else ("explicit" if args.explicit else "pr")


def shape_source(args) -> str:
    return "given" if args.tuning else ("rule" if args.no_autotune else "autotuned")


def pick_shapes(wf, h, args, reps: int):
    """Launch shapes: given on the command line, the launchers' rules, or autotuned on the handle."""
    if args.tuning:
        wf.wf_set_tuning(h, [int(v) for v in args.tuning.split(",")])
    elif not args.no_autotune:
        wf.wf_autotune(h, reps)
    return wf.wf_get_tuning(h)


def _source_sha(name: str) -> str:
    import hashlib

    with open(os.path.join(ROOT, "paper_2604_19370_gb300", "csrc", name), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _traffic_record(kernel_site: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        r = rec[workload][kernel_site]
        if any(r["source_sha"].get(s) != _source_sha(s) for s in r["source_sha"]):
            return None
        return float(r["dram_bytes_per_launch"])
    except Exception:
        return None


def soak(run_chunk, seconds: float) -> int:
    """Untimed steps for about `seconds` just before the timed region.

    nvidia-smi samples every 200 ms, so a timed region of a few milliseconds holds one sample at
    most; the sampler runs over this soak and the timed region together, with the GPU under the
    same load throughout.  run_chunk() enqueues some steps and waits for them; returns the calls.
    """
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < seconds:
        run_chunk()
        n += 1
    return n


class ClockSampler:
    """nvidia-smi clock and throttle sampling over the soak and the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self) -> dict:
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "samples": len(sm), "reasons": sorted(reasons),
                "window": "soak steps of the same workload, then the timed region"}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(x: float, device=None) -> float:
    """Maximum of x over all ranks (x itself without a process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_throughput(units_per_rank: float, local_seconds: float, world: int, device=None):
    """Units all ranks processed / the slowest rank's time (weak scaling: fixed units per rank)."""
    slowest = reduce_max(local_seconds, device)
    return world * units_per_rank / slowest, slowest


def shard(n_items: int, rank: int, world: int):
    """Contiguous share of n_items for one rank (independent scenarios; no exchange between ranks)."""
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def cpu_info() -> dict:
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


# ---- the FP64 CPU oracle (test infrastructure; timed here as the baseline) ------------------

def _oracle_worker(job):
    """One process: the oracle (ads mode) on one scenario; returns wall-clock marks and the state."""
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    sys.path.insert(0, ROOT)
    from oracle.step import Problem
    from scenarios import config_c2, config_c4

    kind, idx, warm, steps, scheme, keep = job
    if kind == "c4":
        shared = config_c4(0).fuel0
        sc = config_c4(idx, shared_fuel=shared)
    else:
        sc = config_c2()
    P = Problem.from_scenario(sc, scheme=scheme, mode="ads")
    T, phi = sc.T0.copy(), sc.fuel0.copy()
    for _ in range(warm):
        T, phi = P.step(T, phi)
    t0 = time.time()
    for _ in range(steps):
        T, phi = P.step(T, phi)
    t1 = time.time()
    return dict(t0=t0, t1=t1, dofs=sc.dofs, steps=steps, T=T if keep else None, phi=phi if keep else None)


def oracle_runs(jobs, procs: int):
    """Run oracle jobs in a pool of `procs` fresh processes (spawned: no GPU state is inherited)."""
    ctx = mp.get_context("spawn")
    env_save = {k: os.environ.get(k) for k in ("CUDA_VISIBLE_DEVICES",)}
    os.environ["CUDA_VISIBLE_DEVICES"] = ""
    try:
        with ctx.Pool(procs) as pool:
            return pool.map(_oracle_worker, jobs)
    finally:
        for k, v in env_save.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def oracle_throughput(results) -> float:
    start = min(r["t0"] for r in results)
    end = max(r["t1"] for r in results)
    return sum(r["dofs"] * r["steps"] for r in results) / (end - start)


def errors_vs_oracle(T, phi, To, po) -> dict:
    import numpy as np

    return {"T": float(np.linalg.norm(T - To) / np.linalg.norm(To)),
            "T_minus_Tamb": float(np.linalg.norm(T - To) / np.linalg.norm(To - T_AMB)),
            "max_abs_T_over_max_T_minus_Tamb": float(np.abs(T - To).max() / np.abs(To - T_AMB).max()),
            "phi": float(np.linalg.norm(phi - po) / np.linalg.norm(po)),
            "max_abs_phi": float(np.abs(phi - po).max())}


# ---- the reference arm -----------------------------------------------------------------------

def run_reference(args) -> None:
    """The FP64 CPU oracle on the machine's host cores, on a bounded sample of the default workload.

    One step of this arm is one PR step of as many ensemble scenarios as there are cores (one
    per process); W warm-up steps are run first and exactly K steps are timed.
    """
    world, rank, _ = _dist()
    if rank != 0:
        return
    procs = os.cpu_count() or 1
    res = oracle_runs([("c4", k, args.warmup, args.steps, "pr", False) for k in range(procs)], procs)
    value = oracle_throughput(res)
    wall = max(r["t1"] for r in res) - min(r["t0"] for r in res)
    dofs = res[0]["dofs"]
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": wall * 1e3 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "c4_ensemble_256x256x256_p2_pr", "nx": 256, "ny": 256, "p": 2,
                   "scenarios_sampled": procs, "dofs_per_scenario": dofs, "scheme": "PR",
                   "impl": "FP64 CPU oracle, ads mode (1-D banded solves), one scenario per process"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                         "sample": f"{args.steps} timed PR steps (after {args.warmup}) of {procs} scenarios of the "
                                   "256-scenario ensemble, one per process", **cpu_info()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---- GPU workloads ---------------------------------------------------------------------------

def _setup_gpu():
    import torch

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2604_19370_gb300.build import build_library

    build_library()
    from paper_2604_19370_gb300 import wf

    return wf, dev, world, rank, local


def _kernel_table(kt: dict) -> dict:
    shares = {k: v[0] for k, v in kt.items() if v[1] > 0}
    tot = sum(shares.values()) or 1.0
    return {k: {"ms_per_launch": v[0] / v[1], "launches": v[1], "share": v[0] / tot} for k, v in kt.items() if v[1] > 0}


def run_ensemble(args) -> None:
    """Batched ensemble: S scenarios of 256^2 elements (p = 2) in one batch handle."""
    import numpy as np
    import torch

    wf, dev, world, rank, local = _setup_gpu()
    from scenarios import config_c4

    S_all = args.scenarios
    mine = list(shard(S_all, rank, world))
    first = config_c4(0)
    shared = first.fuel0
    scs = [config_c4(k, shared_fuel=shared) for k in mine]
    S = len(scs)
    prm = wf.wf_params_default(Lx=first.Lx, Ly=first.Ly, precision=wf.WF_FP32)
    b = wf.Batch(first.nx, first.ny, first.p, first.dt, prm, capacity=S)
    for k, sc in enumerate(scs):
        b.load_scenario(k, sc)
    stream = torch.cuda.Stream(device=dev)
    wf.wf_set_stream(b.h, stream.cuda_stream)
    tuning = pick_shapes(wf, b.h, args, 12)
    dofs = S * first.dofs
    with torch.cuda.stream(stream):
        b.step(args.warmup)
    stream.synchronize()
    if wf.wf_sync(b.h) != wf.WF_OK:
        raise RuntimeError("ensemble unstable or timed out during warm-up")

    def timed(profile):
        wf.wf_set_profiling(b.h, profile)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(stream):
            e0.record(stream)
            wf.wf_step(b.h, args.steps)  # K steps in one call (step graphs of eight and one)
            e1.record(stream)
        stream.synchronize()
        torch.cuda.synchronize(dev)
        wf.wf_set_profiling(b.h, False)
        return e0.elapsed_time(e1) * 1e-3

    def chunk():
        with torch.cuda.stream(stream):
            b.step(64)
        stream.synchronize()

    # timed region: K steps replayed from the step graph (the production launch path); the soak
    # runs first under the clock sampler, then the initial states are put back and warmed up again
    with ClockSampler(local) as clk:
        soak(chunk, args.clock_soak)
        for k, sc in enumerate(scs):
            b.load_scenario(k, sc)
        with torch.cuda.stream(stream):
            b.step(args.warmup)
        stream.synchronize()
        secs = timed(False)
    status = wf.wf_sync(b.h)
    value, slowest = whole_job_throughput(dofs * args.steps, secs, world, dev)
    ms_per_step = slowest * 1e3 / args.steps
    # per-kernel device times: the same K steps launched directly, an event pair around each launch
    wf.wf_kernel_times(b.h)
    n0 = wf.wf_launch_count()
    prof_s = timed(True)
    launches = wf.wf_launch_count() - n0
    kt = wf.wf_kernel_times(b.h)
    peaks = _peaks()
    props = torch.cuda.get_device_properties(dev)
    alu, alu_src = alu_peak(wf, False, props.multi_processor_count, peaks["sm_max_mhz"])
    costs = algorithmic_costs(first.p, fused_x2=tuning[5] != 2)
    ktab = _kernel_table(kt)
    dom = max(ktab, key=lambda k: ktab[k]["share"])
    workload = f"c4_ensemble_{S_all}x256x256_p2_pr"
    roof = roofline(dom, ktab[dom]["ms_per_launch"], dofs, costs, 4, peaks["hbm_gbs"], peaks["src"], alu, alu_src,
                    _traffic_record(dom, "c4_ensemble_256x256x256_p2_pr") if S_all == 256 else None)
    step_flops = costs["step_persistent"]["flops"] * dofs
    # the other step forms, timed the same way with the same shapes (the autotuner times every form
    # and keeps the fastest): per-pass launches; one quadrature launch and one persistent launch over
    # every line pass of every slot; the per-pass launches over two slot groups on two streams
    forms = {1: "per-pass launches", 2: "persistent line passes",
             3: "per-pass launches, two slot groups overlapped on two streams"}
    chosen = tuning[6] if tuning[6] else 1
    other_forms = {}
    for form in (1, 2, 3):
        if form == chosen:
            continue
        other = list(tuning)
        other[6] = form
        wf.wf_set_tuning(b.h, other)
        with torch.cuda.stream(stream):
            b.step(3)
        stream.synchronize()
        other_s = timed(False)
        wf.wf_kernel_times(b.h)
        n1 = wf.wf_launch_count()
        timed(True)
        other_launches = wf.wf_launch_count() - n1
        other_kt = _kernel_table(wf.wf_kernel_times(b.h))
        other_forms[forms[form]] = {"ms_per_step": other_s * 1e3 / args.steps, "value": dofs * args.steps / other_s,
                                    "launches_per_step": other_launches / args.steps, "kernels": other_kt}
    wf.wf_set_tuning(b.h, tuning)
    # end to end through the C ABI: pinned float32 host arrays holding every slot's state
    n = first.dofs
    hT = torch.empty(S * n, dtype=torch.float32, pin_memory=True)
    hP = torch.empty(S * n, dtype=torch.float32, pin_memory=True)
    for k, sc in enumerate(scs):
        hT.numpy()[k * n:(k + 1) * n] = sc.T0.ravel()
        hP.numpy()[k * n:(k + 1) * n] = sc.fuel0.ravel()
    # one call per step: every slot's state from the pinned arrays, one step, every state back
    # (wf_batch_run_f32: the slots in groups whose copies overlap the other groups' steps); the
    # group count is chosen from 1, 2, 4 and 8 by a short trial
    e2e_steps = 5
    e2e_try = {}
    for groups in (1, 2, 4, 8):
        wf.wf_batch_run_ptr(b.h, hT.data_ptr(), hP.data_ptr(), hT.data_ptr(), hP.data_ptr(), S * n, 1, groups, True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(2):
            wf.wf_batch_run_ptr(b.h, hT.data_ptr(), hP.data_ptr(), hT.data_ptr(), hP.data_ptr(), S * n, 1, groups,
                                True)
        e2e_try[groups] = (time.perf_counter() - t0) / 2
    e2e_groups = min(e2e_try, key=e2e_try.get)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        wf.wf_batch_run_ptr(b.h, hT.data_ptr(), hP.data_ptr(), hT.data_ptr(), hP.data_ptr(), S * n, 1, e2e_groups,
                            True)
    e2e_s = reduce_max((time.perf_counter() - t0) / e2e_steps, dev)
    b.close()
    # the host link's own rates, on the same pinned arrays (their contents are no longer needed)
    link = link_bound(wf.wf_measure_host_link_ptr(hT.data_ptr(), hP.data_ptr(), hT.numel() * 4), 2 * 4 * dofs,
                      2 * 4 * dofs, e2e_s * 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "scenarios": S_all, "scenarios_per_rank": S, "nx": 256, "ny": 256,
                   "p": 2, "dofs": S_all * first.dofs, "scheme": "PR",
                   "precision": "fp32 bulk, fp64 1-D factorisation",
                   "l2": f"state of {S} slots x 5 fields (~{5 * S * 258 * 288 * 4 / 2**20:.0f} MiB) > L2, no flush",
                   "parallelism": f"scenarios sharded over {world} rank(s), no collective",
                   "launch_shapes": {**{k: v for k, v in zip(wf.TUNING_NAMES, tuning)}, "source": shape_source(args)}},
        "roofline": roof,
        "step_roofline": {"hbm_frac_of_min_bytes": min_step_bytes("pr") * dofs / (ms_per_step * 1e-3) / 1e9
                          / peaks["hbm_gbs"],
                          "alu_frac": step_flops / (ms_per_step * 1e-3) / 1e12 / alu,
                          "min_bytes_per_dof": min_step_bytes("pr"),
                          "flops_per_dof": costs["step_persistent"]["flops"]},
        "profiled_ms_per_step": prof_s * 1e3 / args.steps,
        "kernels": ktab,
        # the profiled pass launches each kernel once per step over all slots; step form 3 launches
        # every kernel once per slot group
        "gpu_launches": launches * (2 if chosen == 3 and S >= 2 else 1),
        "step_form": forms[chosen],
        "other_step_forms": other_forms,
        "e2e": {"value": world * dofs / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 2 * 4 * dofs,
                "d2h_bytes_per_step": 2 * 4 * dofs, "ms_per_step": e2e_s * 1e3, "host_dtype": "float32",
                "call": "wf_batch_run_f32 (states in, one step, states out)", "groups": e2e_groups,
                "trial_ms_per_step": {str(g): round(t * 1e3, 4) for g, t in e2e_try.items()},
                "host_link": link},
        "clocks": clk.summary(),
        "status": wf.wf_strerror(status),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle: one core on scenario 0 (its state also checks this path), then every core on
        # as many scenarios at once
        ks = args.cpu_steps
        procs = os.cpu_count() or 1
        one = oracle_runs([("c4", 0, 0, ks, "pr", True)], 1)[0]
        allc = oracle_runs([("c4", k, 0, ks, "pr", False) for k in range(procs)], procs)
        chk = wf.simulation_from_scenario(scs[0], precision=wf.WF_FP32)
        wf.wf_set_tuning(chk.h, tuning)
        chk.step(ks)
        Tg, pg = chk.state()
        chk.close()
        line["cpu_baseline"] = {"value": oracle_throughput(allc), "unit": UNIT, "cores": procs, "kind": "oracle",
                                "sample": f"{ks} PR steps of each of {procs} ensemble scenarios, one per process "
                                          "(FP64, ads mode)",
                                "single_core_value": oracle_throughput([one]),
                                "single_core_sample": f"{ks} PR steps of scenario 0", **cpu_info()}
        line["rel_l2_vs_oracle"] = {"steps": ks, "scenario": 0, **errors_vs_oracle(Tg, pg, one["T"], one["phi"])}
    if rank == 0 and world == 1 and not args.no_extras:
        line["fp64_single_instance"] = fp64_c2_extra(wf, dev, args)
        line["serving"] = run_serving(args, wf=wf, as_extra=True)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def fp64_c2_extra(wf, dev, args) -> dict:
    """The single-instance FP64 path on the 1024^2 domain: device throughput and oracle error."""
    import torch

    from scenarios import config_c2

    sc = config_c2()
    sim = wf.simulation_from_scenario(sc, precision=wf.WF_FP64)
    stream = torch.cuda.Stream(device=dev)
    wf.wf_set_stream(sim.h, stream.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        sim.step(3)
    stream.synchronize()
    K = 10
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with torch.cuda.stream(stream):
        for k in range(K):
            flush.zero_()
            ev[k][0].record(stream)
            wf.wf_step(sim.h, 1)
            ev[k][1].record(stream)
    stream.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / K
    st = sim.sync()
    # end to end through the FP64 host boundary: state from pinned float64 arrays, one step, state back
    n = sc.dofs
    hT = torch.empty(n, dtype=torch.float64, pin_memory=True)
    hP = torch.empty(n, dtype=torch.float64, pin_memory=True)
    hT.numpy()[:] = sc.T0.ravel()
    hP.numpy()[:] = sc.fuel0.ravel()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(K):
        wf.wf_set_state_ptr(sim.h, hT.data_ptr(), hP.data_ptr(), n)
        wf.wf_step(sim.h, 1)
        wf.wf_get_state_ptr(sim.h, hT.data_ptr(), hP.data_ptr(), n)
    e2e_s = (time.perf_counter() - t0) / K
    sim.close()
    out = {"workload": "c2_1024x1024_p2_pr_fp64", "value": sc.dofs / (ms * 1e-3), "unit": UNIT,
           "ms_per_step": ms, "steps": K, "l2": "flushed before every timed step (256 MiB write)",
           "status": wf.wf_strerror(st),
           "e2e": {"value": n / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 16 * n, "d2h_bytes_per_step": 16 * n,
                   "ms_per_step": e2e_s * 1e3, "host_dtype": "float64"}}
    if not args.no_cpu_baseline:
        ks = 2
        o = oracle_runs([("c2", 0, 0, ks, "pr", True)], 1)[0]
        chk = wf.simulation_from_scenario(sc, precision=wf.WF_FP64)
        chk.step(ks)
        Tg, pg = chk.state()
        chk.close()
        out["rel_l2_vs_oracle"] = {"steps": ks, **errors_vs_oracle(Tg, pg, o["T"], o["phi"])}
    return out


def run_single(args) -> None:
    """One domain: c2 (1024^2, p = 2) or c3 (4096^2, p = 3, two fuel classes, gaps, three ignitions)."""
    import torch

    wf, dev, world, rank, local = _setup_gpu()
    from scenarios import config_c2, config_c3

    sc = config_c3() if args.workload == "c3" else config_c2(p=args.p)
    prec = wf.WF_FP64 if args.fp64 else wf.WF_FP32
    scheme = {"pr": wf.WF_PR, "strang": wf.WF_STRANG_CN, "explicit": wf.WF_EXPLICIT}[scheme_of(args)]
    sim = wf.simulation_from_scenario(sc, precision=prec, scheme=scheme)
    stream = torch.cuda.Stream(device=dev)
    wf.wf_set_stream(sim.h, stream.cuda_stream)
    tuning = pick_shapes(wf, sim.h, args, 40 if args.workload == "c2" else 6)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        sim.step(args.warmup)
    stream.synchronize()
    if sim.sync() != wf.WF_OK:
        raise RuntimeError("unstable during warm-up")

    def run_steps(profile: bool):
        """K steps, L2 flushed before each, CUDA events around each step on the launching stream."""
        wf.wf_set_profiling(sim.h, profile)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.zero_()
                ev[k][0].record(stream)
                wf.wf_step(sim.h, 1)
                ev[k][1].record(stream)
        stream.synchronize()
        torch.cuda.synchronize(dev)
        wf.wf_set_profiling(sim.h, False)
        return float(sum(a.elapsed_time(b) for a, b in ev))

    # the soak steps a twin of the domain (same shapes), so the timed one keeps its state and status
    twin = wf.simulation_from_scenario(sc, precision=prec, scheme=scheme)
    wf.wf_set_stream(twin.h, stream.cuda_stream)
    wf.wf_set_tuning(twin.h, tuning)

    def chunk():
        with torch.cuda.stream(stream):
            for _ in range(16):
                flush.zero_()
                wf.wf_step(twin.h, 1)
        stream.synchronize()

    with ClockSampler(local) as clk:
        soak(chunk, args.clock_soak)
        ms_total = run_steps(False)
    twin.close()
    status = sim.sync()
    value, slowest_s = whole_job_throughput(sc.dofs * args.steps, ms_total * 1e-3, world, dev)
    ms_per_step = slowest_s * 1e3 / args.steps
    wf.wf_kernel_times(sim.h)
    n0 = wf.wf_launch_count()
    prof_ms_per_step = run_steps(True) / args.steps
    launches = wf.wf_launch_count() - n0
    kt = wf.wf_kernel_times(sim.h)
    # end to end through the C ABI with pinned host buffers in the working precision
    n = sc.dofs
    hdt = torch.float64 if args.fp64 else torch.float32
    es = 8 if args.fp64 else 4
    hT = torch.empty(n, dtype=hdt, pin_memory=True)
    hP = torch.empty(n, dtype=hdt, pin_memory=True)
    hT.numpy()[:] = sc.T0.ravel()
    hP.numpy()[:] = sc.fuel0.ravel()
    set_ptr = wf.wf_set_state_ptr if args.fp64 else wf.wf_set_state_f32_ptr
    get_ptr = wf.wf_get_state_ptr if args.fp64 else wf.wf_get_state_f32_ptr
    e2e_steps = max(3, min(args.steps, 20))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        set_ptr(sim.h, hT.data_ptr(), hP.data_ptr(), n)
        wf.wf_step(sim.h, 1)
        get_ptr(sim.h, hT.data_ptr(), hP.data_ptr(), n)
    e2e_s = reduce_max((time.perf_counter() - t0) / e2e_steps, dev)
    peaks = _peaks()
    props = torch.cuda.get_device_properties(dev)
    alu, alu_src = alu_peak(wf, args.fp64, props.multi_processor_count, peaks["sm_max_mhz"])
    costs = algorithmic_costs(sc.p, fused_x2=tuning[5] != 2 and scheme_of(args) == "pr")
    if scheme_of(args) == "explicit":
        costs["rhs_quadrature_1"]["bytes"] = 16  # no F stored
        costs["ysolve_2"]["bytes"] = 24  # two arrays with their bases
    ktab = _kernel_table(kt)
    dom = max(ktab, key=lambda k: ktab[k]["share"])
    wname = f"{args.workload}_{sc.nx}x{sc.ny}_p{sc.p}_{scheme_of(args)}"
    roof = roofline(dom, ktab[dom]["ms_per_launch"], sc.dofs, costs, es, peaks["hbm_gbs"], peaks["src"], alu, alu_src,
                    _traffic_record(dom, wname) if not args.fp64 else None)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.fp64 else "f32", "data": "synthetic",
        "config": {"workload": wname, "nx": sc.nx, "ny": sc.ny, "p": sc.p, "dofs": sc.dofs,
                   "scheme": {"pr": "PR", "strang": "Strang-CN", "explicit": "explicit L2 projection"}[scheme_of(args)],
                   "precision": "fp64" if args.fp64 else "fp32 bulk, fp64 1-D factorisation",
                   "l2": "flushed before every timed step (256 MiB write)",
                   "launch_shapes": {**{k: v for k, v in zip(wf.TUNING_NAMES, tuning)}, "source": shape_source(args)},
                   "parallelism": f"replicas x{world}"},
        "roofline": roof,
        "step_hbm_frac": min_step_bytes(scheme_of(args)) * (es / 4) * sc.dofs / (ms_per_step * 1e-3) / 1e9
        / peaks["hbm_gbs"],
        "profiled_ms_per_step": prof_ms_per_step,
        "kernels": ktab,
        "gpu_launches": launches,
        "e2e": {"value": world * sc.dofs / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 2 * es * n,
                "d2h_bytes_per_step": 2 * es * n, "ms_per_step": e2e_s * 1e3,
                "host_dtype": "float64" if args.fp64 else "float32"},
        "clocks": clk.summary(),
        "status": wf.wf_strerror(status),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "c2":
        ks = args.cpu_steps
        o = oracle_runs([("c2", 0, 0, ks, scheme_of(args), True)], 1)[0]
        chk = wf.simulation_from_scenario(sc, precision=prec, scheme=scheme)
        chk.step(ks)
        Tg, pg = chk.state()
        chk.close()
        line["cpu_baseline"] = {"value": oracle_throughput([o]), "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{ks} {scheme_of(args)} steps of the same 1026^2-DOF workload, FP64, "
                                          "ads mode (one domain: one core)", **cpu_info()}
        line["rel_l2_vs_oracle"] = {"steps": ks, **errors_vs_oracle(Tg, pg, o["T"], o["phi"])}
    sim.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def link_bound(rates, bytes_in: int, bytes_out: int, e2e_ms: float) -> dict:
    """The host-link bound of an end-to-end step: its copies at the measured rates.

    rates = (host to device, device to host, both directions at once) in GB/s.  The step needs at
    least as long as either direction alone and as both directions' bytes at the combined rate.
    """
    h2d, d2h, both = rates
    bound_ms = max(bytes_in / h2d, bytes_out / d2h, (bytes_in + bytes_out) / both) / 1e6
    return {"h2d_gbs": h2d, "d2h_gbs": d2h, "both_gbs": both, "bound_ms_per_step": bound_ms,
            "frac": bound_ms / e2e_ms,
            "source": "measured: wf_measure_host_link (cudaMemcpyAsync between pinned host arrays and the "
                      "device, each direction alone and both at once, best of three)"}


def _percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q
    f = int(math.floor(k))
    c = min(f + 1, len(xs) - 1)
    return xs[f] + (xs[c] - xs[f]) * (k - f)


def run_serving(args, wf=None, as_extra: bool = False):
    """Served request stream: Poisson arrivals at 80 % of measured capacity, p50/p99 latency."""
    import torch

    world, rank, local = _dist()
    if rank != 0:
        return None
    if wf is None:
        wf, _, world, rank, local = _setup_gpu()
    from scenarios import make_scenario, request_stream_c5

    free, _total = torch.cuda.mem_get_info()
    budget = int(0.8 * free)

    def scenario(r):
        return make_scenario(f"q{r['seed']}", r["n"], r["p"], 1e-3, r["steps"], r["seed"], fuel_sigma=20.0,
                             wind_speed_range=(0.0, 3.0))

    def run(reqs, rate):
        srv = wf.Server(budget, max_slots=args.max_slots)
        prepared = [(scenario(r), r) for r in reqs]
        tickets, lat, dof_steps, fails = {}, [], 0.0, {}
        t_start = time.perf_counter()
        pending = list(prepared)
        while pending or tickets:
            now = time.perf_counter() - t_start
            while pending and (rate is None or pending[0][1]["arrival_s"] <= now):
                sc, r = pending.pop(0)
                prec = wf.WF_FP64 if r["fp64"] else wf.WF_FP32
                tickets[srv.submit(sc, precision=prec)] = sc
            for t in list(tickets):
                out = srv.poll(t)
                if out is not None:
                    sc = tickets.pop(t)
                    if out[0] == wf.WF_OK:
                        lat.append(out[1].latency_s)
                        dof_steps += sc.dofs * sc.steps
                    else:
                        fails[wf.wf_strerror(out[0])] = fails.get(wf.wf_strerror(out[0]), 0) + 1
            time.sleep(0.0005)
        makespan = time.perf_counter() - t_start
        srv.close()
        return lat, dof_steps, makespan, fails

    warm = request_stream_c5(4, 1.0, seed=55)
    run(warm, None)
    closed = request_stream_c5(args.requests, 1.0, seed=5)
    lat_c, ds_c, span_c, _ = run(closed, None)
    capacity = len(lat_c) / span_c
    rate = 0.8 * capacity
    # the same requests (sizes, orders, step counts, precisions, seeds) with Poisson arrival times at
    # the rate: the capacity was measured on exactly this work
    open_reqs = request_stream_c5(args.requests, rate, seed=5)
    lat, ds, span, fails = run(open_reqs, rate)
    res = {"workload": "c5_served_poisson", "requests": len(open_reqs), "arrival_rate_hz": rate,
           "capacity_rps": capacity, "sizes": [128, 256, 512, 1024], "p": [2, 3], "steps": "U[200,2000]",
           "fp64_share": 0.2, "hbm_budget_bytes": budget, "max_slots_per_class": args.max_slots,
           "latency_p50_s": _percentile(lat, 0.5), "latency_p99_s": _percentile(lat, 0.99),
           "completed": len(lat), "failed": sum(fails.values()), "failures": fails, "value": ds / span, "unit": UNIT,
           "closed_loop_dof_steps_per_s": ds_c / span_c}
    if as_extra:
        return res
    line = {
        "metric": METRIC, "value": ds / span, "unit": UNIT, "n_gpus": 1, "steps": len(open_reqs),
        "warmup": len(warm), "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (20% of requests f64)", "data": "synthetic",
        "config": {k: v for k, v in res.items() if k not in ("value", "unit", "latency_p50_s", "latency_p99_s",
                                                              "completed", "failed", "closed_loop_dof_steps_per_s")},
        "latency_p50_s": res["latency_p50_s"], "latency_p99_s": res["latency_p99_s"],
        "completed": res["completed"], "failed": res["failed"], "failures": fails,
        "closed_loop_dof_steps_per_s": res["closed_loop_dof_steps_per_s"],
    }
    print(json.dumps(line), flush=True)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c4", choices=["c2", "c3", "c4", "c5"],
                    help="c4: batched 256-scenario ensemble (default); c2: one 1024^2 domain; c3: one 4096^2 cubic "
                         "domain; c5: served request stream")
    ap.add_argument("--p", type=int, default=2)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--strang", action="store_true")
    ap.add_argument("--explicit", action="store_true", help="explicit L2-projection scheme (the comparator)")
    ap.add_argument("--cpu-steps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="c4 line without the FP64 and serving extra keys")
    ap.add_argument("--no-autotune", action="store_true", help="launch shapes from the launchers' rules")
    ap.add_argument("--tuning", default="", help="the eight tuning values of wf_set_tuning (skips the autotuner)")
    ap.add_argument("--scenarios", type=int, default=256)
    ap.add_argument("--requests", type=int, default=100)
    ap.add_argument("--max-slots", type=int, default=16)
    ap.add_argument("--clock-soak", type=float, default=1.0,
                    help="seconds of untimed steps sampled with the timed region by the clock sampler")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "c4":
        run_ensemble(args)
    elif args.workload == "c5":
        run_serving(args)
    else:
        run_single(args)


if __name__ == "__main__":
    main()
