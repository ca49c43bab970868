#!/usr/bin/env python3
"""Benchmark of the GB300 ADS wildfire time step.

Workload (one time step = one "step"): 1024 x 1024 elements, quadratic
B-splines (1026 x 1026 = 1,052,676 DOFs), Peaceman-Rachford, FP32 bulk with
FP64 1-D factorisations, seeded synthetic terrain (fuel smoothed over 20
elements, wind speed U[0,3] in a random direction plus a 10 % smooth
variation).  The state is resident on the GPU; the L2 cache is flushed (a
256 MiB write) before every timed step, so every step reads its inputs from
HBM.  Each rank runs its own replica: one domain's x and y passes each need
whole lines, so the single domain is not split across GPUs.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ADS DOF-steps/s & HBM roofline frac, FP32 vs FP64 @ rel-L2; serving p50/p99"
UNIT = "DOF-steps/s"
L2_FLUSH_BYTES = 256 << 20
FP64_NOMINAL_TFLOPS = 1.25


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), sm_max_mhz=float(d.get("sm_max_mhz", 2070.0)), src="measured")
    except Exception:
        return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, src="fallback")


def fp32_alu_peak_tflops(sm_count: int, mhz: float) -> float:
    # 128 FP32 lanes per SM, one FMA (2 flops) per lane per clock
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


def algorithmic_costs(p: int, fused_x2: bool = True) -> dict:
    """Algorithmic bytes and flops per DOF of each kernel class (FP32, 4-byte values).

    Flops count the sum-factorised quadrature once per element (no halo
    recomputation), one FMA = 2 flops, 30 flops per Gauss point for the
    pointwise terms (exp and reciprocal counted as one each).  With `fused_x2`
    the second x pass forms its right-hand side from T* and F itself (no
    separate matvec launch).
    """
    q = nb = p + 1
    W = 2 * p + 1
    fma = 3 * q * nb + 4 * q * q * nb + 4 * q * q * nb + 3 * q * nb + 2 * (W * W + W)
    rhs_flops = 2 * fma + 30 * q * q
    return {
        # read T, phi; write F, Phi, R
        "rhs_quadrature_1": dict(bytes=20, flops=rhs_flops),
        # two arrays (R with X_+, Phi with M^x): read + write each
        "xsolve_1": dict(bytes=16, flops=2 * (4 * p + 1) * 2),
        # two arrays: read solve input and base, write result
        "ysolve_1": dict(bytes=24, flops=2 * (4 * p + 2) * 2),
        # read T*, F; write R
        # sum-factorised: both x bands (W taps each) on T, both y bands on the results, scale F
        "matvec_2": dict(bytes=12, flops=2 * (2 * W) * 2 + 2),
        "xsolve_2": (dict(bytes=12, flops=2 * (2 * W) * 2 + 2 + (4 * p + 1) * 2) if fused_x2
                     else dict(bytes=8, flops=(4 * p + 1) * 2)),
        "ysolve_2": dict(bytes=12, flops=(4 * p + 2) * 2),
    }


def min_step_bytes(scheme: str) -> int:
    """Least HBM bytes per DOF of one step (FP32): fields read and written once per pass.

    PR: x1 reads T, phi and writes its two results and F (20); y1 reads and writes two
    fields (16); x2 reads T*, F and writes its result (12); y2 reads and writes one (8).
    Strang-CN: 16 + 16 (substep 1) + 8 (y substep) + 12 + 8 (substep 3).
    Explicit: x reads T, phi and writes two results (16); y reads them and the bases T, phi
    and writes two fields (24).
    """
    return {"pr": 56, "strang": 60, "explicit": 40}[scheme]


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
    with open(os.path.join(ROOT, "paper_2604_19370_gb300", "csrc", name), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _traffic_record(kernel_site: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        r = rec[kernel_site]
        if r["source_sha"] != _source_sha(r["source"]):
            return None
        return float(r["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock and throttle sampling during the timed region."""

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
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "samples": len(sm), "reasons": sorted(reasons)}


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


def _oracle_sample(steps: int, which: str = "c2", scheme: str = "pr") -> dict:
    """Run the FP64 oracle (ads mode) in a fresh single-threaded process; returns timing and state file."""
    out = tempfile.mktemp(suffix=".npz")
    code = f"""
import os, sys, time, json
sys.path.insert(0, {ROOT!r})
import numpy as np
from scenarios import config_c2
from oracle.step import Problem
sc = config_c2()
P = Problem.from_scenario(sc, scheme={scheme!r}, mode='ads')
T, phi = sc.T0.copy(), sc.fuel0.copy()
t0 = time.perf_counter()
for _ in range({steps}):
    T, phi = P.step(T, phi)
dt = time.perf_counter() - t0
np.savez({out!r}, T=T, phi=phi)
print(json.dumps(dict(seconds=dt, dofs=sc.dofs)))
"""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    res = json.loads(r.stdout.strip().splitlines()[-1])
    res["state"] = out
    res["steps"] = steps
    return res


def run_reference(args) -> None:
    world, rank, _ = _dist()
    if rank != 0:
        return
    from scenarios import config_c2

    sc = config_c2()
    # each oracle step takes seconds: warm-up and timed steps are capped to a bounded sample
    nsteps = min(args.warmup + args.steps, 24)
    res = _oracle_sample(nsteps)
    sec_per_step = res["seconds"] / nsteps
    value = sc.dofs / sec_per_step
    os.unlink(res["state"])
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": sec_per_step * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "c2_1024x1024_p2_pr", "nx": 1024, "ny": 1024, "p": 2, "dofs": sc.dofs,
                   "scheme": "PR", "impl": "FP64 CPU oracle, ads mode (1-D banded solves)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{nsteps} PR steps of the 1026^2-DOF workload (FP64, ads mode)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args) -> None:
    import numpy as np
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
    from scenarios import config_c2

    sc = config_c2(p=args.p) if args.nx == 1024 else None
    if sc is None:
        from scenarios import make_scenario

        sc = make_scenario(f"n{args.nx}", args.nx, args.p, 1e-3, 1, 2001, fuel_sigma=20.0,
                           wind_speed_range=(0.0, 3.0))
    prec = wf.WF_FP64 if args.fp64 else wf.WF_FP32
    scheme = {"pr": wf.WF_PR, "strang": wf.WF_STRANG_CN, "explicit": wf.WF_EXPLICIT}[scheme_of(args)]
    sim = wf.simulation_from_scenario(sc, precision=prec, scheme=scheme)
    stream = torch.cuda.Stream(device=dev)
    wf.wf_set_stream(sim.h, stream.cuda_stream)
    # launch shapes tuned on this handle (its state is restored afterwards)
    tuning = pick_shapes(wf, sim.h, args, 40)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    props = torch.cuda.get_device_properties(dev)

    # warm-up: captures the graphs, settles clocks
    with torch.cuda.stream(stream):
        sim.step(args.warmup)
    stream.synchronize()
    if sim.sync() != wf.WF_OK:
        raise RuntimeError("unstable during warm-up")

    def run_steps(profile: bool, sampler=None):
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

    # timed region: K steps replayed from the step's CUDA graph (the production launch path)
    with ClockSampler(local) as clk:
        ms_total = run_steps(False)
    status = sim.sync()
    value, slowest_s = whole_job_throughput(sc.dofs * args.steps, ms_total * 1e-3, world, dev)
    ms_per_step = slowest_s * 1e3 / args.steps

    # kernel durations: the same K steps launched kernel by kernel with a CUDA event pair around
    # each launch on the launching stream (the event records add small gaps between kernels,
    # which is why this pass is not the one that gives the step time)
    wf.wf_kernel_times(sim.h)  # reset
    n0 = wf.wf_launch_count()
    prof_ms_per_step = run_steps(True) / args.steps
    launches = wf.wf_launch_count() - n0  # kernels of the same K steps (the graph replays them)
    kt = wf.wf_kernel_times(sim.h)
    if sim.sync() != wf.WF_OK:
        status = wf.WF_EUNSTABLE

    # end to end through the C ABI with pinned host buffers: set state, one step, read state; the
    # host arrays are in the handle's working precision (float32 calls for the FP32 path)
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

    # roofline of the dominant kernel class
    peaks = _peaks()
    costs = algorithmic_costs(sc.p, fused_x2=("matvec_2" not in kt or kt["matvec_2"][1] == 0)
                              and scheme_of(args) == "pr")
    if scheme_of(args) == "explicit":
        costs["rhs_quadrature_1"]["bytes"] = 16  # no F stored
        costs["ysolve_2"]["bytes"] = 24  # two arrays with their bases
    es = 8 if args.fp64 else 4
    shares = {k: v[0] for k, v in kt.items() if v[1] > 0}
    dom = max(shares, key=shares.get)
    dom_ms = kt[dom][0] / kt[dom][1]
    c = costs.get(dom, dict(bytes=0, flops=0))
    bytes_per_launch = c["bytes"] * (es / 4) * sc.dofs
    flops_per_launch = c["flops"] * sc.dofs
    sm_count = props.multi_processor_count
    if args.fp64:
        alu_peak = FP64_NOMINAL_TFLOPS
        alu_src = "nominal FP64 rate of a GB300 (1.25 TFLOP/s)"
    else:
        alu_peak = fp32_alu_peak_tflops(sm_count, peaks["sm_max_mhz"])
        alu_src = f"derived: {sm_count} SMs x 128 FP32 lanes x 2 flop x {peaks['sm_max_mhz']:.0f} MHz"
    balance = alu_peak * 1e12 / (peaks["hbm_gbs"] * 1e9)
    ai = flops_per_launch / max(bytes_per_launch, 1)
    if ai > balance:
        achieved = flops_per_launch / (dom_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "peak_source": alu_src}
    else:
        achieved = bytes_per_launch / (dom_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "peak_source": f"{peaks['src']} copy bandwidth"}
    tr = _traffic_record(dom)
    roof.update({"kernel": dom, "ms_per_launch": dom_ms, "algorithmic_bytes_per_launch": bytes_per_launch,
                 "algorithmic_flops_per_launch": flops_per_launch, "traffic": tr})
    # whole-step HBM view: algorithmic bytes of all kernels of the step over the step time
    step_bytes = sum(costs[k]["bytes"] for k in costs if k in shares) * (es / 4) * sc.dofs
    kernels = {k: {"ms_per_launch": v[0] / v[1], "launches": v[1], "share": v[0] / sum(shares.values())}
               for k, v in kt.items() if v[1] > 0}

    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.fp64 else "f32",
        "data": "synthetic",
        "config": {"workload": f"c2_{sc.nx}x{sc.ny}_p{sc.p}_{scheme_of(args)}",
                   "nx": sc.nx, "ny": sc.ny, "p": sc.p, "dofs": sc.dofs,
                   "scheme": {"pr": "PR", "strang": "Strang-CN", "explicit": "explicit L2 projection"}[scheme_of(args)],
                   "precision": "fp64" if args.fp64 else "fp32 bulk, fp64 1-D factorisation",
                   "l2": "flushed before every timed step (256 MiB write)",
                   "launch_shapes": {"x_lines_per_cta": tuning[0], "y_lines_per_cta": tuning[1],
                                     "quadrature_segment_rows": tuning[2], "x_lines_per_warp": tuning[3],
                                     "x2_lines_per_cta": tuning[4], "x2_rhs": tuning[5],
                                     "source": shape_source(args)},
                   "parallelism": f"replicas x{world}"},
        "roofline": roof,
        "step_hbm_frac": min_step_bytes(scheme_of(args)) * (es / 4) * sc.dofs / (ms_per_step * 1e-3) / 1e9
        / peaks["hbm_gbs"],
        "step_hbm_frac_kernel_bytes": step_bytes / (ms_per_step * 1e-3) / 1e9 / peaks["hbm_gbs"],
        "profiled_ms_per_step": prof_ms_per_step,
        "kernels": kernels,
        "gpu_launches": launches,
        "e2e": {"value": world * sc.dofs / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 2 * es * n,
                "d2h_bytes_per_step": 2 * es * n, "ms_per_step": e2e_s * 1e3,
                "host_dtype": "float64" if args.fp64 else "float32"},
        "clocks": clk.summary(),
        "status": wf.wf_strerror(status),
    }

    # oracle baseline on a bounded sample (rank 0, N=1) and the rel-L2 of this path on the same steps
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ks = args.cpu_steps
        res = _oracle_sample(ks, scheme=scheme_of(args))
        d = np.load(res["state"])
        os.unlink(res["state"])
        chk = wf.simulation_from_scenario(sc, precision=prec, scheme=scheme)
        chk.step(ks)
        Tg, pg = chk.state()
        chk.close()
        rl = float(np.linalg.norm(Tg - d["T"]) / np.linalg.norm(d["T"]))
        rla = float(np.linalg.norm(Tg - d["T"]) / np.linalg.norm(d["T"] - 300.0))
        rlp = float(np.linalg.norm(pg - d["phi"]) / np.linalg.norm(d["phi"]))
        line["cpu_baseline"] = {"value": sc.dofs * ks / res["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{ks} {scheme_of(args)} steps of the same 1026^2-DOF workload, FP64, "
                                          "ads mode"}
        line["rel_l2_vs_oracle"] = {"steps": ks, "T": rl, "T_minus_Tamb": rla, "phi": rlp}
    sim.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()



def _percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q
    f = int(math.floor(k))
    c = min(f + 1, len(xs) - 1)
    return xs[f] + (xs[c] - xs[f]) * (k - f)


def run_ensemble(args) -> None:
    """Batched ensemble: S scenarios of 256^2 elements (p = 2) stepped together, one launch per kernel."""
    import numpy as np
    import torch

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2604_19370_gb300.build import build_library

    build_library()
    from paper_2604_19370_gb300 import wf
    from scenarios import config_c4

    S = args.scenarios
    first = config_c4(0)
    shared = first.fuel0
    scs = [first] + [config_c4(k, shared_fuel=shared) for k in range(1, S)]
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

    def timed(profile):
        wf.wf_set_profiling(b.h, profile)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(args.steps):
                wf.wf_step(b.h, 1)
            e1.record(stream)
        stream.synchronize()
        wf.wf_set_profiling(b.h, False)
        return e0.elapsed_time(e1) * 1e-3

    with ClockSampler(local) as clk:
        secs = timed(False)
    value, slowest = whole_job_throughput(dofs * args.steps, secs, world, dev)
    wf.wf_kernel_times(b.h)
    n0 = wf.wf_launch_count()
    timed(True)
    ens_launches = wf.wf_launch_count() - n0
    kt = wf.wf_kernel_times(b.h)
    st = b.status()
    peaks = _peaks()
    costs = algorithmic_costs(first.p)
    shares = {k: v[0] for k, v in kt.items() if v[1] > 0}
    dom = max(shares, key=shares.get)
    dom_ms = kt[dom][0] / kt[dom][1]
    props = torch.cuda.get_device_properties(dev)
    alu_peak = fp32_alu_peak_tflops(props.multi_processor_count, peaks["sm_max_mhz"])
    c = costs[dom]
    if c["flops"] / c["bytes"] > alu_peak * 1e12 / (peaks["hbm_gbs"] * 1e9):
        ach = c["flops"] * dofs / (dom_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s", "frac": ach / alu_peak}
    else:
        ach = c["bytes"] * dofs / (dom_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach / peaks["hbm_gbs"]}
    roof.update({"kernel": dom, "ms_per_launch": dom_ms, "traffic": None})
    step_bytes = sum(costs[k]["bytes"] for k in costs if k in shares) * dofs
    # end to end through the C ABI: every slot's state from pinned float32 host arrays in one call,
    # one step, every slot's state back in one call
    n = first.dofs
    hT = torch.empty(S * n, dtype=torch.float32, pin_memory=True)
    hP = torch.empty(S * n, dtype=torch.float32, pin_memory=True)
    for k, sc in enumerate(scs):
        hT.numpy()[k * n:(k + 1) * n] = sc.T0.ravel()
        hP.numpy()[k * n:(k + 1) * n] = sc.fuel0.ravel()
    wf.wf_batch_states_ptr(b.h, hT.data_ptr(), hP.data_ptr(), S * n, True, True)  # staging allocated here
    e2e_steps = 5
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        wf.wf_batch_states_ptr(b.h, hT.data_ptr(), hP.data_ptr(), S * n, True, True)
        wf.wf_step(b.h, 1)
        wf.wf_batch_states_ptr(b.h, hT.data_ptr(), hP.data_ptr(), S * n, True, False)
    e2e_s = reduce_max((time.perf_counter() - t0) / e2e_steps, dev)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": slowest * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"c4_ensemble_{S}x256x256_p2_pr", "scenarios": S, "nx": 256, "ny": 256, "p": 2,
                   "dofs": dofs, "l2": f"state {S} x 5 fields > L2, no flush", "parallelism": f"replicas x{world}",
                   "launch_shapes": {"x_lines_per_cta": tuning[0], "y_lines_per_cta": tuning[1],
                                     "quadrature_segment_rows": tuning[2], "x_lines_per_warp": tuning[3],
                                     "x2_lines_per_cta": tuning[4], "x2_rhs": tuning[5],
                                     "source": shape_source(args)}},
        "roofline": roof,
        "step_hbm_frac": min_step_bytes("pr") * dofs / (slowest / args.steps) / 1e9 / peaks["hbm_gbs"],
        "step_hbm_frac_kernel_bytes": step_bytes / (slowest / args.steps) / 1e9 / peaks["hbm_gbs"],
        "kernels": {k: {"ms_per_launch": v[0] / v[1], "launches": v[1]} for k, v in kt.items() if v[1] > 0},
        "gpu_launches": ens_launches,
        "e2e": {"value": world * dofs / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 2 * 4 * dofs,
                "d2h_bytes_per_step": 2 * 4 * dofs, "ms_per_step": e2e_s * 1e3, "host_dtype": "float32"},
        "clocks": clk.summary(),
        "unstable_slots": int(st.sum()),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle.step import Problem

        ks = 2
        P = Problem.from_scenario(scs[0], mode="ads")
        t0 = time.perf_counter()
        To, po = P.run(scs[0].T0, scs[0].fuel0, ks)
        cpu_s = time.perf_counter() - t0
        chk = wf.simulation_from_scenario(scs[0], precision=wf.WF_FP32)
        chk.step(ks)
        Tg, pg = chk.state()
        chk.close()
        line["cpu_baseline"] = {"value": first.dofs * ks / cpu_s, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{ks} PR steps of scenario 0 of the ensemble, FP64, ads mode"}
        line["rel_l2_vs_oracle"] = {"steps": ks, "T": float(np.linalg.norm(Tg - To) / np.linalg.norm(To))}
    b.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_serving(args) -> None:
    """Served request stream: Poisson arrivals at 80 % of measured capacity, p50/p99 latency."""
    import torch

    world, rank, local = _dist()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    from paper_2604_19370_gb300.build import build_library

    build_library()
    from paper_2604_19370_gb300 import wf
    from scenarios import make_scenario, request_stream_c5

    free, _total = torch.cuda.mem_get_info()
    budget = int(0.8 * free)

    def scenario(r):
        return make_scenario(f"q{r['seed']}", r["n"], r["p"], 1e-3, r["steps"], r["seed"], fuel_sigma=20.0,
                             wind_speed_range=(0.0, 3.0))

    def run(reqs, rate):
        srv = wf.Server(budget, max_slots=args.max_slots)
        prepared = [(scenario(r), r) for r in reqs]
        tickets, lat, dof_steps = {}, [], 0.0
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
            time.sleep(0.0005)
        makespan = time.perf_counter() - t_start
        srv.close()
        return lat, dof_steps, makespan

    # capacity: closed loop, every request submitted at once
    warm = request_stream_c5(4, 1.0, seed=55)
    run(warm, None)
    closed = request_stream_c5(args.requests, 1.0, seed=5)
    lat_c, ds_c, span_c = run(closed, None)
    capacity = len(lat_c) / span_c
    rate = 0.8 * capacity
    open_reqs = request_stream_c5(args.requests, rate, seed=6)
    lat, ds, span = run(open_reqs, rate)
    line = {
        "metric": METRIC, "value": ds / span, "unit": UNIT, "n_gpus": 1, "steps": len(open_reqs),
        "warmup": len(warm), "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (20% of requests f64)", "data": "synthetic",
        "config": {"workload": "c5_served_poisson", "requests": len(open_reqs), "arrival_rate_hz": rate,
                   "capacity_rps": capacity, "sizes": [128, 256, 512, 1024], "p": [2, 3],
                   "steps": "U[200,2000]", "fp64_share": 0.2, "hbm_budget_bytes": budget,
                   "max_slots_per_class": args.max_slots},
        "latency_p50_s": _percentile(lat, 0.5), "latency_p99_s": _percentile(lat, 0.99),
        "completed": len(lat), "closed_loop_dof_steps_per_s": ds_c / span_c,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--nx", type=int, default=1024)
    ap.add_argument("--p", type=int, default=2)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--strang", action="store_true")
    ap.add_argument("--explicit", action="store_true", help="explicit L2-projection scheme (the comparator)")
    ap.add_argument("--cpu-steps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="launch shapes from the launchers' rules")
    ap.add_argument("--tuning", default="", help="launch shapes x_cta,y_cta,seg,x_per_warp,x2_cta,x2_rhs (skips the autotuner)")
    ap.add_argument("--workload", default="c2", choices=["c2", "c4", "c5"],
                    help="c2: one 1024^2 domain (default); c4: batched ensemble; c5: served request stream")
    ap.add_argument("--scenarios", type=int, default=256)
    ap.add_argument("--requests", type=int, default=40)
    ap.add_argument("--max-slots", type=int, default=16)
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
        run_gpu(args)


if __name__ == "__main__":
    main()
