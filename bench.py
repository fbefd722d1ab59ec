"""Benchmark: DOF-updates/s of SSP-RK steps of the nodal DG SRHD solver on one GB300.

Default workload: the 2D advected density wave, 512 x 512 elements, p = 3 (16 Gauss-Legendre
nodes per element, 4,194,304 DOF), ideal EOS Gamma = 4/3, closed-form con2prim, LLF, SSPRK3,
FP64.  A DOF update is one node updated by one RK stage; DOF-updates/s = DOF x steps x stages /
seconds (the definition of the paper's performance section).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload advected_wave|kh2d|kh3d]

--gpus N > 1 runs one replica of the workload per rank (torchrun, one GPU each; the method has no
cross-replica exchange), barrier + synchronize around the timed region, max time over ranks.
--impl reference times the FP64 CPU oracle on the host cores on a bounded sample of the same
workload.  One JSON line is printed by rank 0.  Besides the FP64 value it carries the split-
precision form on the same workload (its rate, speed-up and L1 difference from FP64, and on the
advected wave both L1 errors against the exact solution), the adjoint/forward time ratio of the
checkpointed Kelvin-Helmholtz rollout, an end-to-end rate through dgsrhd_step_host with the
state in pinned host memory, the oracle's rate on a sample (cpu_baseline), the dominant
kernel's roofline, the per-kernel time shares, the kernel launch count and the SM clocks
sampled during the timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "DOF-updates/s at p=3 (FP64 vs split-precision, fixed L1 error); adjoint/forward ratio"
UNIT = "DOF-updates/s"
FP64_PEAK_TFLOPS = 1.25  # GB300 nominal dense FP64 (no FP64 figure in MEASURED_PEAKS.json)


def make_spec(name: str, c2p: str | None = None) -> dict:
    if name == "advected_wave":
        return wl.advected_wave(n=512, degree=3, c2p=c2p or "analytic")
    if name == "kh2d":
        return wl.kh2d(nx=256, ny=512, degree=3, c2p=c2p or "default")
    if name == "kh3d":
        return wl.kh3d(n=128, degree=3, c2p=c2p or "default")
    raise SystemExit(f"unknown workload {name}")


def workload_desc(spec: dict) -> str:
    n = "x".join(str(v) for v in spec["n_elem"][: spec["dim"]])
    return (f"{spec['name']} {n} elements p={spec['degree']} {spec['eos']} EOS "
            f"c2p={spec['c2p']} flux={spec['flux']} SSPRK{spec['rk_stages']} FP64")


def dof(spec: dict) -> int:
    E, Nn = wl.shape(spec)
    return E * Nn


# ----------------------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, log_dir: str | None = None):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(log_dir or tempfile.gettempdir(), f"clocks_bench_{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smmax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smmax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smmax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------------------
# algorithmic work (per DOF update, p = 3, 2D) used for the roofline of the volume kernel
# ----------------------------------------------------------------------------------------
# Algorithmic FP64 operations per node of the volume kernel, counted from the method's arithmetic
# as the oracle writes it (add, sub, mul, div = 1; fma = 2; sqrt, cbrt and other library calls
# = 1 each; comparisons not counted):
#   con2prim, closed-form ideal quartic:    12 (xi, eta, admissibility) + 87 (quartic
#       coefficients, resolvent cubic, Cardano root, two quadratic factors) + 21 (rho, v, P)
#   con2prim, Newton on the Riccardi quartic: 12 + 20 (series start) + 19 per iteration
#       (Horner value and derivative, step) + 17 (rho, v, P)
#   con2prim, Taub-Matthews cubic closed form: 12 + 25 (coefficients) + 16 (Cardano) + 24
#   con2prim, Taub-Matthews Brent: 12 + 25 + 14 per iteration (cubic value 6, interpolation 8)
#       + 24
#   nodal flux 7 per axis; volume term 2 N 5 per axis (pre-scaled Dhat); face traces 2 N 5 per
#   face point, 2 dim N^(dim-1) face points per N^dim nodes.
C2P_FLOPS = {
    ("ideal", "analytic"): lambda it: 120.0,
    ("ideal", "iterative"): lambda it: 12.0 + 20.0 + 19.0 * it + 17.0,
    ("tm", "analytic"): lambda it: 12.0 + 25.0 + 16.0 + 24.0,
    ("tm", "iterative"): lambda it: 12.0 + 25.0 + 14.0 * it + 24.0,
}


def volume_kernel_flops_per_node(spec: dict, mean_iters: float = 0.0) -> float:
    d, N = spec["dim"], spec["degree"] + 1
    c2p = spec["c2p"]
    if c2p == "default":
        c2p = "analytic" if spec["eos"] == "ideal" else "iterative"
    flux = 7.0 * d
    volume = 2.0 * N * 5 * d
    traces = (2.0 * d * N ** (d - 1) / N ** d) * 5 * 2.0 * N
    return C2P_FLOPS[(spec["eos"], c2p)](mean_iters) + flux + volume + traces


def _capture_record(kernel: str, workload_name: str):
    """The committed ncu record of `kernel` on this workload, or None when there is none or the
    kernel sources changed since it was taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "dram_traffic_advected_wave_512x512_p3.json")
    if workload_name != "advected_wave" or not os.path.exists(path):
        return None
    d = json.load(open(path))
    h = hashlib.sha1()
    for f in d["source_files"]:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    if h.hexdigest() != d["source_sha1"] or kernel not in d["kernels"]:
        return None
    return d["kernels"][kernel]


def measured_traffic(kernel: str, workload_name: str):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu capture."""
    k = _capture_record(kernel, workload_name)
    return None if k is None else k["dram_bytes_read"] + k["dram_bytes_write"]


def measured_fp64_pipe(kernel: str, workload_name: str):
    """Fraction of active cycles the FP64 pipe was busy in the committed ncu capture."""
    k = _capture_record(kernel, workload_name)
    return None if k is None or "fp64_pipe_busy_pct" not in k else k["fp64_pipe_busy_pct"] / 100.0


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except (OSError, ValueError):
        return None


# ----------------------------------------------------------------------------------------
# reference arm / CPU baseline: the oracle on a bounded sample
# ----------------------------------------------------------------------------------------
def oracle_sample_spec(spec: dict, target_s: float = 1.0):
    """A sample of the workload (same field, p, EOS, solver) small enough for one oracle step to
    take about target_s seconds on one core."""
    import oracle
    s = dict(spec)
    d = spec["dim"]
    n = 8 if d == 3 else 32
    s["n_elem"] = [n] * d if spec["name"] != "kh_2d" else [n, 2 * n]
    X = oracle.node_coords(s)
    U = oracle.prim2cons(s, wl.initial_primitive(s, X))
    t0 = time.perf_counter()
    oracle.step(s, U, oracle.cfl_dt(s, 0.2), 1)
    t = time.perf_counter() - t0
    scale = max(1.0, (target_s / max(t, 1e-6)) ** (1.0 / d))
    # never larger than the workload itself
    s["n_elem"] = [min(int(full), max(2, int(v * scale))) for v, full in zip(s["n_elem"], spec["n_elem"])]
    return s


def run_oracle(spec: dict, steps: int, warmup: int):
    import oracle
    X = oracle.node_coords(spec)
    U = oracle.prim2cons(spec, wl.initial_primitive(spec, X))
    dt = oracle.cfl_dt(spec, 0.2)
    for _ in range(warmup):
        U, _ = oracle.step(spec, U, dt, 1)
    t0 = time.perf_counter()
    for _ in range(steps):
        U, _ = oracle.step(spec, U, dt, 1)
    t = time.perf_counter() - t0
    return dof(spec) * steps * spec["rk_stages"] / t, t


def reduce_max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over the ranks (the slowest replica's time); x itself on one rank."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, ndof: int, steps: int, stages: int, t_ms: float) -> float:
    """Whole-job DOF-updates/s: every replica advances ndof nodes through steps x stages stage
    updates; the job takes the slowest replica's t_ms."""
    return world * ndof * steps * stages / (t_ms * 1e-3)


def reference_arm(args, rank, world):
    if rank != 0:
        return
    spec = make_spec(args.workload, args.c2p)
    sample = oracle_sample_spec(spec, target_s=min(20.0, 60.0 / max(1, args.steps + args.warmup)))
    value, t = run_oracle(sample, args.steps, args.warmup)
    desc = (f"{args.steps} oracle SSPRK steps on {'x'.join(map(str, sample['n_elem']))} elements of the "
            f"same workload ({dof(sample)} DOF), 1 thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_desc(spec), "sample": desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------------
def ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2205_00095_gb300 import Solver, build

    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    spec = make_spec(args.workload, args.c2p)
    stream = torch.cuda.Stream(device=dev)
    s = Solver(spec, stream=stream, device=dev)
    with torch.cuda.stream(stream):
        U0 = s.initial_state(wl.initial_primitive(spec, s.node_coords_device()))
        s.enforce(U0)
        U = U0.clone()
    dt = s.cfl_dt(0.2)
    stages = spec["rk_stages"]
    ndof = dof(spec)

    # warm-up (also captures the step graph)
    s.step(U, dt, max(1, args.warmup))
    torch.cuda.synchronize(dev)
    s.stats(reset=True)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # timed region: K steps with every kernel bracketed by CUDA events on the solver's stream
    s.set_profiling(True)
    s.kernel_times(reset=True)
    launches0 = s.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(local_rank, args.clock_log_dir) as clk:
        ev0.record(stream)
        s.step(U, dt, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    ms = ev0.elapsed_time(ev1)
    launches = s.kernel_launches() - launches0
    ktimes = s.kernel_times(reset=True)
    s.set_profiling(False)
    status, st = s.stats()
    t_max = reduce_max_over_ranks(ms, world, dev)
    value = job_throughput(world, ndof, args.steps, stages, t_max)

    # end to end through the C ABI with a pinned host state: per step H2D, one step (graph), D2H
    e2e = None
    if not args.no_e2e:
        Uh = U0.cpu().pin_memory()
        nbytes = Uh.numel() * 8
        s.step_host(Uh, dt, 1)  # warm
        Uh.copy_(U0.cpu())
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            s.step_host(Uh, dt, 1)
        barrier()
        e2e_s = time.perf_counter() - t0
        e2e_max = reduce_max_over_ranks(e2e_s, world, dev)
        e2e = {"value": job_throughput(world, ndof, args.steps, stages, 1e3 * e2e_max), "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "transfer": "dgsrhd_step_host on a pinned host state: the first kernel of each step "
                           "reads it over the host link and the last writes it back, overlapped "
                           "with compute"}

    # split-precision form on the same workload: tensor-core contractions, FP64 elsewhere
    split = None
    if not args.no_split:
        ss = Solver(dict(spec, precision="split"), stream=stream, device=dev)
        with torch.cuda.stream(stream):
            V = U0.clone()
        ss.step(V, dt, max(1, args.warmup))
        ss.set_profiling(True)
        ss.kernel_times(reset=True)
        barrier()
        ev0.record(stream)
        ss.step(V, dt, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        sms = ev0.elapsed_time(ev1)
        sk = ss.kernel_times(reset=True)
        ss.set_profiling(False)
        with torch.cuda.stream(stream):
            l1 = float(((V - U).abs().sum() / U.abs().sum()).item())
        exact = {}
        if args.workload == "advected_wave":
            # both runs against the translated wave at t = (warm-up + timed steps) dt
            t_end = (max(1, args.warmup) + args.steps) * dt
            with torch.cuda.stream(stream):
                Ue = s.initial_state(wl.advected_wave_ic(spec, s.node_coords_device(), t_end))
                nrm = Ue.abs().sum()
                exact = {"t": t_end,
                         "l1_err_vs_exact_fp64": float(((U - Ue).abs().sum() / nrm).item()),
                         "l1_err_vs_exact_split": float(((V - Ue).abs().sum() / nrm).item())}
        sstatus, _ = ss.stats()
        split = {"value": world * ndof * args.steps * stages / (sms * 1e-3), "unit": UNIT,
                 "ms_per_step": sms / args.steps, "speedup_vs_fp64": ms / sms,
                 "l1_rel_vs_fp64": l1, **exact, "device_status": sstatus,
                 "contractions": "volume term and traces 3xTF32 mma.sync m16n8k8 with FP32 accumulation, lift as FP32 FMAs, deviation form",
                 "kernel_ms_per_launch": {k: round(v[0] / max(v[1], 1), 4) for k, v in sk.items() if v[1]}}
        ss.close()

    # adjoint: gradient of the transverse kinetic energy after 200 SSPRK3 steps of the 2D
    # Kelvin-Helmholtz set-up at 128 x 256, p = 3, checkpoint every 20 steps, against the forward
    adj = None
    if not args.no_adjoint:
        from paper_2205_00095_gb300 import adjoint as adjm
        spec4 = wl.kh2d(nx=128, ny=256, degree=3)
        sa = Solver(spec4, stream=stream, device=dev)
        with torch.cuda.stream(stream):
            A0 = sa.initial_state(wl.kh2d_ic(spec4, sa.node_coords_device()))
            sa.enforce(A0)
            Af = A0.clone()
        dta = sa.cfl_dt(0.2)
        sa.step(Af, dta, 3)  # warm-up and graph capture
        with torch.cuda.stream(stream):
            Af.copy_(A0)
        barrier()
        ev0.record(stream)
        sa.step(Af, dta, 200)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        fwd_ms = ev0.elapsed_time(ev1)
        barrier()
        # untimed warm-up rollout: one checkpoint segment, so that the stage buffers of a
        # segment come from the allocator's cache in the timed run
        with torch.cuda.stream(stream):
            Uw = A0.clone().requires_grad_(True)
            adjm.transverse_kinetic_energy(sa, adjm.rollout(sa, Uw, dta, 40, 20)).backward()
            del Uw
            U0g = A0.clone().requires_grad_(True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            UT = adjm.rollout(sa, U0g, dta, 200, 20)
            Jv = adjm.transverse_kinetic_energy(sa, UT)
            Jv.backward()
        torch.cuda.synchronize(dev)
        adj_ms = 1e3 * (time.perf_counter() - t0)
        ast, ast_counts = sa.stats()
        adj = {"workload": "kh_2d 128x256 elements p=3 TM Brent HLL SSPRK3, 200 steps, checkpoint every 20",
               "objective": "sum rho gamma^2 v_y^2 at t_final", "forward_ms": fwd_ms,
               "forward_plus_adjoint_ms": adj_ms, "adjoint_forward_ratio": adj_ms / fwd_ms,
               "grad_norm": float(U0g.grad.norm()), "enforced_cells": ast_counts["enforced_cells"]}
        sa.close()

    # oracle on the host cores (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = oracle_sample_spec(spec, target_s=5.0)
        cv, ct = run_oracle(sample, 2, 0)
        cpu = {"value": cv, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"2 oracle SSPRK3 steps on {'x'.join(map(str, sample['n_elem']))} elements of the "
                         f"same workload ({dof(sample)} DOF, {ct:.1f} s), 1 thread"}

    # roofline of the dominant kernel (largest share of the timed region)
    dom = max(ktimes, key=lambda k: ktimes[k][0])
    dom_ms, dom_n = ktimes[dom]
    avg_s = dom_ms / max(dom_n, 1) * 1e-3
    roofline = None
    if dom == "volume":
        mean_it = st["c2p_iters_total"] / max(st["c2p_calls"], 1)
        fpn = volume_kernel_flops_per_node(spec, mean_it)
        flops = fpn * ndof
        achieved = flops / avg_s / 1e12
        roofline = {"kernel": "volume_kernel", "bound": "alu", "achieved": achieved,
                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                    "traffic": measured_traffic("volume_kernel", args.workload),
                    "fp64_pipe_busy_ncu": measured_fp64_pipe("volume_kernel", args.workload),
                    "peak_source": "GB300 nominal dense FP64 1.25 TFLOP/s (DFMA probe measured 1.256)",
                    "algorithmic_flops_per_node": fpn,
                    "avg_launch_ms": avg_s * 1e3}
    else:
        roofline = {"kernel": dom, "bound": "alu", "achieved": None, "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": None, "traffic": None, "avg_launch_ms": avg_s * 1e3}
    shares = {k: round(v[0] / max(sum(x[0] for x in ktimes.values()), 1e-12), 4)
              for k, v in ktimes.items() if v[1]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(spec), "dof": ndof, "stages_per_step": stages,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": f"inputs larger than L2 (state {40 * ndof / 1e6:.0f} MB + scratch)",
                       "precision": "fp64",
                       **({"seed": spec["seed"]} if "seed" in spec else {})},
            "roofline": roofline, "kernel_shares": shares,
            "split_precision": split,
            "adjoint": adj,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "device_status": status,
            "stats": st,
        }
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="advected_wave", choices=["advected_wave", "kh2d", "kh3d"])
    ap.add_argument("--c2p", default=None, choices=["analytic", "iterative", "default"],
                    help="con2prim solver (default: the workload's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end timing")
    ap.add_argument("--no-split", action="store_true", help="skip the split-precision run")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/forward timing")
    ap.add_argument("--clock-log-dir", default=None,
                    help="where the nvidia-smi clock samples of the timed region are written "
                         "(default: the system temporary directory)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
