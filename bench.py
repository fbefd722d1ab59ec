"""Benchmark: DOF-updates/s of SSP-RK steps of the nodal DG SRHD solver on one GB300.

Default workload: the 2D advected density wave, 512 x 512 elements, p = 3 (16 Gauss-Legendre
nodes per element, 4,194,304 DOF), ideal EOS Gamma = 4/3, closed-form con2prim, LLF, SSPRK3,
FP64.  A DOF update is one node updated by one RK stage; DOF-updates/s = DOF x steps x stages /
seconds (the definition of the paper's performance section).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload advected_wave|kh2d|kh3d]

--gpus N > 1 runs one replica of the workload per rank (torchrun, one GPU each; the method has no
cross-replica exchange), barrier + synchronize around the timed region, max time over ranks.
--impl reference times the FP64 CPU oracle on all host cores (one process per core, each
stepping its own copy of a bounded sample of the same workload).  One JSON line is printed by
rank 0.  Keys beyond the common ones:
  value / ms_per_step  K steps replayed from the captured CUDA graph (the production path of
                       dgsrhd_step), CUDA events on the solver's stream;
  kernel_timing        a second pass of K steps with every kernel bracketed by CUDA events
                       (launched directly): per-kernel mean launch time and share, and that
                       pass's own ms_per_step;
  roofline / rooflines the dominant kernel's and every stage kernel's algorithmic FP64 rate
                       against the FP64 ALU peak derived from the unit counts (152 SMs x 2 FMA
                       lanes x 2 flops) and the SM clock of the timed region, with the counting
                       rule, and the dominant kernel's rate against the probe's DFMA rate;
  fp64_peak            the library's DFMA probe (a DFMA loop reaches 0.84 of the ALU peak), FP32
                       FMA throughput, the cost of division, square root, reciprocal square root
                       and reciprocal cube root in DFMA-equivalents, and the SM clock during it;
  split_precision      the split-precision form on the same workload (rate, speed-up, L1
                       difference from FP64; on the advected wave both L1 errors against the
                       exact solution);
  workloads            the 2D Taub-Matthews Kelvin-Helmholtz problem at 256 x 512 and the 3D one
                       at 128^3 (FP64 and split rates, L1 difference, con2prim iterations,
                       volume-kernel roofline);
  adjoint              adjoint/forward time ratio of the checkpointed 128 x 256 Kelvin-Helmholtz
                       rollout, with its dJ/dA against the oracle's central differences stored in
                       tests/golden/kh_adjoint_c4.json;
  e2e                  the same metric through dgsrhd_step_host with the state in pinned host
                       memory (host link traffic inside the timed region);
  cpu_baseline         the oracle on all host cores and on one thread;
  clocks               SM clocks sampled with nvidia-smi during the timed region.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
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


def make_spec(name: str, c2p: str | None = None, n: int | None = None) -> dict:
    """The named workload at its benchmark size, or with n elements along x (a smaller case for
    a profiler capture: n x n, n x 2n and n^3)."""
    if name == "advected_wave":
        return wl.advected_wave(n=n or 512, degree=3, c2p=c2p or "analytic")
    if name == "kh2d":
        return wl.kh2d(nx=n or 256, ny=2 * n if n else 512, degree=3, c2p=c2p or "default")
    if name == "kh3d":
        return wl.kh3d(n=n or 128, degree=3, c2p=c2p or "default")
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
    """nvidia-smi samples every 50 ms, each stamped with its wall-clock time. The sampler starts
    before the warm-up (nvidia-smi itself takes a while to start), and `begin()` / `end()` mark
    the timed region: the summary keeps the samples inside it."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,timestamp")

    def __init__(self, gpu_index: int, log_dir: str | None = None, tag: str = "bench"):
        self.gpu = gpu_index
        self.proc = None
        self.window = None
        self.path = os.path.join(log_dir or tempfile.gettempdir(), f"clocks_{tag}_{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return self
        t0 = time.time()  # wait (3 s at most) for the first sample, so the timed region is covered
        while self.proc.poll() is None and time.time() - t0 < 3.0 and os.path.getsize(self.path) == 0:
            time.sleep(0.02)
        return self

    def begin(self):
        self.window = [time.time(), None]

    def end(self):
        if self.window is not None:
            self.window[1] = time.time()

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
        w = tuple(self.window) if self.window and self.window[1] is not None else None
        return summarize_clock_lines(open(self.path).read().splitlines(), w)


def _stamp(text):
    """nvidia-smi's timestamp field ("2026/12/04 10:11:12.345", local time) in seconds."""
    import datetime
    try:
        return datetime.datetime.strptime(text.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
    except ValueError:
        return None


def summarize_clock_lines(lines, window=None):
    """Median SM clock, max clock and the throttle reasons seen in nvidia-smi CSV samples; with a
    (begin, end) window, only the samples stamped inside it (the nearest one if none is)."""
    rows = []
    for line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm, smmax = float(f[1]), float(f[2])
        except ValueError:
            continue
        rows.append((sm, smmax, f[5:9], _stamp(f[9]) if len(f) > 9 else None))
    scope = "all samples"
    if window is not None and rows and all(r[3] is not None for r in rows):
        inside = [r for r in rows if window[0] <= r[3] <= window[1]]
        if inside:
            rows, scope = inside, "timed region"
        else:
            mid = 0.5 * (window[0] + window[1])
            rows, scope = [min(rows, key=lambda r: abs(r[3] - mid))], "nearest sample to the timed region"
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = {n for r in rows for n, v in zip(names, r[2]) if v.lower() == "active"}
    return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
            "reasons": sorted(reasons), "samples": len(rows), "scope": scope}


# ----------------------------------------------------------------------------------------
# algorithmic work per unit of each stage kernel (FP64 roofline)
# ----------------------------------------------------------------------------------------
# Counting rule: the method's arithmetic as the oracle writes it, each add, sub, mul, div,
# sqrt, cbrt or library call = 1 flop, a fused multiply-add = 2, comparisons not counted.
# Volume kernel, per node:
#   con2prim, closed-form ideal quartic:    12 (xi, eta, admissibility) + 87 (quartic
#       coefficients, resolvent cubic, Cardano root, two quadratic factors) + 21 (rho, v, P)
#   con2prim, Newton on the Riccardi quartic: 12 + 20 (series start) + 19 per iteration
#       (Horner value and derivative, step) + 17 (rho, v, P)
#   con2prim, Taub-Matthews cubic closed form: 12 + 25 (coefficients) + 16 (Cardano) + 24
#   con2prim, Taub-Matthews Brent: 12 + 25 + 14 per iteration (cubic value 6, interpolation 8)
#       + 24
#   nodal flux 7 per axis; volume term 2 N 5 per axis; face traces 2 N 5 per face point,
#   2 dim N^(dim-1) face points per N^dim nodes.
# Face kernel, per face point: two face states from (rho, u, P) (u^2 5, gamma 2, v_d 1, h - 1 2
#   ideal / 9 Taub-Matthews, D 1, rho h gamma^2 3, S 3, tau 7: 24 / 31), their normal fluxes
#   (7 each), their wavespeeds (sound speed 2 ideal / 10 Taub-Matthews, sigma 3, root 5,
#   lambda 5: 15 / 23), and the combination: LLF 26 (5 x (sum, difference, two products,
#   difference) + a/2), HLL 32 (5 x 6 + S_L S_R + the denominator), HLLC 72 (HLL averages 40,
#   contact speed 8, star state and flux 24).
# Update kernel, per node: lift 2 x 2 x 5 per axis, Shu-Osher combination 2 per variable in the
#   first stage and 5 in the later ones (averaged over the stages), admissibility test 8.
C2P_FLOPS = {
    ("ideal", "analytic"): lambda it: 120.0,
    ("ideal", "iterative"): lambda it: 12.0 + 20.0 + 19.0 * it + 17.0,
    ("tm", "analytic"): lambda it: 12.0 + 25.0 + 16.0 + 24.0,
    ("tm", "iterative"): lambda it: 12.0 + 25.0 + 14.0 * it + 24.0,
}
FACE_STATE_FLOPS = {"ideal": 24.0 + 7.0 + 15.0, "tm": 31.0 + 7.0 + 23.0}
FACE_COMBINE_FLOPS = {"llf": 26.0, "hll": 32.0, "hllc": 72.0}
COUNTING_RULE = ("algorithmic FP64 flops of the method as the oracle writes it (add, sub, mul, div, "
                 "sqrt, cbrt, library call = 1; fma = 2; comparisons 0); per node for the volume and "
                 "update kernels, per face point for the face kernel")

# FP64 FMA lanes per SM per clock: the count that gives the nominal 1.25 TFLOP/s of GB300 at its
# 2070 MHz maximum SM clock (152 x 2 x 2 x 2.07e9 = 1.2586e12), and the one ncu's FP64-pipe
# utilisation is taken against (the library's DFMA probe, 0.505e12 DFMA/s at 1985 MHz, reads
# as 84 % busy).
FP64_FMA_PER_SM_CLK = 2


def fp64_alu_peak_tflops(sms: int, sm_mhz: float) -> float:
    """The FP64 ALU peak from the unit counts and the SM clock: SMs x FMA lanes x 2 flops x clock."""
    return sms * FP64_FMA_PER_SM_CLK * 2.0 * sm_mhz * 1e6 / 1e12


def resolved_c2p(spec: dict) -> str:
    c2p = spec["c2p"]
    if c2p == "default":
        c2p = "analytic" if spec["eos"] == "ideal" else "iterative"
    return c2p


def volume_kernel_flops_per_node(spec: dict, mean_iters: float = 0.0) -> float:
    d, N = spec["dim"], spec["degree"] + 1
    flux = 7.0 * d
    volume = 2.0 * N * 5 * d
    traces = (2.0 * d * N ** (d - 1) / N ** d) * 5 * 2.0 * N
    return C2P_FLOPS[(spec["eos"], resolved_c2p(spec))](mean_iters) + flux + volume + traces


def face_kernel_flops_per_point(spec: dict) -> float:
    return 2.0 * FACE_STATE_FLOPS[spec["eos"]] + FACE_COMBINE_FLOPS[spec["flux"]]


def update_kernel_flops_per_node(spec: dict) -> float:
    d, ns = spec["dim"], spec["rk_stages"]
    rk = (2.0 * 5 + (ns - 1) * 5.0 * 5) / ns
    return 20.0 * d + rk + 8.0


def face_points(spec: dict) -> int:
    """Face points of one face-kernel launch: every face of every axis, N^(dim-1) points each
    (a non-periodic axis has n_d + 1 faces per line of elements)."""
    E, _ = wl.shape(spec)
    d, N = spec["dim"], spec["degree"] + 1
    total = 0
    for a in range(d):
        bc = (spec.get("bc") or [("periodic", "periodic")] * d)[a]
        nf = E + (0 if bc[0] == "periodic" else E // spec["n_elem"][a])
        total += nf * N ** (d - 1)
    return total


def _capture_record(kernel: str, workload_name: str):
    """The committed ncu record of `kernel` on this workload, or None when there is none or the
    kernel sources changed since it was taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"dram_traffic_{workload_name}_512x512_p3.json")
    if not os.path.exists(path):
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


def kernel_roofline(name: str, flops_per_unit: float, units: int, avg_ms: float, peak_tflops: float,
                    traffic=None, pipe=None) -> dict:
    """Algorithmic FP64 rate of one kernel: flops_per_unit x units per launch / mean launch
    time, against the FP64 ALU peak."""
    achieved = flops_per_unit * units / (avg_ms * 1e-3) / 1e12 if avg_ms > 0 else None
    return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak_tflops,
            "unit": "TFLOP/s", "frac": None if achieved is None else achieved / peak_tflops,
            "traffic": traffic, "fp64_pipe_busy_ncu": pipe,
            "algorithmic_flops_per_unit": flops_per_unit, "units_per_launch": units,
            "avg_launch_ms": avg_ms}


# ----------------------------------------------------------------------------------------
# reference arm / CPU baseline: the oracle on a bounded sample, on all host cores
# ----------------------------------------------------------------------------------------
def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


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


def _oracle_worker(args):
    spec, steps, warmup = args
    return run_oracle(spec, steps, warmup)


def run_oracle_all_cores(spec: dict, steps: int, warmup: int, procs: int):
    """procs oracle processes (spawned), each stepping its own copy of `spec`: the summed
    DOF-updates/s and the slowest process's time."""
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_oracle_worker, [(spec, steps, warmup)] * procs, chunksize=1)
    return sum(r[0] for r in res), max(r[1] for r in res)


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
    spec = make_spec(args.workload, args.c2p, args.n)
    procs = host_cores()
    sample = oracle_sample_spec(spec, target_s=min(20.0, 60.0 / max(1, args.steps + args.warmup)))
    value, t = run_oracle_all_cores(sample, args.steps, args.warmup, procs)
    desc = (f"{args.steps} oracle SSPRK steps on {'x'.join(map(str, sample['n_elem']))} elements of the "
            f"same workload ({dof(sample)} DOF) in each of {procs} processes, one per host core")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_desc(spec), "sample": desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------------
PROBE_KINDS = ("dfma", "ffma", "ddiv", "dsqrt", "drsqrt", "drcbrt", "recip", "sqrt", "rcbrt",
               "rsqrt")


def measure_fp64_peak(dev, stream, clock_dir, local_rank, target_ms=150.0):
    """Throughput of the library's arithmetic probe kernels (one kernel per operation, four
    independent chains per thread, 8 blocks of 256 threads per SM), timed with CUDA events."""
    import torch
    from paper_2205_00095_gb300.solver import arith_probe
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.empty(sms * 8 * 256, dtype=torch.float64, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rates = {}
    with ClockSampler(local_rank, clock_dir, tag="probe") as clk:
        for kind in PROBE_KINDS:
            iters = 64
            with torch.cuda.stream(stream):
                arith_probe(kind, iters, sink, stream)  # warm-up
            for _ in range(2):  # calibrate to ~target_ms, then time
                ev0.record(stream)
                ops = arith_probe(kind, iters, sink, stream)
                ev1.record(stream)
                torch.cuda.synchronize(dev)
                ms = ev0.elapsed_time(ev1)
                if ms >= 0.5 * target_ms:
                    break
                iters = max(iters, int(iters * target_ms / max(ms, 1e-3)))
            rates[kind] = ops / (ms * 1e-3)
    dfma = rates["dfma"]
    return {
        "dfma_per_s": dfma, "tflops": 2.0 * dfma / 1e12, "ffma_tflops": 2.0 * rates["ffma"] / 1e12,
        "fp32_fp64_fma_ratio": rates["ffma"] / dfma,
        "dfma_equivalents": {k: dfma / rates[k] for k in PROBE_KINDS if k not in ("dfma", "ffma")},
        "method": (f"dgsrhd_arith_probe: {sms * 8 * 256} threads x 4 independent chains, "
                   f"~{target_ms:.0f} ms per operation, CUDA events"),
        "clocks": clk.summary(),
    }


class Timed:
    """K steps of one workload: graph replay (value), then a profiling pass with per-kernel
    CUDA events."""

    def __init__(self, spec, steps, warmup, dev, stream, barrier, clock=None):
        import torch
        from paper_2205_00095_gb300 import Solver
        self.spec, self.steps = spec, steps
        self.s = Solver(spec, stream=stream, device=dev)
        with torch.cuda.stream(stream):
            self.U0 = self.s.initial_state(wl.initial_primitive(spec, self.s.node_coords_device()))
            self.s.enforce(self.U0)
            self.U = self.U0.clone()
        self.dt = self.s.cfl_dt(0.2)
        s = self.s
        if clock is not None:
            clock.__enter__()
        s.step(self.U, self.dt, max(1, warmup))  # warm-up, captures the step graph
        torch.cuda.synchronize(dev)
        s.stats(reset=True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = s.kernel_launches()
        barrier()
        if clock is not None:
            clock.begin()
        ev0.record(stream)
        s.step(self.U, self.dt, steps)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        if clock is not None:
            clock.end()
            clock.__exit__()
        barrier()
        self.ms = ev0.elapsed_time(ev1)
        self.launches = s.kernel_launches() - l0
        self.status, self.st = s.stats(reset=True)
        # second pass: every kernel bracketed by CUDA events (launched directly)
        s.set_profiling(True)
        s.kernel_times(reset=True)
        V = self.U.clone()
        barrier()
        ev0.record(stream)
        s.step(V, self.dt, steps)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        self.ms_prof = ev0.elapsed_time(ev1)
        self.ktimes = s.kernel_times(reset=True)
        s.set_profiling(False)
        del V

    def mean_iters(self):
        return self.st["c2p_iters_total"] / max(self.st["c2p_calls"], 1)

    def rooflines(self, peak, workload_name):
        spec, nd = self.spec, dof(self.spec)
        out = {}
        for kind, kname, fpu, units in (
                ("volume", "volume_kernel", volume_kernel_flops_per_node(spec, self.mean_iters()), nd),
                ("face", "face_kernel", face_kernel_flops_per_point(spec), face_points(spec)),
                ("update", "update_kernel", update_kernel_flops_per_node(spec), nd)):
            ms, n = self.ktimes[kind]
            if n:
                out[kind] = kernel_roofline(kname, fpu, units, ms / n, peak,
                                            measured_traffic(kname, workload_name),
                                            measured_fp64_pipe(kname, workload_name))
        return out

    def shares(self):
        tot = sum(v[0] for v in self.ktimes.values())
        return {k: round(v[0] / max(tot, 1e-12), 4) for k, v in self.ktimes.items() if v[1]}

    def close(self):
        self.s.close()


def run_split(spec, U0, U_fp64, dt, steps, warmup, dev, stream, barrier):
    """The split-precision form from the same initial state: (ms, solver stats, L1 difference
    from the FP64 state, per-kernel ms per launch, final state)."""
    import torch
    from paper_2205_00095_gb300 import Solver
    ss = Solver(dict(spec, precision="split"), stream=stream, device=dev)
    with torch.cuda.stream(stream):
        V = U0.clone()
    ss.step(V, dt, max(1, warmup))
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    ss.step(V, dt, steps)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    sms = ev0.elapsed_time(ev1)
    # per-kernel times in a separate pass (on a copy; V keeps the graph-replayed state)
    ss.set_profiling(True)
    ss.kernel_times(reset=True)
    with torch.cuda.stream(stream):
        V2 = V.clone()
    ss.step(V2, dt, steps)
    sk = ss.kernel_times(reset=True)
    ss.set_profiling(False)
    del V2
    with torch.cuda.stream(stream):
        l1 = float(((V - U_fp64).abs().sum() / U_fp64.abs().sum()).item())
    sstatus, _ = ss.stats()
    ss.close()
    return sms, sstatus, l1, {k: round(v[0] / max(v[1], 1), 4) for k, v in sk.items() if v[1]}, V


def run_workload_entry(spec, steps, warmup, dev, stream, barrier, peak, world, with_split=True):
    """FP64 and split rates of one extra workload, its volume-kernel roofline and con2prim
    iterations."""
    import torch
    T = Timed(spec, steps, warmup, dev, stream, barrier)
    nd, stages = dof(spec), spec["rk_stages"]
    rl = T.rooflines(peak, spec["name"])
    entry = {"workload": workload_desc(spec), "dof": nd, "steps": steps,
             "value": job_throughput(world, nd, steps, stages, T.ms), "unit": UNIT,
             "ms_per_step": T.ms / steps, "mean_c2p_iterations": T.mean_iters(),
             "device_status": T.status, "stats": T.st,
             "volume_roofline": rl.get("volume"), "kernel_shares": T.shares()}
    if "seed" in spec:
        entry["seed"] = spec["seed"]
    if with_split:
        sms, sstatus, l1, sk, V = run_split(spec, T.U0, T.U, T.dt, steps, warmup, dev, stream, barrier)
        del V
        entry["split_precision"] = {"value": job_throughput(world, nd, steps, stages, sms),
                                    "ms_per_step": sms / steps, "speedup_vs_fp64": T.ms / sms,
                                    "l1_rel_vs_fp64": l1, "device_status": sstatus,
                                    "kernel_ms_per_launch": sk}
    T.close()
    torch.cuda.empty_cache()
    return entry


def adjoint_block(dev, stream, barrier):
    """Adjoint/forward time ratio of the checkpointed Kelvin-Helmholtz rollout (128 x 256, p = 3,
    200 SSPRK3 steps, checkpoint every 20), and its dJ/dA against the oracle's stored central
    differences."""
    import torch
    from paper_2205_00095_gb300 import Solver
    from paper_2205_00095_gb300 import adjoint as adjm
    spec4 = wl.kh2d(nx=128, ny=256, degree=3)
    sa = Solver(spec4, stream=stream, device=dev)
    X = sa.node_coords_device()
    with torch.cuda.stream(stream):
        W0 = wl.kh2d_ic(spec4, X)
        A0 = sa.initial_state(W0)
        Af = A0.clone()
    dta = sa.cfl_dt(0.2)
    sa.step(Af, dta, 3)  # warm-up and graph capture
    with torch.cuda.stream(stream):
        Af.copy_(A0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    sa.step(Af, dta, 200)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    fwd_ms = ev0.elapsed_time(ev1)
    barrier()
    # untimed warm-up rollout: one checkpoint segment, so that the stage buffers of a segment
    # come from the allocator's cache in the timed run
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
    # dJ/dA: the adjoint contracted with the tangent of prim -> cons along dW/dA (v_y only)
    with torch.cuda.stream(stream):
        dW = torch.zeros_like(W0)
        dW[2] = wl.kh2d_ic(spec4, X, amplitude=1.0)[2]
        h = 1e-6
        tang = (sa.initial_state(W0 + h * dW) - sa.initial_state(W0 - h * dW)) / (2 * h)
        g_adj = float((U0g.grad * tang).sum().item())
        J = float(Jv.detach().item())
    torch.cuda.synchronize(dev)
    adj = {"workload": "kh_2d 128x256 elements p=3 TM Brent HLL SSPRK3, 200 steps, checkpoint every 20",
           "objective": "sum rho gamma^2 v_y^2 at t_final", "forward_ms": fwd_ms,
           "forward_plus_adjoint_ms": adj_ms, "adjoint_forward_ratio": adj_ms / fwd_ms,
           "J": J, "dJ_dA_adjoint": g_adj, "grad_norm": float(U0g.grad.norm()),
           "enforced_cells": ast_counts["enforced_cells"], "device_status": ast}
    golden = os.path.join(ROOT, "tests", "golden", "kh_adjoint_c4.json")
    if os.path.exists(golden):
        g = json.load(open(golden))
        fd = g["dJ_dA"]["fd_h"]
        adj.update({"dJ_dA_oracle_fd": fd, "rel_err_vs_oracle_fd": abs(g_adj - fd) / abs(fd),
                    "J_rel_err_vs_oracle": abs(J - g["J"]) / abs(g["J"]),
                    "oracle_dt": g["configuration"]["dt"], "dt": dta})
    sa.close()
    return adj


def ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2205_00095_gb300 import build

    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # FP64 throughput of this GPU, measured by the probe before the workload; the roofline's
    # peak is derived from the unit counts and the SM clock sampled during the timed region
    probe = None if args.no_probe else measure_fp64_peak(dev, stream, args.clock_log_dir, local_rank)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count

    spec = make_spec(args.workload, args.c2p, args.n)
    stages = spec["rk_stages"]
    ndof = dof(spec)
    clk = ClockSampler(local_rank, args.clock_log_dir)
    T = Timed(spec, args.steps, args.warmup, dev, stream, barrier, clock=clk)
    s, U0, U, dt = T.s, T.U0, T.U, T.dt
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or (probe or {}).get("clocks", {}).get("sm_mhz") or 2070.0
    peak = fp64_alu_peak_tflops(n_sm, sm_mhz)
    t_max = reduce_max_over_ranks(T.ms, world, dev)
    value = job_throughput(world, ndof, args.steps, stages, t_max)

    # end to end through the C ABI with a pinned host state: per step H2D, one step, D2H
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
        sms, sstatus, l1, sk, V = run_split(spec, U0, U, dt, args.steps, args.warmup, dev, stream, barrier)
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
        del V
        split = {"value": job_throughput(world, ndof, args.steps, stages, sms), "unit": UNIT,
                 "ms_per_step": sms / args.steps, "speedup_vs_fp64": T.ms / sms,
                 "l1_rel_vs_fp64": l1, **exact, "device_status": sstatus,
                 "contractions": "volume term and traces 3xTF32 mma.sync m16n8k8 with FP32 accumulation, lift as FP32 FMAs, deviation form",
                 "kernel_ms_per_launch": sk}

    # the committed ncu record covers the benchmark size only
    rooflines = T.rooflines(peak, args.workload if args.n is None else f"{args.workload}_n{args.n}")
    shares = T.shares()
    ktimes = T.ktimes
    launches, status, st = T.launches, T.status, T.st
    T.close()
    del s, U0, U
    torch.cuda.empty_cache()

    # the larger configurations: 2D Taub-Matthews KH 256 x 512 and 3D KH 128^3
    extra = None
    if not args.no_workloads:
        extra = {}
        for name, steps in (("kh2d", args.steps), ("kh3d", min(args.steps, 20))):
            if name == args.workload:
                continue
            extra[name] = run_workload_entry(make_spec(name), steps, args.warmup, dev, stream, barrier,
                                             peak, world, with_split=not args.no_split)

    adj = None if args.no_adjoint else adjoint_block(dev, stream, barrier)

    # oracle on the host cores (rank 0, N = 1 only): all cores and one thread
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        procs = host_cores()
        sample = oracle_sample_spec(spec, target_s=5.0)
        v1, t1 = run_oracle(sample, 2, 0)
        vn, tn = run_oracle_all_cores(sample, 2, 0, procs)
        n = "x".join(map(str, sample["n_elem"]))
        cpu = {"value": vn, "unit": UNIT, "cores": procs, "kind": "oracle",
               "sample": f"2 oracle SSPRK3 steps on {n} elements of the same workload ({dof(sample)} DOF) "
                         f"in each of {procs} processes, one per host core ({tn:.1f} s)",
               "single_thread": {"value": v1, "cores": 1,
                                 "sample": f"2 oracle SSPRK3 steps on {n} elements, one process ({t1:.1f} s)"}}

    # roofline of the dominant kernel (largest share of the profiled pass)
    dom = max(("volume", "face", "update"), key=lambda k: ktimes[k][0])
    probe_note = ("" if probe is None else
                  f"; the library's DFMA probe measured {probe['tflops']:.4f} TFLOP/s "
                  f"({probe['tflops'] / peak:.2f} of it) in this run")
    roofline = dict(rooflines[dom], peak_source=(
        f"derived FP64 ALU peak: {n_sm} SMs x {FP64_FMA_PER_SM_CLK} FMA/clock x 2 flops x {sm_mhz:.0f} MHz "
        f"(median SM clock of the timed region){probe_note}; {COUNTING_RULE}"),
        frac_of_probe=None if probe is None else rooflines[dom]["achieved"] / probe["tflops"])

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(spec), "dof": ndof, "stages_per_step": stages,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": f"inputs larger than L2 (state {40 * ndof / 1e6:.0f} MB + scratch)",
                       "precision": "fp64", "timed_path": "dgsrhd_step graph replay",
                       **({"seed": spec["seed"]} if "seed" in spec else {})},
            "roofline": roofline, "rooflines": rooflines, "fp64_peak": probe,
            "kernel_timing": {"pass": "second pass of the same K steps, every kernel launched directly "
                                      "between CUDA events (no graph)",
                              "ms_per_step": T.ms_prof / args.steps,
                              "graph_gain": T.ms_prof / T.ms,
                              "kernel_shares": shares,
                              "kernel_ms_per_launch": {k: round(v[0] / max(v[1], 1), 4)
                                                       for k, v in ktimes.items() if v[1]}},
            "split_precision": split,
            "workloads": extra,
            "adjoint": adj,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
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
    ap.add_argument("--n", type=int, default=None,
                    help="elements along x instead of the benchmark size (n x n, n x 2n, n^3), for "
                         "profiler captures of a smaller case")
    ap.add_argument("--c2p", default=None, choices=["analytic", "iterative", "default"],
                    help="con2prim solver (default: the workload's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end timing")
    ap.add_argument("--no-split", action="store_true", help="skip the split-precision runs")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/forward timing")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the 2D and 3D Kelvin-Helmholtz workloads")
    ap.add_argument("--no-probe", action="store_true",
                    help="skip the arithmetic throughput probe (the roofline's peak is derived "
                         "from the unit counts and clocks either way)")
    ap.add_argument("--clock-log-dir", default=None,
                    help="where the nvidia-smi clock samples are written "
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
