"""Conserved-to-primitive solvers on GB300: the accuracy and throughput study of the paper's
Sec. 3.3 rerun through the library's con2prim kernel.

The paper's grid: 25 Lorentz factors log-spaced in [1, 100] x 25 pressures log-spaced in
[1e5, 1e10] N/m^2, D = 1 kg/m^3, c = 3e8 m/s (here in units c = 1); each primitive state goes
prim -> cons -> prim and the relative error of the recovered velocity is recorded.  Timings use
the paper's batch of 10^3 cells x 27 points per grid state and a large batch (the whole grid
tiled to 2^24 recoveries) that fills the GPU.  The iterations the iterative solvers need to
match the closed forms' accuracy (the paper's Fig. 3) come from reruns with iteration caps
1, 2, ... (the caps count the FP32 and FP64 phases together).

    python -m paper_2205_00095_gb300.c2p_study [--reps R]   (prints one JSON object)
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from .solver import Solver

METHODS = [("ideal", "analytic"), ("ideal", "iterative"), ("tm", "analytic"), ("tm", "iterative")]


def _grid():
    import workloads as wl  # the repository's input generators (repository root on the path)
    W, lor, P_si = wl.e2_grid()
    return W.reshape(5, -1), np.tile(lor, 25), np.repeat(P_si, 25)


def accuracy(eos: str, c2p: str, max_iter: int = 0, gamma_ad: float = 5.0 / 3.0):
    """Relative velocity error and iteration count of every grid state (625,)."""
    Wf, lor, _ = _grid()
    n = Wf.shape[1]
    spec = dict(dim=1, degree=0, n_elem=[n], eos=eos, gamma_ad=gamma_ad, c2p=c2p, c2p_max_iter=max_iter)
    s = Solver(spec)
    W = torch.from_numpy(np.ascontiguousarray(Wf[:, :, None])).cuda()
    U = s.prim2cons(W)
    Wr, it = s.con2prim(U, with_iters=True)
    torch.cuda.synchronize()
    Wr = Wr.cpu().numpy()[:, :, 0]
    v = Wf[1]
    err = np.where(v > 0, np.abs(Wr[1] - v) / np.where(v > 0, v, 1.0), np.abs(Wr[1]))
    return err, it.cpu().numpy()[:, 0], lor


def iterations_to_parity(eos: str, kmax: int = 40):
    """Per grid state the smallest iteration cap at which the iterative solver's velocity error
    is no larger than the closed form's (the paper's Fig. 3); -1 where no cap up to kmax gets
    there, -2 where the closed form recovers the velocity exactly.  Returns (need, lor)."""
    err_a, _, lor = accuracy(eos, "analytic")
    need = np.where(err_a == 0.0, -2, -1)
    for k in range(1, kmax + 1):
        err_k, _, _ = accuracy(eos, "iterative", max_iter=k)
        hit = (need == -1) & (err_k <= err_a)
        need[hit] = k
    return need, lor


def parity_summary(need, lor) -> dict:
    """Median and quartiles over the pressures at each Lorentz factor, and the extremes."""
    gam = np.unique(lor)
    rows = []
    for g in gam:
        k = need[(lor == g) & (need > 0)]
        rows.append([float(g)] + ([float(np.median(k)), float(np.percentile(k, 25)),
                                   float(np.percentile(k, 75))] if k.size else [None] * 3))
    ok = need[need > 0]
    return {"by_gamma_median_q1_q3": rows, "max": int(ok.max()) if ok.size else None,
            "min": int(ok.min()) if ok.size else None,
            "analytic_exact_states": int((need == -2).sum()), "unreached": int((need == -1).sum())}


def throughput(eos: str, c2p: str, batch: int, reps: int = 20, gamma_ad: float = 5.0 / 3.0):
    """Recoveries per second of the grid states tiled to `batch` points."""
    Wf, _, _ = _grid()
    tiles = -(-batch // Wf.shape[1])
    Wb = np.tile(Wf, (1, tiles))[:, :batch]
    spec = dict(dim=1, degree=0, n_elem=[batch], eos=eos, gamma_ad=gamma_ad, c2p=c2p)
    stream = torch.cuda.Stream()
    s = Solver(spec, stream=stream)
    with torch.cuda.stream(stream):
        U = s.prim2cons(torch.from_numpy(np.ascontiguousarray(Wb[:, :, None])).cuda())
    W = s.empty()
    for _ in range(3):
        s.lib.dgsrhd_con2prim(s.ctx, U.data_ptr(), W.data_ptr(), None)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        s.lib.dgsrhd_con2prim(s.ctx, U.data_ptr(), W.data_ptr(), None)
    e1.record(stream)
    torch.cuda.synchronize()
    return batch * reps / (e0.elapsed_time(e1) * 1e-3)


def per_state_throughput(eos: str, c2p: str, points: int = 27000, reps: int = 10):
    """Recoveries per second for each grid state alone, in batches of `points` (the paper's
    10^3 cells x 27 points), one state at a time."""
    Wf, _, _ = _grid()
    spec = dict(dim=1, degree=0, n_elem=[points], eos=eos, gamma_ad=5.0 / 3.0, c2p=c2p)
    stream = torch.cuda.Stream()
    s = Solver(spec, stream=stream)
    out = np.zeros(Wf.shape[1])
    W = s.empty()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for j in range(Wf.shape[1]):
        Wj = np.repeat(Wf[:, j:j + 1], points, axis=1)[:, :, None]
        with torch.cuda.stream(stream):
            U = s.prim2cons(torch.from_numpy(np.ascontiguousarray(Wj)).cuda())
        s.lib.dgsrhd_con2prim(s.ctx, U.data_ptr(), W.data_ptr(), None)
        e0.record(stream)
        for _ in range(reps):
            s.lib.dgsrhd_con2prim(s.ctx, U.data_ptr(), W.data_ptr(), None)
        e1.record(stream)
        e1.synchronize()
        out[j] = points * reps / (e0.elapsed_time(e1) * 1e-3)
    return out


def study(reps: int = 20) -> dict:
    res = {"grid": "25 gamma in [1,100] x 25 P in [1e5,1e10] N/m^2, D = 1, c = 3e8 (units c = 1)"}
    for eos, c2p in METHODS:
        err, it, lor = accuracy(eos, c2p)
        key = f"{eos}_{c2p}"
        res[key] = {
            "max_rel_err_v_gamma_below_3": float(err[lor < 3].max()),
            "max_rel_err_v_gamma_below_10": float(err[lor < 10].max()),
            "max_rel_err_v_gamma_100": float(err[lor == lor.max()].max()),
            "mean_iterations": float(it.mean()),
            "recoveries_per_s_batch_2^24": throughput(eos, c2p, 1 << 24, reps),
        }
        pst = per_state_throughput(eos, c2p)
        res[key]["recoveries_per_s_27000_per_state_median"] = float(np.median(pst))
        res[key]["recoveries_per_s_27000_per_state_min_max"] = [float(pst.min()), float(pst.max())]
    for eos in ("ideal", "tm"):
        res[f"{eos}_iterations_to_parity"] = parity_summary(*iterations_to_parity(eos))
    for eos in ("ideal", "tm"):
        a = res[f"{eos}_analytic"]["recoveries_per_s_batch_2^24"]
        i = res[f"{eos}_iterative"]["recoveries_per_s_batch_2^24"]
        res[f"{eos}_analytic_time_over_iterative_time_minus_1"] = i / a - 1.0
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--reps", type=int, default=20)
    args = ap.parse_args()
    from . import build
    build.build()
    print(json.dumps(study(args.reps)))


if __name__ == "__main__":
    main()
