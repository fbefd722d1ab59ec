"""The paper's 2D Riemann problems (Sec. 4.4) at a chosen resolution on GB300: quadrant states
on [-1, 1]^2, ideal EOS Gamma = 5/3, HLLC, a limiter and the physicality operator, to t = 0.8.
Reports the step count, time and DOF-updates/s, the device counters, the smallest density
and pressure at the nodes, and for test 3 (symmetric about the diagonal x = y) the largest
departure from that symmetry.

    python -m paper_2205_00095_gb300.riemann2d [--test 1 2 3] [--n 1024] [--degree 1]
                                               [--limiter moe|minmod]   (one JSON per test)
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from .solver import Solver


def _workloads():
    import workloads as wl  # the repository's input generators (repository root on the path)
    return wl


def run(test: int, n: int = 1024, degree: int = 1, limiter: str = "moe") -> dict:
    """Run 2D Riemann test 1, 2 or 3 on an n x n mesh to t = 0.8; one result dict."""
    wl = _workloads()
    spec = dict(wl.riemann_2d(test, n=n, degree=degree), limiter=limiter)
    stream = torch.cuda.Stream()
    s = Solver(spec, stream=stream)
    with torch.cuda.stream(stream):
        U = s.initial_state(wl.initial_primitive(spec, s.node_coords_device()))
        s.enforce(U)
    T = spec["t_final"]
    nsteps = int(np.ceil(T / s.cfl_dt(spec["cfl"])))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.synchronize()
    ev0.record(stream)
    s.step(U, T / nsteps, nsteps)
    ev1.record(stream)
    s.synchronize()
    ms = ev0.elapsed_time(ev1)
    status, st = s.stats()
    W = s.con2prim(U)
    s.synchronize()
    N = degree + 1
    out = {"test": test, "n": n, "degree": degree, "limiter": limiter, "steps": nsteps,
           "seconds": ms * 1e-3,
           "dof_updates_per_s": n * n * N * N * nsteps * spec["rk_stages"] / (ms * 1e-3),
           "status": int(status), "stats": st,
           "rho_min": float(W[0].min().item()), "P_min": float(W[4].min().item())}
    if test == 3:
        # mirror about x = y: swap the element axes, the node axes and the two momenta
        V = U.cpu().numpy().reshape(5, n, n, N, N)
        M = V.transpose(0, 2, 1, 4, 3).copy()
        M[[1, 2]] = M[[2, 1]]
        out["symmetry_rel"] = float(np.abs(M - V).max() / np.abs(V).max())
    s.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--test", nargs="+", type=int, default=[1, 2, 3])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--degree", type=int, default=1)
    ap.add_argument("--limiter", default="moe", choices=["moe", "minmod"])
    a = ap.parse_args(argv)
    for t in a.test:
        print(json.dumps(run(t, a.n, a.degree, a.limiter)), flush=True)


if __name__ == "__main__":
    main()
