"""Growth of the Kelvin-Helmholtz instability in the paper's set-up (Sec. 4.5) on GB300: the
spatial mean <v_y^2>(t) sampled during the run, and the growth rate r from a least-squares fit
of log <v_y^2> = A + r t over t in [1.5, 3.0], the window the paper fits.

    python -m paper_2205_00095_gb300.kh_growth [--nx 256] [--degree 1] [--flux hll]
                                               [--t-end 3.0]   (prints one JSON object)
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from .solver import Solver


def _workloads():
    import workloads as wl  # the repository's input generators (repository root on the path)
    return wl


def fit_growth(t, m, lo: float = 1.5, hi: float = 3.0):
    """Least-squares line through (t, log m) over lo <= t <= hi: (rate, intercept, r^2)."""
    t, m = np.asarray(t, dtype=np.float64), np.asarray(m, dtype=np.float64)
    sel = (t >= lo) & (t <= hi) & (m > 0)
    if sel.sum() < 3:
        return float("nan"), float("nan"), float("nan")
    x, y = t[sel], np.log(m[sel])
    r, a = np.polyfit(x, y, 1)
    res = y - (a + r * x)
    r2 = 1.0 - float((res ** 2).sum()) / float(((y - y.mean()) ** 2).sum())
    return float(r), float(a), r2


def run(nx: int = 256, degree: int = 1, flux: str = "hll", t_end: float = 3.0,
        sample_dt: float = 0.05) -> dict:
    wl = _workloads()
    spec = wl.kh_single(nx=nx, ny=2 * nx, degree=degree, flux=flux)
    stream = torch.cuda.Stream()
    s = Solver(spec, stream=stream)
    with torch.cuda.stream(stream):
        U = s.initial_state(wl.kh_single_ic(spec, s.node_coords_device()))
        s.enforce(U)
    dt = s.cfl_dt(spec["cfl"])
    nsub = max(1, int(round(sample_dt / dt)))
    times, msq = [0.0], [s.mean_square_velocity(U, 1)]
    nsteps, step_s = 0, 0.0
    while times[-1] < t_end - 1e-12:
        n = min(nsub, int(np.ceil((t_end - times[-1]) / dt - 1e-9)))
        t0 = time.perf_counter()
        s.step(U, dt, n)
        s.synchronize()
        step_s += time.perf_counter() - t0
        nsteps += n
        times.append(nsteps * dt)
        msq.append(s.mean_square_velocity(U, 1))
    status, st = s.stats()
    r, a, r2 = fit_growth(times, msq)
    E, Nn = wl.shape(spec)
    s.close()
    return {"workload": f"kh_single {nx}x{2 * nx} elements p={degree} {flux.upper()} ideal Gamma=4/3 "
                        f"iterative con2prim SSPRK{spec['rk_stages']}, periodic x, outflow y",
            "dof": E * Nn, "dt": dt, "steps": nsteps, "t_end": nsteps * dt,
            "growth_rate_fit_1p5_to_3": r, "fit_intercept": a, "fit_r2": r2,
            "t": times, "mean_vy2": msq, "device_status": status, "stats": st,
            "dof_updates_per_s": E * Nn * nsteps * spec["rk_stages"] / step_s}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=256)
    ap.add_argument("--degree", type=int, default=1)
    ap.add_argument("--flux", default="hll", choices=["hll", "hllc", "llf"])
    ap.add_argument("--t-end", type=float, default=3.0)
    args = ap.parse_args()
    from . import build
    build.build()
    print(json.dumps(run(args.nx, args.degree, args.flux, args.t_end)))


if __name__ == "__main__":
    main()
