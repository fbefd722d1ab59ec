"""Throughput of the paper's Kelvin-Helmholtz set-up on GB300 (the performance study of Sec. 4.6):
DOF-updates/s = DOF x steps x stages / time with DOF = n_x n_y (p + 1)^2, for the paper's
resolutions 256 x 512, 512 x 1024 and 1024 x 2048, basis orders p = 0, 1, 2 paired with RK1,
SSPRK2 and SSPRK3, HLL and HLLC, plus smaller meshes that show where the GPU saturates.  Each
point times a fixed number of steps between CUDA events on the solver's stream after a warm-up.

    python -m paper_2205_00095_gb300.kh_perf [--steps 50] [--flux hll hllc]
                                             (prints one JSON object per point)
"""
from __future__ import annotations

import argparse
import json

import torch

from .solver import Solver


def _workloads():
    import workloads as wl  # the repository's input generators (repository root on the path)
    return wl


# (n_x, n_y): the paper's three resolutions and smaller ones down to saturation
PAPER_MESHES = [(256, 512), (512, 1024), (1024, 2048)]
SMALL_MESHES = [(16, 32), (32, 64), (64, 128), (128, 256)]


def measure(nx: int, ny: int, degree: int, flux: str = "hll", steps: int = 50,
            warmup: int = 3) -> dict:
    """Time `steps` steps of the single-layer Kelvin-Helmholtz problem on an n_x x n_y mesh at
    basis order `degree` after `warmup` untimed steps; one result dict."""
    wl = _workloads()
    spec = wl.kh_single(nx=nx, ny=ny, degree=degree, flux=flux)
    stream = torch.cuda.Stream()
    s = Solver(spec, stream=stream)
    with torch.cuda.stream(stream):
        U = s.initial_state(wl.kh_single_ic(spec, s.node_coords_device()))
        s.enforce(U)
    dt = s.cfl_dt(spec["cfl"])
    s.step(U, dt, warmup)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.synchronize()
    ev0.record(stream)
    s.step(U, dt, steps)
    ev1.record(stream)
    s.synchronize()
    ms = ev0.elapsed_time(ev1)
    status, st = s.stats()
    dof = nx * ny * (degree + 1) ** 2
    stages = spec["rk_stages"]
    s.close()
    return {"n_x": nx, "n_y": ny, "degree": degree, "rk_stages": stages, "flux": flux,
            "dof": dof, "steps": steps, "ms_per_step": ms / steps,
            "dof_updates_per_s": dof * steps * stages / (ms * 1e-3), "status": int(status),
            "launches_per_step": 3 * stages}


def sweep(steps: int = 50, fluxes=("hll", "hllc"), degrees=(0, 1, 2), small: bool = True):
    """measure() over every flux, degree and mesh (the small meshes first when `small`)."""
    meshes = (SMALL_MESHES if small else []) + PAPER_MESHES
    for flux in fluxes:
        for degree in degrees:
            for nx, ny in meshes:
                yield measure(nx, ny, degree, flux, steps)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--flux", nargs="+", default=["hll", "hllc"], choices=["llf", "hll", "hllc"])
    ap.add_argument("--degrees", nargs="+", type=int, default=[0, 1, 2])
    ap.add_argument("--no-small", action="store_true", help="only the paper's three meshes")
    a = ap.parse_args(argv)
    for r in sweep(a.steps, a.flux, a.degrees, not a.no_small):
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
