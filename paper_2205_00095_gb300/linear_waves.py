"""Linear-wave convergence (Sec. 4.1) on GB300: for each eigenpair j in {-, 0(1), 0(2), 0(3), +}
a wave of amplitude 1e-6 on the base state (rho, v, P) = (1, 0, 1), ideal EOS Gamma = 5/3, runs
to t = 0.5 at four resolutions (refinement doubles the elements per axis; the time step follows
the CFL rule), and the L1 errors of the conserved (D, S, E) and primitive (rho, u = gamma v, P)
variables against the travelling wave are fitted to L1(dx) = p0 + p1 dx^p2 as the paper does;
p2 is the order (expected p + 1 with the SSP-RK of p + 1 stages).  The default configuration is
the one of the paper's table: oblique 3D box, p = 2, SSPRK3.

    python -m paper_2205_00095_gb300.linear_waves [--frame 3d_oblique] [--degree 2]
                                                  [--n-base 4] [--levels 4]   (one JSON object)
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np
import torch

from .solver import Solver

WAVES = ("-", "0(1)", "0(2)", "0(3)", "+")
NAMES = ("D", "S_x", "S_y", "S_z", "E", "rho", "u_x", "u_y", "u_z", "P")


def _workloads():
    import workloads as wl  # the repository's input generators (repository root on the path)
    return wl


def eigenpair(wave: str, rho0: float = 1.0, P0: float = 1.0, gamma_ad: float = 5.0 / 3.0):
    """Right eigenvector (rho, v_par, v_perp1, v_perp2, P) and eigenvalue at rest for the ideal
    gas: acoustic (rho, +-c_s, 0, 0, rho h c_s^2) at +-c_s with h = 1 + Gamma P / ((Gamma - 1)
    rho) and c_s^2 = Gamma P / (rho h); entropy (1, 0, 0, 0, 0) and shear (unit transverse
    velocity) at 0."""
    if wave in ("-", "+"):
        h = 1.0 + gamma_ad / (gamma_ad - 1.0) * P0 / rho0
        cs = math.sqrt(gamma_ad * P0 / (rho0 * h))
        s = 1.0 if wave == "+" else -1.0
        return (rho0, s * cs, 0.0, 0.0, rho0 * h * cs * cs), s * cs
    return {"0(1)": (1.0, 0.0, 0.0, 0.0, 0.0), "0(2)": (0.0, 0.0, 1.0, 0.0, 0.0),
            "0(3)": (0.0, 0.0, 0.0, 1.0, 0.0)}[wave], 0.0


def fit_order(dx, err):
    """p2 of L1(dx) = p0 + p1 dx^p2 (least squares; p0 >= 0), and the slope of the finest two."""
    dx, err = np.asarray(dx, dtype=np.float64), np.asarray(err, dtype=np.float64)
    slope = float(np.log(err[-2] / err[-1]) / np.log(dx[-2] / dx[-1]))
    try:
        from scipy.optimize import curve_fit
        f = lambda h, p0, lp1, p2: p0 + np.exp(lp1) * h ** p2
        popt, _ = curve_fit(f, dx, err, p0=[0.0, math.log(err[-1] / dx[-1] ** slope), slope],
                            bounds=([0.0, -200.0, 0.0], [err.min(), 200.0, 20.0]), maxfev=20000)
        return float(popt[2]), slope
    except Exception:
        return float("nan"), slope


def errors(s: Solver, spec: dict, U: torch.Tensor, t: float, wl):
    X = s.node_coords_device()
    We = wl.linear_wave_ic(spec, X, t)
    Ue = s.initial_state(We)
    W = s.con2prim(U)
    from .solver import node_weights_nd
    dim = int(spec["dim"])
    wq = torch.from_numpy(node_weights_nd(spec)).to(U.device)
    jac = np.prod([(spec["hi"][d] - spec["lo"][d]) / spec["n_elem"][d] / 2.0 for d in range(dim)])
    vol = np.prod([spec["hi"][d] - spec["lo"][d] for d in range(dim)])
    E = U[4] + U[0]
    Ee = Ue[4] + Ue[0]

    def four_velocity(Wv):
        g = 1.0 / torch.sqrt(1.0 - (Wv[1:4] ** 2).sum(0))
        return [g * Wv[1 + c] for c in range(3)]

    u, ue = four_velocity(W), four_velocity(We)
    pairs = [(U[0], Ue[0]), (U[1], Ue[1]), (U[2], Ue[2]), (U[3], Ue[3]), (E, Ee), (W[0], We[0]),
             (u[0], ue[0]), (u[1], ue[1]), (u[2], ue[2]), (W[4], We[4])]
    out = []
    for a, b in pairs:
        out.append(float(((a - b).abs() * wq).sum()) * jac / vol)
    # variables the wave leaves alone (their exact perturbation is zero): None
    base = [float((b - b.mean()).abs().max()) for _, b in pairs]
    return out, base


def run_wave(frame, wave, degree, n_base, levels, wl):
    r, lam = eigenpair(wave)
    dxs, errs, bases = [], [], None
    for lev in range(levels):
        spec = wl.linear_wave(frame, degree, n_base, lev, r, lam)
        stream = torch.cuda.Stream()
        s = Solver(spec, stream=stream)
        with torch.cuda.stream(stream):
            U = s.initial_state(wl.linear_wave_ic(spec, s.node_coords_device()))
        T = spec["t_final"]
        nsteps = int(math.ceil(T / s.cfl_dt(spec["cfl"])))
        s.step(U, T / nsteps, nsteps)
        with torch.cuda.stream(stream):
            e, base = errors(s, spec, U, T, wl)
        s.synchronize()
        status, _ = s.stats()
        assert status == 0, status
        dxs.append((spec["hi"][0] - spec["lo"][0]) / spec["n_elem"][0])
        errs.append(e)
        bases = base
        s.close()
    errs = np.array(errs)
    res = {}
    for k, name in enumerate(NAMES):
        if bases[k] == 0.0:
            res[name] = None
            continue
        p2, slope = fit_order(dxs, errs[:, k])
        res[name] = {"order_fit": p2, "order_finest_pair": slope, "l1": errs[:, k].tolist()}
    return {"dx": dxs, "variables": res}


def study(frame="3d_oblique", degree=2, n_base=4, levels=4) -> dict:
    wl = _workloads()
    out = {"frame": frame, "degree": degree, "rk_stages": min(degree + 1, 3), "n_base": n_base,
           "levels": levels, "base_state": "rho = 1, v = 0, P = 1, Gamma = 5/3, A = 1e-6, t = 0.5"}
    for wave in WAVES:
        out[wave] = run_wave(frame, wave, degree, n_base, levels, wl)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--frame", default="3d_oblique")
    ap.add_argument("--degree", type=int, default=2)
    ap.add_argument("--n-base", type=int, default=4)
    ap.add_argument("--levels", type=int, default=4)
    args = ap.parse_args()
    from . import build
    build.build()
    print(json.dumps(study(args.frame, args.degree, args.n_base, args.levels)))


if __name__ == "__main__":
    main()
