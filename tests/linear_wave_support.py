"""Linear-wave eigenpairs from the oracle's equation of state and the L1 errors of a state
against the travelling wave (test infrastructure for the linear-wave tests of Sec. 4.1)."""
import math

import numpy as np

import oracle
import workloads as wl

WAVES = ("-", "0(1)", "0(2)", "0(3)", "+")


def eigenpair(wave: str, rho0=1.0, P0=1.0, gamma_ad=5.0 / 3.0):
    """Right eigenvector (rho, v_par, v_perp1, v_perp2, P) and eigenvalue at rest: acoustic
    waves (rho, +-c_s, 0, 0, rho h c_s^2) at +-c_s, the entropy wave (1, 0, 0, 0, 0) and the two
    shear waves (unit transverse velocity) at 0."""
    spec = dict(dim=1, degree=0, n_elem=[1], eos="ideal", gamma_ad=gamma_ad)
    if wave in ("-", "+"):
        cs = math.sqrt(oracle.cs2(spec, rho0, P0))
        h = oracle.enthalpy(spec, rho0, P0)
        s = 1.0 if wave == "+" else -1.0
        return (rho0, s * cs, 0.0, 0.0, rho0 * h * cs * cs), s * cs
    return {"0(1)": (1.0, 0.0, 0.0, 0.0, 0.0), "0(2)": (0.0, 0.0, 1.0, 0.0, 0.0),
            "0(3)": (0.0, 0.0, 0.0, 1.0, 0.0)}[wave], 0.0


def make(frame, wave, degree, n_base, refine, **kw):
    r, lam = eigenpair(wave)
    return wl.linear_wave(frame, degree, n_base, refine, r, lam, **kw)


def l1_errors(spec, U, t):
    """L1 norms over the box of U - U_exact(t) for the five conserved variables, divided by
    the box volume (nodal quadrature)."""
    X = oracle.node_coords(spec)
    Ue = oracle.prim2cons(spec, wl.linear_wave_ic(spec, X, t))
    N = spec["degree"] + 1
    w1 = np.polynomial.legendre.leggauss(N)[1]
    w = w1
    for _ in range(spec["dim"] - 1):
        w = np.multiply.outer(w1, w).ravel()
    jac, vol = 1.0, 1.0
    for d in range(spec["dim"]):
        dx = (spec["hi"][d] - spec["lo"][d]) / spec["n_elem"][d]
        jac *= dx / 2.0
        vol *= spec["hi"][d] - spec["lo"][d]
    return (np.abs(U - Ue) * w).sum(axis=(1, 2)) * jac / vol


def order(e_coarse, e_fine, h_coarse, h_fine):
    return math.log(e_coarse / e_fine) / math.log(h_coarse / h_fine)
