"""The oracle's DG solution of the 1D blast wave (Sec. 4.2, problem 1) against the exact
Riemann solution: the physicality operator keeps it admissible at p = 1 and p = 2, the L1
error falls with resolution and with degree."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as wl
from oracle.exact_riemann import ExactRiemann

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "blast_wave_problem1.json")


def run(n, degree):
    spec = wl.blast_wave(n=n, degree=degree)
    X = oracle.node_coords(spec)
    U = oracle.prim2cons(spec, wl.blast_wave_ic(spec, X))
    U, _, _ = oracle.enforce(spec, U)
    T = spec["t_final"]
    dt = oracle.cfl_dt(spec, spec["cfl"])
    nsteps = int(round(T / dt))
    U, st = oracle.step(spec, U, T / nsteps, nsteps)
    g = json.load(open(GOLDEN))
    ex = ExactRiemann((g["left"]["rho"], 0.0, g["left"]["P_workload"]),
                      (g["right"]["rho"], 0.0, g["right"]["P_workload"]), g["gamma_ad"],
                      g["interface"])
    Uex = oracle.prim2cons(spec, ex.sample(X[0], T))
    w = np.polynomial.legendre.leggauss(degree + 1)[1]
    l1 = (np.abs(U - Uex) * w).sum(axis=(1, 2)) / (2 * n)
    return l1, st


def test_blast_wave_workload_matches_paper_problem():
    g = json.load(open(GOLDEN))
    spec = wl.blast_wave()
    assert spec["left"][0] == g["left"]["rho"] and spec["right"][0] == g["right"]["rho"]
    assert spec["left"][4] == g["left"]["P_workload"] and spec["right"][4] == g["right"]["P_workload"]
    assert spec["t_final"] == g["t_final"] and spec["gamma_ad"] == g["gamma_ad"]


def test_blast_wave_converges_to_exact_solution():
    l1_64, st64 = run(64, 1)
    l1_128, st128 = run(128, 1)
    l1_256, _ = run(256, 1)
    for st in (st64, st128):
        assert st["c2p_invalid_input"] == 0 and st["mean_inadmissible_cells"] == 0
        assert st["enforced_cells"] > 0
    # shocks limit the order to about one (Sec. 4.2); require a clear decrease
    k = [0, 1, 4]  # D, S_x, tau (the transverse momenta stay zero)
    assert np.all(l1_128[k] < 0.8 * l1_64[k]) and np.all(l1_256[k] < 0.8 * l1_128[k])
    assert l1_128[0] < 0.1


def test_higher_degree_is_more_accurate():
    l0, _ = run(128, 0)
    l1, _ = run(128, 1)
    l2, st = run(128, 2)
    assert l1[0] < 0.3 * l0[0] and l2[0] < l1[0]
    assert st["c2p_invalid_input"] == 0


def test_gll_nodes_converge_without_the_face_guard():
    """The same blast wave on Gauss-Lobatto nodes (p = 1): no face guard hits, and the L1
    error still falls with resolution."""
    errs = []
    for n in (64, 128):
        spec = dict(wl.blast_wave(n=n, degree=1), nodes="gll")
        X = oracle.node_coords(spec)
        U = oracle.prim2cons(spec, wl.blast_wave_ic(spec, X))
        U, _, _ = oracle.enforce(spec, U)
        T = spec["t_final"]
        nsteps = int(round(T / oracle.cfl_dt(spec, spec["cfl"])))
        U, st = oracle.step(spec, U, T / nsteps, nsteps)
        assert st["face_guard_hits"] == 0 and st["mean_inadmissible_cells"] == 0
        g = json.load(open(GOLDEN))
        ex = ExactRiemann((g["left"]["rho"], 0.0, g["left"]["P_workload"]),
                          (g["right"]["rho"], 0.0, g["right"]["P_workload"]), g["gamma_ad"],
                          g["interface"])
        Uex = oracle.prim2cons(spec, ex.sample(X[0], T))
        errs.append(np.abs(U[0] - Uex[0]).mean())
    assert errs[1] < 0.8 * errs[0], errs
