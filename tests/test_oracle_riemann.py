"""The oracle's DG solution of the paper's 1D Riemann problems 2-5 and of its Taub-Matthews blast
wave (Sec. 4.2, HLLC) against the exact Riemann solution: the workloads hold the paper's states,
the L1 error falls with resolution, and HLLC resolves the Sod contact better than HLL.
Problem 5 (a flow into a reflecting wall at x = 1) is the left half of the collision of the
state with its mirror image at x0 = 1.  Problem 3 and the Taub-Matthews blast carry transverse
velocity; their reference is the exact solution with transverse velocity and either EOS."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as wl
from oracle.exact_riemann import ExactRiemann
from oracle.exact_riemann_general import GeneralExactRiemann

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "riemann_problems_2_to_5.json")


def exact(spec):
    L, R, G = spec["left"], spec["right"], spec["gamma_ad"]
    if spec["eos"] != "ideal" or L[2] != 0.0 or R[2] != 0.0:
        return GeneralExactRiemann((L[0], L[1], L[2], L[4]), (R[0], R[1], R[2], R[4]),
                                   spec["eos"], G, 0.5)
    if spec["bc"][0][1] == "reflect":
        return ExactRiemann((L[0], L[1], L[4]), (L[0], -L[1], L[4]), G, 1.0)
    return ExactRiemann((L[0], L[1], L[4]), (R[0], R[1], R[4]), G, 0.5)


def spec_of(problem, n, degree, flux="hllc"):
    if problem in ("tm", "ideal4/3", "ideal5/3"):
        eos, G = {"tm": ("tm", 4.0 / 3.0), "ideal4/3": ("ideal", 4.0 / 3.0),
                  "ideal5/3": ("ideal", 5.0 / 3.0)}[problem]
        return wl.tm_blast(eos, G, n=n, degree=degree, flux=flux)
    return wl.riemann_1d(problem, n=n, degree=degree, flux=flux)


def run(problem, n, degree, flux="hllc", limiter=False):
    spec = dict(spec_of(problem, n, degree, flux), limiter=limiter)
    X = oracle.node_coords(spec)
    U = oracle.prim2cons(spec, wl.initial_primitive(spec, X))
    U, _, _ = oracle.enforce(spec, U)
    T = spec["t_final"]
    nsteps = int(np.ceil(T / oracle.cfl_dt(spec, spec["cfl"])))
    U, st = oracle.step(spec, U, T / nsteps, nsteps)
    Uex = oracle.prim2cons(spec, exact(spec).sample(X[0], T))
    w = np.polynomial.legendre.leggauss(degree + 1)[1]
    l1 = (np.abs(U - Uex) * w).sum(axis=(1, 2)) / (2 * n)
    return l1, st


def test_workloads_hold_the_paper_problems():
    g = json.load(open(GOLDEN))["problems"]
    for k, P in g.items():
        spec = wl.riemann_1d(int(k))
        L, R = spec["left"], spec["right"]
        assert [L[0], L[1], L[2], L[4]] == P["left"] and [R[0], R[1], R[2], R[4]] == P["right"]
        assert spec["gamma_ad"] == P["gamma_ad"] and spec["t_final"] == P["t_final"]
        assert (spec["bc"][0][1] == "reflect") == (P["right_boundary"] == "reflecting")


# Problems 2 and 5 run at p = 0: at p >= 1 the paper adds a slope limiter (Moe et al.), which
# the method as built here does not have, and without it the element means of these two strong
# blasts leave the admissible set within a few steps at every flux.
# Problem 2's blast shell is a thin dense spike; at p = 0 its density error only settles into
# a steady decrease from 128 cells on (the paper notes the same difficulty at basis order 0).
@pytest.mark.parametrize("problem,degree,n0,ratio", [(2, 0, 128, 0.9), (4, 1, 64, 0.85),
                                                     (5, 0, 64, 0.85)])
def test_riemann_problem_converges_with_hllc(problem, degree, n0, ratio):
    l1a, st = run(problem, n0, degree)
    l1b, _ = run(problem, 2 * n0, degree)
    l1c, _ = run(problem, 4 * n0, degree)
    assert st["c2p_invalid_input"] == 0 and st["mean_inadmissible_cells"] == 0
    assert st["c2p_nonconverged"] == 0
    k = [0, 1, 4]  # D, S_x, tau
    assert np.all(l1b[k] < ratio * l1a[k]) and np.all(l1c[k] < ratio * l1b[k]), (l1a, l1b, l1c)


def test_hllc_resolves_the_sod_contact_better_than_hll():
    l1c, _ = run(4, 128, 1, flux="hllc")
    l1h, _ = run(4, 128, 1, flux="hll")
    assert l1c[0] < l1h[0], (l1c[0], l1h[0])


@pytest.mark.parametrize("problem", [2, 4, 5])
def test_riemann_problem_with_the_limiter_at_p1(problem):
    """With the scaling limiter (reading for the paper's Moe limiter) the blasts run at p = 1:
    admissible means throughout and errors falling with resolution."""
    l1a, st = run(problem, 64, 1, limiter=True)
    l1b, _ = run(problem, 128, 1, limiter=True)
    l1c, _ = run(problem, 256, 1, limiter=True)
    assert st["mean_inadmissible_cells"] == 0 and st["c2p_invalid_input"] == 0
    assert st["limited_cells"] > 0
    k = [0, 1, 4]
    assert np.all(l1b[k] < 0.9 * l1a[k]) and np.all(l1c[k] < 0.9 * l1b[k]), (l1a, l1b, l1c)


def test_tm_blast_workload_holds_the_paper_states():
    g = json.load(open(os.path.join(os.path.dirname(GOLDEN), "tm_blast_wave.json")))
    spec = wl.tm_blast()
    L, R = spec["left"], spec["right"]
    assert [L[0], L[1], L[2], L[4]] == g["left"] and [R[0], R[1], R[2], R[4]] == g["right"]
    assert spec["t_final"] == g["t_final"] and L[3] == R[3] == 0.0


@pytest.mark.parametrize("problem", [3, "tm", "ideal4/3", "ideal5/3"])
@pytest.mark.parametrize("degree,limiter,n0", [(0, False, 128), (1, True, 64)])
def test_transverse_velocity_blasts_converge(problem, degree, limiter, n0):
    """Riemann problem 3 and the Taub-Matthews blast with the three EOS of Fig. 9: admissible
    throughout, and the L1 error of every conserved component falls with each refinement."""
    l1 = []
    for n in (n0, 2 * n0, 4 * n0):
        e, st = run(problem, n, degree, limiter=limiter)
        assert st["mean_inadmissible_cells"] == 0 and st["c2p_invalid_input"] == 0
        assert st["c2p_nonconverged"] == 0
        l1.append(e[[0, 1, 2, 4]])
    l1 = np.array(l1)
    assert np.all(l1[1:] < 0.9 * l1[:-1]), l1
