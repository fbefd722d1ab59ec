"""Pins for the exact 1D SRHD Riemann solution (test infrastructure for the blast wave of
Sec. 4.2): jump conditions at the shock, self-similar rarefaction, and the integral
conservation law that every wave of the solution must satisfy together."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import oracle
from oracle.exact_riemann import ExactRiemann

PROBLEMS = [
    ((10.0, 0.0, 13.33), (1.0, 0.0, 1e-6), 5.0 / 3.0),          # blast wave (problem 1)
    ((1.0, 0.0, 1e3), (1.0, 0.0, 1e-2), 5.0 / 3.0),             # strong blast (problem 2)
    ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 5.0 / 3.0),            # Sod-like
    ((1.0, 0.3, 1.0), (1.0, -0.3, 1.0), 4.0 / 3.0),             # two shocks
    ((1.0, -0.5, 1.0), (1.0, 0.5, 1.0), 4.0 / 3.0),             # two rarefactions
]


def cons(G, rho, v, p):
    W = 1.0 / math.sqrt(1.0 - v * v)
    h = 1.0 + G / (G - 1.0) * p / rho
    return np.array([W * rho, W * W * rho * h * v, W * W * rho * h - p - W * rho])


def flux(G, rho, v, p):
    U = cons(G, rho, v, p)
    return np.array([U[0] * v, U[1] * v + p, (U[2] + p) * v])


@pytest.mark.parametrize("L,R,G", PROBLEMS)
def test_shock_jump_conditions(L, R, G):
    ex = ExactRiemann(L, R, G)
    for state, rho_s, Vs in ((ex.L, ex.rho_Ls, ex.Vs_L), (ex.R, ex.rho_Rs, ex.Vs_R)):
        if Vs is None:
            continue
        a = cons(G, *state)
        b = cons(G, rho_s, ex.v_star, ex.p_star)
        res = (flux(G, rho_s, ex.v_star, ex.p_star) - flux(G, *state)) - Vs * (b - a)
        assert np.all(np.abs(res) < 1e-12 * (np.abs(a) + np.abs(b) + 1.0))
        assert abs(Vs) < 1.0


@pytest.mark.parametrize("L,R,G", PROBLEMS)
def test_integral_conservation(L, R, G):
    """d/dt int U dx = F(U_L) - F(U_R) for the self-similar solution: over xi in [-1, 1],
    int U dxi = U_L + U_R + F_L - F_R."""
    ex = ExactRiemann(L, R, G)
    cuts = [-1.0, ex.v_star, 1.0]
    if ex.Vs_L is not None:
        cuts.append(ex.Vs_L)
    else:
        cuts += [ex._lambda(*ex.L, -1), ex._lambda(ex.rho_Ls, ex.v_star, ex.p_star, -1)]
    if ex.Vs_R is not None:
        cuts.append(ex.Vs_R)
    else:
        cuts += [ex._lambda(*ex.R, +1), ex._lambda(ex.rho_Rs, ex.v_star, ex.p_star, +1)]
    cuts = sorted(cuts)
    total = np.zeros(3)
    for a, b in zip(cuts, cuts[1:]):
        for k in range(3):
            total[k] += quad(lambda xi: cons(G, *ex.sample_xi(xi))[k], a, b,
                             epsabs=1e-13, epsrel=1e-12, limit=200)[0]
    want = cons(G, *ex.L) + cons(G, *ex.R) + flux(G, *ex.L) - flux(G, *ex.R)
    assert np.all(np.abs(total - want) < 1e-9 * (1.0 + np.abs(want)))


def test_rarefaction_fan_is_self_similar_and_isentropic():
    L, R, G = PROBLEMS[0]
    ex = ExactRiemann(L, R, G)
    spec = dict(dim=1, degree=0, n_elem=[1], eos="ideal", gamma_ad=G)
    head = ex._lambda(*ex.L, -1)
    tail = ex._lambda(ex.rho_Ls, ex.v_star, ex.p_star, -1)
    K = ex.L[2] / ex.L[0] ** G
    for xi in np.linspace(head, tail, 12)[1:-1]:
        rho, v, p = ex.sample_xi(xi)
        lm, _ = oracle.wavespeeds(spec, np.array([rho, v, 0.0, 0.0, p]), 0)
        assert abs(lm - xi) < 1e-11
        assert abs(p / rho ** G - K) < 1e-11 * K
