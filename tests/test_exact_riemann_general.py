"""Pins for the exact 1D SRHD Riemann solution with transverse velocity and the Taub-Matthews
EOS (test infrastructure for Riemann problem 3 and the Taub-Matthews blast wave of Sec. 4.3):
agreement with the independent solver without transverse velocity, the rarefaction ODE against
the acoustic eigenvectors of the system's own Jacobian, the Rankine-Hugoniot conditions at
every shock, the integral conservation law of the whole self-similar solution, the simple-wave
invariants inside fans, and the paper's reading of its Taub-Matthews blast (Fig. 9)."""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad

import oracle
from oracle.exact_riemann import ExactRiemann
from oracle.exact_riemann_general import GeneralExactRiemann

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tm_blast_wave.json")

NO_TRANSVERSE = [
    ((10.0, 0.0, 13.33), (1.0, 0.0, 1e-6), 5.0 / 3.0),
    ((1.0, 0.0, 1e3), (1.0, 0.0, 1e-2), 5.0 / 3.0),
    ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 5.0 / 3.0),
    ((1.0, 0.3, 1.0), (1.0, -0.3, 1.0), 4.0 / 3.0),
    ((1.0, -0.5, 1.0), (1.0, 0.5, 1.0), 4.0 / 3.0),
]

# (left, right, eos, Gamma): primitive (rho, v_x, v_t, P)
TRANSVERSE = [
    ((1.0, 0.0, 0.0, 1e3), (1.0, 0.0, 0.99, 1e-2), "ideal", 5.0 / 3.0),   # problem 3
    ((1.0, 0.0, 0.9, 1e3), (1.0, 0.0, 0.99, 1e-2), "tm", 5.0 / 3.0),      # TM blast, three EOS
    ((1.0, 0.0, 0.9, 1e3), (1.0, 0.0, 0.99, 1e-2), "ideal", 4.0 / 3.0),
    ((1.0, 0.0, 0.9, 1e3), (1.0, 0.0, 0.99, 1e-2), "ideal", 5.0 / 3.0),
    ((1.0, 0.3, 0.5, 1.0), (0.5, -0.3, -0.4, 2.0), "tm", 5.0 / 3.0),       # two shocks
    ((1.0, -0.5, 0.6, 1.0), (1.0, 0.4, 0.2, 0.5), "ideal", 4.0 / 3.0),    # two rarefactions
    ((1.0, 0.0, 0.5, 1.0), (0.125, 0.0, -0.5, 0.1), "tm", 5.0 / 3.0),     # Sod-like
]


def ids(cases):
    return [f"case{k}" for k in range(len(cases))]


def U_of(ex, W):
    rho, vx, vt, p = W
    return ex.cons(ex.to_u(W))


def F_of(ex, W):
    return ex.flux(ex.to_u(W))


def cuts(ex):
    c = [-1.0, ex.v_star, 1.0]
    for sign, Vs in ((-1, ex.Vs_L), (+1, ex.Vs_R)):
        c += [Vs] if Vs is not None else list(ex.fan_edges(sign))
    return sorted(c)


@pytest.mark.parametrize("L,R,G", NO_TRANSVERSE, ids=ids(NO_TRANSVERSE))
def test_reduces_to_the_solution_without_transverse_velocity(L, R, G):
    """Two different constructions (rapidity quadrature and the closed-form Taub adiabat, against
    the integrated simple-wave ODE and a root-found adiabat) give the same solution."""
    a = GeneralExactRiemann((L[0], L[1], 0.0, L[2]), (R[0], R[1], 0.0, R[2]), "ideal", G)
    b = ExactRiemann(L, R, G)
    assert abs(a.p_star / b.p_star - 1.0) < 1e-11
    assert abs(a.v_star - b.v_star) < 1e-12
    assert abs(a.WLs[0] / b.rho_Ls - 1.0) < 1e-11 and abs(a.WRs[0] / b.rho_Rs - 1.0) < 1e-11
    for x, y in ((a.Vs_L, b.Vs_L), (a.Vs_R, b.Vs_R)):
        assert (x is None) == (y is None)
        if x is not None:
            assert abs(x - y) < 1e-12
    x = np.linspace(0.0, 1.0, 101)
    A, B = a.sample(x, 0.4), b.sample(x, 0.4)
    assert np.all(np.abs(A - B) <= 1e-8 * (1.0 + np.abs(B)))
    assert np.all(A[2] == 0.0)


STATES = [(1.0, 0.3, 0.5, 1.0), (0.2, -0.4, 0.7, 0.05), (3.0, 0.1, -0.2, 10.0),
          (1.0, 0.6, 0.6, 0.5), (1.0, 0.9, 0.3, 100.0), (1.0, 0.0, 0.99, 0.01)]


@pytest.mark.parametrize("eos,G", [("ideal", 5.0 / 3.0), ("ideal", 4.0 / 3.0), ("tm", 5.0 / 3.0)])
def test_rarefaction_ode_is_the_acoustic_eigenvector(eos, G):
    """The closed forms the solver integrates (lambda-+, drho/dP = 1/(h c^2), dv_x/dP, h u_t
    constant) against the acoustic eigenpair of A = (dU/dY)^-1 dF/dY taken numerically from the
    definitions of U and F; c_s^2 also against the oracle's EOS (Sec. 2.2)."""
    ex = GeneralExactRiemann((1.0, 0.0, 0.0, 1.0), (1.0, 0.0, 0.0, 0.5), eos, G)
    spec = dict(dim=1, degree=0, n_elem=[1], eos=eos, gamma_ad=G)
    for W in STATES:
        rho, vx, vt, p = W
        assert abs(ex.cs2(rho, p) / oracle.cs2(spec, rho, p) - 1.0) < 1e-13
        assert abs(ex.h(rho, p) / oracle.enthalpy(spec, rho, p) - 1.0) < 1e-14
        Y = ex.to_u(W)
        lor = math.sqrt(1.0 + Y[1] ** 2 + Y[2] ** 2)
        h, c2 = ex.h(rho, p), ex.cs2(rho, p)
        for sign in (-1, +1):
            lam, r = ex.acoustic(Y, sign)
            assert abs(lam - ex.lam_closed(W, sign)) < 1e-13
            lm, lp = oracle.wavespeeds(spec, np.array([rho, vx, vt, 0.0, p]), 0)
            assert abs(lam - (lm if sign < 0 else lp)) < 1e-13
            assert abs(r[0] * h * c2 - 1.0) < 1e-12                   # isentrope
            dlor = (Y[1] * r[1] + Y[2] * r[2]) / lor
            dvx = (r[1] - vx * dlor) / lor
            want = sign * math.sqrt(1.0 - vx * vx - c2 * vt * vt) / (rho * h * lor * math.sqrt(c2))
            assert abs(dvx / want - 1.0) < 1e-11
            # d(h u_t) = h_rho drho + h_P dP times u_t plus h du_t: zero along the wave
            e = 1e-30
            dh = ex.h(rho + 1j * e, p).imag / e * r[0] + ex.h(rho, p + 1j * e).imag / e
            assert abs(dh * Y[2] + h * r[2]) < 1e-12 * (abs(dh * Y[2]) + abs(h * r[2]) + 1e-300) + 1e-15


@pytest.mark.parametrize("L,R,eos,G", TRANSVERSE, ids=ids(TRANSVERSE))
def test_shock_jump_conditions(L, R, eos, G):
    """[F] = V_s [U] in all four components at every shock, |V_s| < 1."""
    ex = GeneralExactRiemann(L, R, eos, G)
    for state, star, Vs in ((ex.L, ex.WLs, ex.Vs_L), (ex.R, ex.WRs, ex.Vs_R)):
        if Vs is None:
            continue
        a, b = U_of(ex, state), U_of(ex, star)
        res = (F_of(ex, star) - F_of(ex, state)) - Vs * (b - a)
        assert np.all(np.abs(res) < 1e-12 * (np.abs(a) + np.abs(b) + 1.0)), res
        assert abs(Vs) < 1.0


@pytest.mark.parametrize("L,R,eos,G", TRANSVERSE, ids=ids(TRANSVERSE))
def test_integral_conservation(L, R, eos, G):
    """Over xi in [-1, 1] the self-similar solution holds int U dxi = U_L + U_R + F_L - F_R
    (all four components), which fails if any wave or the middle state is wrong."""
    ex = GeneralExactRiemann(L, R, eos, G)
    c = cuts(ex)
    total = np.zeros(4)
    for a, b in zip(c, c[1:]):
        for k in range(4):
            total[k] += quad(lambda xi: U_of(ex, ex.sample_xi(xi))[k], a, b,
                             epsabs=1e-13, epsrel=1e-12, limit=200)[0]
    want = U_of(ex, ex.L) + U_of(ex, ex.R) + F_of(ex, ex.L) - F_of(ex, ex.R)
    assert np.all(np.abs(total - want) < 1e-8 * (1.0 + np.abs(want))), (total, want)


@pytest.mark.parametrize("L,R,eos,G", TRANSVERSE, ids=ids(TRANSVERSE))
def test_fans_are_self_similar_isentropic_with_h_u_t_constant(L, R, eos, G):
    ex = GeneralExactRiemann(L, R, eos, G)
    for sign, state in ((-1, ex.L), (+1, ex.R)):
        edges = ex.fan_edges(sign)
        if edges is None:
            continue
        hu_a = ex.h(state[0], state[3]) * ex.to_u(state)[2]
        h_a = ex.h(state[0], state[3])
        lo, hi = sorted(edges)
        for xi in np.linspace(lo, hi, 9)[1:-1]:
            W = ex.sample_xi(xi)
            assert abs(ex.lam(W, sign) - xi) < 1e-11                    # x/t = lambda
            assert abs(ex.h(W[0], W[3]) * ex.to_u(W)[2] - hu_a) < 1e-11 * (1.0 + abs(hu_a))
            # isentrope: h - h_a = int_{P_a}^{P} dP / rho
            integral = quad(lambda q: 1.0 / ex._rarefaction(state, q, sign)[0], state[3], W[3],
                            epsabs=1e-14, epsrel=1e-12, limit=200)[0]
            assert abs(ex.h(W[0], W[3]) - h_a - integral) < 1e-10 * h_a


def test_paper_reading_of_the_taub_matthews_blast():
    """Fig. 9 (Sec. 4.3): the Taub-Matthews blast runs slightly ahead of both ideal gases, and
    its transverse velocity behind the blast is the lowest of the three."""
    g = json.load(open(GOLDEN))
    L, R = g["left"], g["right"]
    sol = {k: GeneralExactRiemann((L[0], L[1], L[2], L[3]), (R[0], R[1], R[2], R[3]), eos, G)
           for k, (eos, G) in {"tm": ("tm", 5.0 / 3.0), "4/3": ("ideal", 4.0 / 3.0),
                               "5/3": ("ideal", 5.0 / 3.0)}.items()}
    for s in sol.values():
        assert s.Vs_L is None and s.Vs_R is not None            # rarefaction left, shock right
    assert sol["tm"].Vs_R > sol["4/3"].Vs_R > sol["5/3"].Vs_R
    x = np.linspace(0.0, 1.0, 2001)
    umin = {k: (s.sample(x, g["t_final"])[2] / np.sqrt(1.0 - (s.sample(x, g["t_final"])[1:4] ** 2)
                                                      .sum(axis=0))).min()
            for k, s in sol.items()}
    assert umin["tm"] < umin["4/3"] and umin["tm"] < umin["5/3"]
