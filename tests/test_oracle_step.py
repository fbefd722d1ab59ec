"""Pins for the oracle's time integration (SSP-RK, Shu-Osher form) and its full solution on
smooth problems: the RK stability polynomial on a linearised problem, and order p + 1
convergence on the advected density wave against the exact translated solution."""
import math

import numpy as np
import pytest

import oracle
import workloads as wl


@pytest.mark.parametrize("stages", [1, 2, 3])
def test_rk_stability_polynomial(stages):
    """Near a uniform state R is linear, R(U0 + eps V) = eps J V + O(eps^2).  One step must then
    equal U0 + eps P(dt J) V with P(z) = sum_{k <= stages} z^k / k!, the stability polynomial
    of RK1 / SSPRK2 / SSPRK3."""
    spec = wl.smooth_random(1, [5], 1, seed=3, rk_stages=stages)
    spec["enforce"] = False
    E, Nn = oracle.shape(spec)
    U0 = oracle.prim2cons(spec, np.broadcast_to(np.array([1.0, 0.3, 0.1, 0.0, 0.8])[:, None, None],
                                                (5, E, Nn)).copy())
    n = U0.size
    eps = 1e-6
    J = np.zeros((n, n))
    for j in range(n):
        dU = np.zeros(n)
        dU[j] = eps
        Rp, _ = oracle.rhs(spec, U0 + dU.reshape(U0.shape))
        Rm, _ = oracle.rhs(spec, U0 - dU.reshape(U0.shape))
        J[:, j] = (Rp - Rm).ravel() / (2 * eps)
    dt = oracle.cfl_dt(spec, 0.2)
    V = np.random.default_rng(1).normal(size=n)
    Z = dt * J
    P = np.eye(n)
    term = np.eye(n)
    for k in range(1, stages + 1):
        term = term @ Z / k
        P = P + term
    amp = 1e-7
    U1, _ = oracle.step(spec, U0 + amp * V.reshape(U0.shape), dt, 1)
    got = (U1 - U0).ravel() / amp
    want = P @ V
    assert np.linalg.norm(got - want) < 1e-5 * np.linalg.norm(want)
    # a different polynomial would be far away
    assert np.linalg.norm(term) * np.linalg.norm(V) > 1e-4 * np.linalg.norm(want)


def test_cfl_rule():
    spec = wl.blast_wave(n=128, degree=1)
    assert abs(oracle.cfl_dt(spec, 0.2) - 0.2 / (3 * 128)) < 1e-18
    spec = wl.advected_wave(n=10, degree=3)
    assert abs(oracle.cfl_dt(spec, 0.2) - 0.2 / (7 * 20)) < 1e-18


def l1_density_error(spec, U, t):
    X = oracle.node_coords(spec)
    W, _, _ = oracle.con2prim(spec, U)
    ex = wl.advected_wave_ic(spec, X, t)
    N = spec["degree"] + 1
    w = np.polynomial.legendre.leggauss(N)[1]
    w2 = np.multiply.outer(w, w).ravel()
    return float((np.abs(W[0] - ex[0]) * w2).sum() / (w2.sum() * X.shape[1]))


@pytest.mark.parametrize("degree,ns", [(1, [8, 16, 32]), (2, [16, 32]), (3, [6, 12])])
def test_advected_wave_converges_at_order_p_plus_1(degree, ns):
    errs = []
    T = 0.1
    for n in ns:
        spec = wl.advected_wave(n=n, degree=degree, c2p="iterative")
        X = oracle.node_coords(spec)
        U = oracle.prim2cons(spec, wl.advected_wave_ic(spec, X))
        dt = oracle.cfl_dt(spec, 0.2)
        nsteps = math.ceil(T / dt)
        U, st = oracle.step(spec, U, T / nsteps, nsteps)
        assert st["enforced_cells"] == 0
        errs.append(l1_density_error(spec, U, T))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > degree + 1 - 0.25), (errs, orders)
