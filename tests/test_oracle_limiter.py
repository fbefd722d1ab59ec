"""The scaling limiter (reading: a limiter of the Moe et al. kind, which the paper uses for
p >= 1 without printing it), applied alone as one forward-Euler stage with dt = 0: it keeps
every element mean, leaves resolved smooth data untouched, and brings the nodal values of a
discontinuity inside the neighbour-mean bounds; with it the paper's blast waves run at p = 1."""
import numpy as np
import pytest

import oracle
import workloads as wl


def limit_only(spec, U):
    spec = dict(spec, rk_stages=1, enforce=False, limiter=True)
    return oracle.step(spec, U, 0.0, 1)


def means(spec, U):
    N = spec["degree"] + 1
    w1 = np.polynomial.legendre.leggauss(N)[1]
    w = w1
    for _ in range(spec["dim"] - 1):
        w = np.multiply.outer(w1, w).ravel()
    return (U * w).sum(-1) / w.sum()


def test_limiter_keeps_means_and_smooth_data():
    spec = dict(wl.advected_wave(n=32, degree=3), limiter_alpha=50.0)
    U = oracle.prim2cons(spec, wl.initial_primitive(spec, oracle.node_coords(spec)))
    V, st = limit_only(spec, U.copy())
    assert st["limited_cells"] == 0 and np.array_equal(V, U)


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_limiter_bounds_a_discontinuity_and_keeps_means(degree):
    n = 40
    spec = dict(dim=1, degree=degree, n_elem=[n], lo=[0.0], hi=[1.0], eos="ideal",
                gamma_ad=5.0 / 3.0, c2p="iterative", bc=[("outflow", "outflow")],
                limiter_alpha=1.0)
    X = oracle.node_coords(spec)
    x = X[0]
    W = np.stack([np.where(x < 0.43, 10.0, 1.0), 0.0 * x, 0.0 * x, 0.0 * x,
                  np.where(x < 0.43, 13.0, 0.1)])
    U = oracle.prim2cons(spec, W)
    # oscillating nodal values around the jump (every variable of a node scaled by one factor,
    # which keeps the state admissible)
    U = U * (1.0 + 0.3 * np.sin(37.0 * x) * (np.abs(x - 0.43) < 0.03))[None]
    V, st = limit_only(spec, U.copy())
    assert st["limited_cells"] > 0
    mU, mV = means(spec, U), means(spec, V)
    assert np.allclose(mU, mV, rtol=1e-15, atol=1e-15 * np.abs(mU).max())
    alpha = 1.0 * (1.0 / n) ** 1.5
    for e in range(n):
        for v in range(5):
            nb = [mU[v, e]] + [mU[v, k] for k in (e - 1, e + 1) if 0 <= k < n]
            assert V[v, e].max() <= max(nb) + alpha + 1e-12 * abs(max(nb))
            assert V[v, e].min() >= min(nb) - alpha - 1e-12 * abs(min(nb))
    # the factor is the largest that keeps the bounds: in a limited element some variable's
    # extreme over the nodes and the two face traces (phi_i(-1), phi_i(+1) from the Lagrange
    # basis on the Gauss-Legendre nodes) lands on its relaxed bound
    xg = np.polynomial.legendre.leggauss(degree + 1)[0]
    lag = [np.polynomial.Polynomial.fromroots(np.delete(xg, i)) for i in range(degree + 1)]
    em = np.array([p(-1.0) / p(xg[i]) for i, p in enumerate(lag)])
    ep = np.array([p(1.0) / p(xg[i]) for i, p in enumerate(lag)])
    limited = [e for e in range(n) if not np.array_equal(V[:, e], U[:, e])]
    assert len(limited) == st["limited_cells"]
    for e in limited:
        touches = False
        for v in range(5):
            nb = [mU[v, e]] + [mU[v, k] for k in (e - 1, e + 1) if 0 <= k < n]
            vals = np.concatenate([V[v, e], [em @ V[v, e], ep @ V[v, e]]])
            tol = 1e-12 * max(abs(max(nb)), abs(min(nb)), alpha)
            touches |= abs(vals.max() - (max(nb) + alpha)) <= tol
            touches |= abs(vals.min() - (min(nb) - alpha)) <= tol
        assert touches, f"element {e} is limited further than its bounds require"
