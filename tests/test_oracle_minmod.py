"""The minmod limiter (reading: Sec. 2.3 names the minmod limiter after van Leer without printing
it; here the minmod bound of Cockburn and Shu on the face deviations, with a TVB threshold
M h^2, applied through one convex factor per element), applied alone as one forward-Euler stage
with dt = 0: it keeps every element mean, leaves linear data untouched on any mesh and degree,
flattens an element holding a strict local extremum, scales a limited element toward its mean
until every face-mean deviation lies within the neighbour-mean differences (the minmod bound),
and with it the paper's strong blasts run admissibly and converge at p = 1."""
import numpy as np
import pytest

import oracle
import workloads as wl


def limit_only(spec, U):
    spec = dict(spec, rk_stages=1, enforce=False, limiter="minmod")
    return oracle.step(spec, U, 0.0, 1)


def weights(spec):
    N = spec["degree"] + 1
    w1 = np.polynomial.legendre.leggauss(N)[1]
    w = w1
    for _ in range(spec["dim"] - 1):
        w = np.multiply.outer(w1, w).ravel()
    return w


def means(spec, U):
    w = weights(spec)
    return (U * w).sum(-1) / w.sum()


def box(dim, n, degree, M=0.0, bc="outflow"):
    return dict(dim=dim, degree=degree, n_elem=[n] * dim, lo=[0.0] * dim, hi=[1.0] * dim,
                eos="ideal", gamma_ad=5.0 / 3.0, c2p="iterative", bc=[(bc, bc)] * dim,
                limiter_alpha=M)


def conserved_from(X, f):
    """An admissible conserved field whose every component is the scalar field f(X) (or a
    positive multiple of it): D = f, S = 0.1 f e_x, tau = 2 f."""
    q = f(X)
    return np.stack([q, 0.1 * q, 0.0 * q, 0.0 * q, 2.0 * q])


@pytest.mark.parametrize("dim,degree", [(1, 1), (1, 3), (2, 1), (2, 2), (3, 1)])
def test_linear_data_untouched(dim, degree):
    """For q linear in x every element has c = a+ = a- = slope dx / 2 and neighbour differences
    slope dx, so minmod keeps a+-: no element is limited, boundaries included."""
    n = 6 if dim == 3 else 10
    spec = box(dim, n, degree)
    X = oracle.node_coords(spec)
    U = conserved_from(X, lambda X: 1.0 + 0.3 * X[0] + (0.2 * X[1] if dim > 1 else 0.0))
    V, st = limit_only(spec, U.copy())
    assert st["limited_cells"] == 0 and np.array_equal(V, U)


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_local_extremum_is_flattened_and_means_kept(degree):
    n = 12
    spec = box(1, n, degree)
    X = oracle.node_coords(spec)
    # a bump centred in element 5: its mean is a strict local maximum of the element means
    U = conserved_from(X, lambda X: 1.0 + np.exp(-((X[0] - 5.5 / n) * n / 0.6) ** 2))
    V, st = limit_only(spec, U.copy())
    assert st["limited_cells"] > 0
    mU, mV = means(spec, U), means(spec, V)
    assert np.allclose(mU, mV, rtol=1e-14, atol=0.0)
    assert mU[0, 5] > mU[0, 4] and mU[0, 5] > mU[0, 6]
    # flattened to its mean: slopes of opposite sign give minmod = 0
    assert np.allclose(V[:, 5], mU[:, 5][:, None], rtol=1e-14, atol=0.0)


def face_mean_devs(spec, U, mU):
    """(a+, a-) per variable and element in 1D: the traces at xi = +-1 minus / from the mean."""
    N = spec["degree"] + 1
    xi = np.polynomial.legendre.leggauss(N)[0]
    ep = np.array([np.prod([(1.0 - xi[k]) / (xi[i] - xi[k]) for k in range(N) if k != i]) for i in range(N)])
    em = np.array([np.prod([(-1.0 - xi[k]) / (xi[i] - xi[k]) for k in range(N) if k != i]) for i in range(N)])
    return U @ ep - mU, mU - U @ em


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_limited_elements_scale_toward_the_mean_within_the_minmod_bound(degree):
    """Seeded data: a limited element is ub + theta (U - ub) with one theta in [0, 1) for all five
    variables, and afterwards every face-mean deviation shares the sign of the neighbour-mean
    differences and is no larger (the minmod bound), so face values lie between neighbour means."""
    n = 40
    spec = box(1, n, degree)
    rng = np.random.default_rng(7)
    X = oracle.node_coords(spec)
    # a smooth wave, a jump and light nodal noise: some elements limited, not all
    U = conserved_from(X, lambda X: 1.5 + 0.3 * np.sin(2.0 * np.pi * X[0]) + 0.5 * (X[0] > 0.51)
                       + 0.002 * rng.standard_normal(X[0].shape))
    U[1] *= np.sign(rng.standard_normal((n, 1)))   # momentum of either sign
    V, st = limit_only(spec, U.copy())
    assert 0 < st["limited_cells"] < n
    mU = means(spec, U)
    assert np.allclose(means(spec, V), mU, rtol=1e-14, atol=1e-15)
    ap, am = face_mean_devs(spec, V, mU)
    for e in range(n):
        if np.array_equal(V[:, e], U[:, e]):
            continue
        d = U[:, e] - mU[:, e][:, None]
        th = ((V[:, e] - mU[:, e][:, None]) * d).sum() / (d * d).sum()
        assert -1e-12 <= th < 1.0
        assert np.allclose(V[:, e], mU[:, e][:, None] + th * d, rtol=0.0, atol=1e-13)
        for v in range(5):
            D = [mU[v, k] - mU[v, e] if k > e else mU[v, e] - mU[v, k]
                 for k in (e - 1, e + 1) if 0 <= k < n]
            for a in (ap[v, e], am[v, e]):
                for Dk in D:
                    assert a * Dk >= -1e-13 and abs(a) <= abs(Dk) + 1e-13


def test_tvb_threshold_keeps_small_deviations():
    """Deviations below M h^2 are kept even at an extremum (the TVB correction), larger ones
    are limited."""
    n = 12
    X = oracle.node_coords(box(1, n, 2))
    U = conserved_from(X, lambda X: 1.0 + 1e-6 * np.cos(2.0 * np.pi * X[0]))
    V, st = limit_only(box(1, n, 2, M=1.0), U.copy())
    assert st["limited_cells"] == 0 and np.array_equal(V, U)
    V, st = limit_only(box(1, n, 2, M=0.0), U.copy())
    assert st["limited_cells"] > 0
    # the threshold scales as h^2: face deviations near 0.03 at the extrema exceed M h^2 = 1/144
    # (limited) although they are below M h = 1/12
    U = conserved_from(X, lambda X: 1.0 + 0.1 * np.cos(2.0 * np.pi * X[0]))
    V, st = limit_only(box(1, n, 2, M=1.0), U.copy())
    assert st["limited_cells"] > 0


@pytest.mark.parametrize("problem", [2, 3, 4])
def test_riemann_problem_converges_with_minmod(problem):
    from tests.test_oracle_riemann import run
    l1 = []
    for n in (64, 128, 256):
        spec = dict(wl.riemann_1d(problem, n=n, degree=1), limiter="minmod", limiter_alpha=0.0)
        X = oracle.node_coords(spec)
        U = oracle.prim2cons(spec, wl.initial_primitive(spec, X))
        U, _, _ = oracle.enforce(spec, U)
        T = spec["t_final"]
        nsteps = int(np.ceil(T / oracle.cfl_dt(spec, spec["cfl"])))
        U, st = oracle.step(spec, U, T / nsteps, nsteps)
        assert st["mean_inadmissible_cells"] == 0 and st["c2p_invalid_input"] == 0
        assert st["limited_cells"] > 0
        from tests.test_oracle_riemann import exact
        Ue = oracle.prim2cons(spec, exact(spec).sample(X[0], T))
        w = np.polynomial.legendre.leggauss(2)[1]
        l1.append(((np.abs(U - Ue) * w).sum(axis=(1, 2)) / (2 * n))[[0, 1, 4]])
    l1 = np.array(l1)
    assert np.all(l1[1:] < 0.9 * l1[:-1]), l1


def test_wall_problem_5_at_p2_runs_and_converges_with_minmod():
    """Riemann problem 5 (gamma = 224 flow into a reflecting wall) at p = 2: the scaling limiter
    loses admissible element means there, the minmod limiter keeps them all and the L1 error
    halves with each refinement."""
    from tests.test_oracle_riemann import exact
    l1 = []
    for n in (64, 128, 256):
        spec = dict(wl.riemann_1d(5, n=n, degree=2), limiter="minmod", limiter_alpha=0.0)
        X = oracle.node_coords(spec)
        U = oracle.prim2cons(spec, wl.initial_primitive(spec, X))
        U, _, _ = oracle.enforce(spec, U)
        T = spec["t_final"]
        nsteps = int(np.ceil(T / oracle.cfl_dt(spec, spec["cfl"])))
        U, st = oracle.step(spec, U, T / nsteps, nsteps)
        assert st["mean_inadmissible_cells"] == 0 and st["c2p_invalid_input"] == 0
        Ue = oracle.prim2cons(spec, exact(spec).sample(X[0], T))
        w = np.polynomial.legendre.leggauss(3)[1]
        l1.append(((np.abs(U - Ue) * w).sum(axis=(1, 2)) / (2 * n))[[0, 1, 4]])
    l1 = np.array(l1)
    assert np.all(l1[1:] < 0.6 * l1[:-1]), l1
