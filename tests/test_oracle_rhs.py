"""Pins for the oracle's DG right-hand side (Sec. 2.3): free stream, the p = 0 finite-volume
special case, conservation, and symmetries that catch sign, index and transposition slips."""
import numpy as np
import pytest

import oracle
import workloads as wl


def uniform_state(spec, W0):
    E, Nn = oracle.shape(spec)
    W = np.broadcast_to(np.asarray(W0, dtype=float)[:, None, None], (5, E, Nn)).copy()
    return oracle.prim2cons(spec, W)


@pytest.mark.parametrize("dim,n", [(1, [5]), (2, [3, 4]), (3, [2, 3, 2])])
@pytest.mark.parametrize("degree", [0, 1, 2, 3])
@pytest.mark.parametrize("eos", ["ideal", "tm"])
def test_free_stream(dim, n, degree, eos):
    spec = wl.smooth_random(dim, n, degree, eos=eos)
    U = uniform_state(spec, [1.3, 0.3, -0.4, 0.2, 0.7])
    R, st = oracle.rhs(spec, U)
    assert np.abs(R).max() < 1e-12 * np.abs(U).max() * max(n)
    assert st["c2p_invalid_input"] == 0


def fv_rhs(spec, U):
    """First-order finite volume: R_e = -sum_d (F*_{e+1/2} - F*_{e-1/2}) / dx_d with the
    oracle's numerical flux on cell values (the p = 0 reduction of Sec. 2.3)."""
    W, _, _ = oracle.con2prim(spec, U)
    W = W[:, :, 0]
    dim = spec["dim"]
    n = spec["n_elem"][:dim] + [1] * (3 - dim)
    dx = [(spec["hi"][d] - spec["lo"][d]) / n[d] for d in range(dim)]
    R = np.zeros((5, W.shape[1]))

    def idx(c):
        return c[0] + n[0] * (c[1] + n[1] * c[2])

    for e in range(W.shape[1]):
        c = [e % n[0], (e // n[0]) % n[1], e // (n[0] * n[1])]
        for d in range(dim):
            def neighbour(off):
                cc = list(c)
                cc[d] += off
                if 0 <= cc[d] < n[d]:
                    return W[:, idx(cc)]
                side = 0 if off < 0 else 1
                kind = spec["bc"][d][side]
                if kind == "periodic":
                    cc[d] %= n[d]
                    return W[:, idx(cc)]
                if kind == "dirichlet":
                    return np.array(spec["bc_state"][d][side], dtype=float)
                return W[:, e]
            Fr = oracle.numerical_flux(spec, W[:, e], neighbour(+1), d)
            Fl = oracle.numerical_flux(spec, neighbour(-1), W[:, e], d)
            R[:, e] -= (Fr - Fl) / dx[d]
    return R


@pytest.mark.parametrize("dim,n,bc", [
    (1, [7], [("periodic", "periodic")]),
    (1, [6], [("dirichlet", "outflow")]),
    (2, [4, 3], [("periodic", "periodic"), ("outflow", "dirichlet")]),
    (3, [3, 2, 2], [("periodic", "periodic")] * 3)])
@pytest.mark.parametrize("flux", ["llf", "hll"])
def test_p0_is_first_order_finite_volume(dim, n, bc, flux):
    spec = wl.smooth_random(dim, n, 0, flux=flux, seed=4, bc=bc)
    X = oracle.node_coords(spec)
    U = oracle.prim2cons(spec, wl.smooth_random_ic(spec, X))
    R, _ = oracle.rhs(spec, U)
    Rfv = fv_rhs(spec, U)
    assert np.allclose(R[:, :, 0], Rfv, rtol=1e-12, atol=1e-12 * np.abs(Rfv).max())


def weights(spec):
    b = oracle.basis(spec["degree"] + 1)
    w = b["w"]
    out = w
    for _ in range(spec["dim"] - 1):
        out = np.multiply.outer(w, out).ravel()  # node index x-fastest
    return out


@pytest.mark.parametrize("dim,n", [(1, [6]), (2, [4, 5]), (3, [3, 3, 2])])
@pytest.mark.parametrize("degree", [1, 2, 3])
@pytest.mark.parametrize("eos,flux", [("ideal", "llf"), ("tm", "hll")])
def test_periodic_conservation(dim, n, degree, eos, flux):
    """sum_e sum_i w_i R_i = 0 on a periodic mesh: every lifted face flux enters its two
    neighbours with opposite signs."""
    spec = wl.smooth_random(dim, n, degree, eos=eos, flux=flux, seed=degree)
    X = oracle.node_coords(spec)
    U = oracle.prim2cons(spec, wl.smooth_random_ic(spec, X))
    R, _ = oracle.rhs(spec, U)
    w = weights(spec)
    tot = (R * w[None, None, :]).sum(axis=(1, 2))
    scale = (np.abs(R) * w[None, None, :]).sum(axis=(1, 2))
    assert np.all(np.abs(tot) < 1e-13 * scale)


@pytest.mark.parametrize("degree", [1, 3])
def test_2d_state_varying_in_x_matches_1d(degree):
    s1 = wl.smooth_random(1, [6], degree, seed=9)
    s2 = wl.smooth_random(2, [6, 3], degree, seed=9)
    s2["hi"] = [1.0, 0.7]
    X1 = oracle.node_coords(s1)
    W1 = wl.smooth_random_ic(s1, X1)
    N = degree + 1
    # 2D field: the 1D field repeated along y, node index a + N b
    W2 = np.empty((5, 18, N * N))
    for e in range(18):
        ex = e % 6
        for b in range(N):
            W2[:, e, b * N:(b + 1) * N] = W1[:, ex, :]
    R1, _ = oracle.rhs(s1, oracle.prim2cons(s1, W1))
    R2, _ = oracle.rhs(s2, oracle.prim2cons(s2, W2))
    for e in range(18):
        for b in range(N):
            assert np.allclose(R2[:, e, b * N:(b + 1) * N], R1[:, e % 6, :], rtol=1e-12,
                               atol=1e-11 * np.abs(R1).max())


@pytest.mark.parametrize("degree", [1, 2])
def test_2d_axis_exchange(degree):
    """Swapping x and y in the state (and v_x with v_y) swaps them in R."""
    spec = wl.smooth_random(2, [4, 4], degree, seed=13)
    X = oracle.node_coords(spec)
    W = wl.smooth_random_ic(spec, X)
    N = degree + 1

    def transpose(A):
        B = A.reshape(A.shape[0], 4, 4, N, N)       # [v][ey][ex][b][a]
        return B.transpose(0, 2, 1, 4, 3).reshape(A.shape)

    Wt = transpose(W)[[0, 2, 1, 3, 4]]
    R, _ = oracle.rhs(spec, oracle.prim2cons(spec, W))
    Rt, _ = oracle.rhs(spec, oracle.prim2cons(spec, Wt))
    assert np.allclose(transpose(R)[[0, 2, 1, 3, 4]], Rt, rtol=1e-12, atol=1e-11 * np.abs(R).max())


@pytest.mark.parametrize("degree", [0, 1, 3])
def test_1d_mirror_symmetry(degree):
    """x -> 1 - x with v_x -> -v_x maps R to its mirror image with S_x negated."""
    spec = wl.smooth_random(1, [8], degree, seed=17)
    X = oracle.node_coords(spec)
    W = wl.smooth_random_ic(spec, X)
    Wm = W[:, ::-1, ::-1].copy()
    Wm[1] *= -1
    R, _ = oracle.rhs(spec, oracle.prim2cons(spec, W))
    Rm, _ = oracle.rhs(spec, oracle.prim2cons(spec, Wm))
    Rmm = Rm[:, ::-1, ::-1].copy()
    Rmm[1] *= -1
    assert np.allclose(R, Rmm, rtol=1e-12, atol=1e-11 * np.abs(R).max())
