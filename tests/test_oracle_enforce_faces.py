"""Pins for the face-point variant of the oracle's physicality operator (Sec. 2.5 applied to the
element's nodes and to the face points of its conserved polynomial, enforce = "faces").

The face values are formed here independently of the oracle: Gauss-Legendre nodes from numpy,
the Lagrange basis evaluated at -1 and +1 by numpy's polynomial fit of the cardinal functions,
and the tensor-product lines of the node layout (x fastest)."""
import numpy as np
import pytest

import oracle
import workloads as wl


def q_stable(U):
    S2 = U[1] ** 2 + U[2] ** 2 + U[3] ** 2
    return U[4] - S2 / (U[0] + np.sqrt(U[0] ** 2 + S2))


def admissible(U):
    return (U[0] > 0) & (q_stable(U) > 0)


def end_values(N):
    """phi_i(-1), phi_i(+1) of the Lagrange basis on the N Gauss-Legendre nodes."""
    x = np.polynomial.legendre.leggauss(N)[0]
    em, ep = np.empty(N), np.empty(N)
    for i in range(N):
        c = np.polynomial.polynomial.polyfit(x, np.eye(N)[i], N - 1)
        em[i] = np.polynomial.polynomial.polyval(-1.0, c)
        ep[i] = np.polynomial.polynomial.polyval(1.0, c)
    return em, ep


def face_values(U, N, dim):
    """Conserved polynomial of every element at its 2 dim N^(dim-1) face points:
    shape (5, E, 2 dim N^(dim-1))."""
    em, ep = end_values(N)
    E = U.shape[1]
    V = U.reshape((5, E) + (N,) * dim)  # axes (..., z, y, x): x fastest
    out = []
    for d in range(dim):
        ax = 2 + (dim - 1 - d)
        for c in (em, ep):
            out.append(np.tensordot(V, c, axes=([ax], [0])).reshape(5, E, -1))
    return np.concatenate(out, axis=2)


def weights(N, dim):
    w = np.polynomial.legendre.leggauss(N)[1]
    out = w
    for _ in range(dim - 1):
        out = np.multiply.outer(w, out).ravel()
    return out


CASES = [(1, 3), (2, 2), (2, 3), (3, 2)]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"dim{c[0]}p{c[1]}")
def case(request):
    dim, p = request.param
    N = p + 1
    U = wl.random_conserved_cells(400, N ** dim, seed=40 + dim + p, bad_fraction=0.15)
    # 20 cells with admissible nodes whose polynomial leaves the admissible set at a face: D
    # linear along x with slope 1.15 D0 at rest (D > 0 at the outermost node, < 0 at x = -1)
    x = np.polynomial.legendre.leggauss(N)[0][np.arange(N ** dim) % N]
    D0 = np.linspace(0.5, 2.0, 20)[:, None]
    U[:, :20] = 0.0
    U[0, :20] = D0 * (1.0 + 1.15 * x)
    U[4, :20] = 0.3 * D0
    spec = dict(dim=dim, degree=p, n_elem=[400] + [1] * (dim - 1), eos="ideal", gamma_ad=5.0 / 3.0,
                enforce="faces")
    w = weights(N, dim)
    mean = (U * w).sum(-1) / w.sum()
    F = face_values(U, N, dim)
    nodes_ok = admissible(U).all(-1)
    faces_ok = admissible(F).all(-1)
    return spec, U, w, mean, F, nodes_ok, faces_ok, N, dim


def test_fixture_has_cells_flagged_by_their_faces_alone(case):
    spec, U, w, mean, F, nodes_ok, faces_ok, N, dim = case
    assert (nodes_ok & ~faces_ok & admissible(mean)).sum() >= 3
    assert (nodes_ok & faces_ok).sum() >= 30


def test_identity_where_nodes_and_faces_are_admissible(case):
    spec, U, w, mean, F, nodes_ok, faces_ok, N, dim = case
    Un, s, _ = oracle.enforce(spec, U)
    keep = nodes_ok & faces_ok
    assert np.array_equal(Un[:, keep], U[:, keep]) and np.all(s[keep] == 1.0)


def test_nodes_and_face_points_admissible_and_mean_kept(case):
    spec, U, w, mean, F, nodes_ok, faces_ok, N, dim = case
    Un, s, st = oracle.enforce(spec, U)
    fix = ~(nodes_ok & faces_ok) & admissible(mean)
    assert admissible(Un[:, fix]).all()
    assert admissible(face_values(Un, N, dim)[:, fix]).all()
    new_mean = (Un * w).sum(-1) / w.sum()
    assert np.allclose(new_mean[:, fix], mean[:, fix], rtol=0, atol=1e-14 * np.abs(U).max())
    assert st["enforced_cells"] == fix.sum()


def test_factor_is_largest_admissible_over_nodes_and_faces_by_bisection(case):
    """s = (1 - 1e-12) x the largest s in [0, 1] for which every smoothed node and every smoothed
    face point s X + (1 - s) Ubar is admissible (200 bisection steps per cell)."""
    spec, U, w, mean, F, nodes_ok, faces_ok, N, dim = case
    _, s, _ = oracle.enforce(spec, U)
    fix = np.where(~(nodes_ok & faces_ok) & admissible(mean))[0]
    P = np.concatenate([U, F], axis=2)[:, fix]
    M = mean[:, fix][:, :, None]
    lo, hi = np.zeros(len(fix)), np.ones(len(fix))
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        ok = admissible(mid[None, :, None] * P + (1 - mid[None, :, None]) * M).all(-1)
        lo, hi = np.where(ok, mid, lo), np.where(ok, hi, mid)
    assert np.allclose(s[fix] / (1 - 1e-12), lo, rtol=1e-12, atol=1e-14)


def test_face_variant_is_never_weaker_than_the_nodal_operator(case):
    spec, U, w, mean, F, nodes_ok, faces_ok, N, dim = case
    _, s_faces, _ = oracle.enforce(spec, U)
    _, s_nodes, _ = oracle.enforce(dict(spec, enforce=True), U)
    assert np.all(s_faces <= s_nodes)
    assert np.any(s_faces < s_nodes)
