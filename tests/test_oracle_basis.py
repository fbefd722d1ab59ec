"""Pins for the oracle's basis tables (Sec. 2.3): Gauss-Legendre rule, Lagrange derivative
and extrapolation tables."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("N", range(1, 9))
def test_gauss_legendre_matches_library(N):
    x, w = oracle.gauss_legendre(N)
    xr, wr = np.polynomial.legendre.leggauss(N)
    assert np.allclose(x, xr, rtol=0, atol=2e-15)
    assert np.allclose(w, wr, rtol=0, atol=2e-15)


@pytest.mark.parametrize("N", range(1, 9))
def test_quadrature_exact_to_degree_2N_minus_1(N):
    x, w = oracle.gauss_legendre(N)
    for k in range(2 * N):
        exact = (1.0 - (-1.0) ** (k + 1)) / (k + 1)
        assert abs(w @ x ** k - exact) < 1e-14


@pytest.mark.parametrize("N", range(1, 8))
def test_summation_by_parts(N):
    """For any f of degree <= N: sum_a w_i Dhat_ia f(x_a) = phi_i(1) f(1) - phi_i(-1) f(-1)
    - w_i f'(x_i) (integration by parts, exact under the N-point rule)."""
    b = oracle.basis(N)
    x, w, D, em, ep = b["x"], b["w"], b["Dhat"], b["em"], b["ep"]
    rng = np.random.default_rng(N)
    for _ in range(5):
        f = np.polynomial.Polynomial(rng.normal(size=N + 1))
        fp = f.deriv()
        lhs = (w[:, None] * D) @ f(x)
        rhs = ep * f(1.0) - em * f(-1.0) - w * fp(x)
        assert np.allclose(lhs, rhs, rtol=0, atol=1e-12 * (1 + np.abs(rhs).max()))


@pytest.mark.parametrize("N", range(1, 8))
def test_extrapolation_exact_on_polynomials(N):
    b = oracle.basis(N)
    for k in range(N):
        assert abs(b["ep"] @ b["x"] ** k - 1.0) < 1e-13
        assert abs(b["em"] @ b["x"] ** k - (-1.0) ** k) < 1e-13


def test_node_coordinates_2d():
    spec = dict(dim=2, degree=2, n_elem=[3, 2], lo=[-1.0, 0.5], hi=[2.0, 1.5])
    X = oracle.node_coords(spec)
    x, _ = np.polynomial.legendre.leggauss(3)
    assert X.shape == (2, 6, 9)
    for e in range(6):
        ex, ey = e % 3, e // 3
        for n in range(9):
            a, b = n % 3, n // 3
            assert abs(X[0, e, n] - (-1.0 + (ex + 0.5 * (1 + x[a])) * 1.0)) < 1e-14
            assert abs(X[1, e, n] - (0.5 + (ey + 0.5 * (1 + x[b])) * 0.5)) < 1e-14


# ---------------------------------------------------------------------------------------
# Gauss-Lobatto-Legendre variant (the node family the paper leaves open)
# ---------------------------------------------------------------------------------------
GLL_TABLE = {
    2: ([-1.0, 1.0], [1.0, 1.0]),
    3: ([-1.0, 0.0, 1.0], [1 / 3, 4 / 3, 1 / 3]),
    4: ([-1.0, -1 / np.sqrt(5), 1 / np.sqrt(5), 1.0], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    5: ([-1.0, -np.sqrt(3 / 7), 0.0, np.sqrt(3 / 7), 1.0], [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
}


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_gll_nodes_and_weights_match_the_closed_forms(N):
    b = oracle.basis(N, "gll")
    x, w = GLL_TABLE[N]
    assert np.allclose(b["x"], x, rtol=0, atol=1e-15) and np.allclose(b["w"], w, rtol=0, atol=1e-15)


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_gll_quadrature_degree_and_summation_by_parts(N):
    """Exact for degree 2N - 3; end-point traces are the end nodes; the collocated
    differentiation satisfies W D + (W D)^T = diag(-1, 0, ..., 0, 1) (summation by parts)."""
    b = oracle.basis(N, "gll")
    x, w = b["x"], b["w"]
    for k in range(2 * N - 2):
        assert abs((w * x ** k).sum() - (2.0 / (k + 1) if k % 2 == 0 else 0.0)) < 1e-14
    assert np.allclose(b["em"], np.eye(N)[0]) and np.allclose(b["ep"], np.eye(N)[-1])
    # Dhat[i][a] = w_a phi_i'(x_a) / w_i, so w_i Dhat[i][a] = w_a phi_i'(x_a) = (W D)[a][i]
    WD = (w[:, None] * b["Dhat"]).T
    B = np.zeros((N, N))
    B[0, 0], B[-1, -1] = -1.0, 1.0
    assert np.allclose(WD + WD.T, B, atol=1e-13)
