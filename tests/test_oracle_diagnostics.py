"""Oracle pins of the Kelvin-Helmholtz diagnostic <v_a^2> = (1/|Omega|) int v_a^2 dV (Sec. 4.5)
and of the paper's Kelvin-Helmholtz initial field."""
import math

import numpy as np

import oracle
import workloads as wl


def _state(spec, W):
    return oracle.prim2cons(spec, W)


def test_mean_square_velocity_closed_form():
    """v_y = 0.3 sin(2 pi x), v_x = 0.2 on the periodic unit square, 8 x 8 elements, p = 3.  The
    nodal quadrature of sin^2 = (1 - cos(4 pi x)) / 2 on a uniform mesh of 8 elements is exact:
    the cos part sums e^{i pi e / 2} over e = 0..7, a full set of roots of unity, to zero.  So
    <v_y^2> = 0.3^2 / 2 and <v_x^2> = 0.2^2 up to rounding (and the con2prim round trip)."""
    spec = dict(dim=2, degree=3, n_elem=[8, 8], lo=[0.0, 0.0], hi=[1.0, 1.0], eos="ideal",
                gamma_ad=4.0 / 3.0, c2p="iterative", bc=[("periodic", "periodic")] * 2)
    X = oracle.node_coords(spec)
    W = np.stack([np.ones_like(X[0]), 0.2 + 0.0 * X[0], 0.3 * np.sin(2 * np.pi * X[0]),
                  0.0 * X[0], np.ones_like(X[0])])
    U = _state(spec, W)
    assert abs(oracle.mean_square_velocity(spec, U, 1) - 0.045) < 1e-14
    assert abs(oracle.mean_square_velocity(spec, U, 0) - 0.04) < 1e-14
    assert oracle.mean_square_velocity(spec, U, 2) == 0.0


def test_mean_square_velocity_scales_with_the_domain():
    """The same field on [0, 2] x [0, 3] with the wavelength scaled to the domain has the same
    mean: the (dx/2) Jacobians and 1/|Omega| cancel."""
    spec = dict(dim=2, degree=2, n_elem=[8, 4], lo=[0.0, 0.0], hi=[2.0, 3.0], eos="ideal",
                gamma_ad=5.0 / 3.0, c2p="iterative", bc=[("periodic", "periodic")] * 2)
    X = oracle.node_coords(spec)
    W = np.stack([np.ones_like(X[0]), 0.0 * X[0], 0.3 * np.sin(np.pi * X[0]), 0.0 * X[0],
                  np.ones_like(X[0])])
    assert abs(oracle.mean_square_velocity(spec, _state(spec, W), 1) - 0.045) < 1e-14


def test_kh_single_initial_field_against_its_integral():
    """t = 0 of the paper's set-up: v_y = A sin(2 pi x) exp(-y^2 / sigma^2) on [-0.5, 0.5] x
    [-1, 1] gives <v_y^2> = (1/2) (1/2) A^2 sigma sqrt(pi / 2) erf(sqrt(2) / sigma)
    (the Gaussian integral; erf = 1 to double precision here)."""
    spec = wl.kh_single(nx=64, ny=128, degree=3)
    X = oracle.node_coords(spec)
    U = _state(spec, wl.kh_single_ic(spec, X))
    A, s = spec["amplitude"], spec["sigma"]
    exact = 0.25 * A * A * s * math.sqrt(math.pi / 2.0) * math.erf(math.sqrt(2.0) / s)
    got = oracle.mean_square_velocity(spec, U, 1)
    assert abs(got - exact) <= 1e-9 * exact, (got, exact)
    # v_x = 0.25 tanh(y / a): <v_x^2> = 0.25^2 (1 - a tanh(1/a) / 1) over y in [-1, 1]
    a = spec["layer"]
    ex_x = spec["shear"] ** 2 * (1.0 - a * math.tanh(1.0 / a))
    assert abs(oracle.mean_square_velocity(spec, U, 0) - ex_x) <= 1e-6 * ex_x
