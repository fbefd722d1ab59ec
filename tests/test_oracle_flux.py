"""Pins for the oracle's flux (Eq. srhd_flux), wavespeeds (Sec. 2.4) and numerical fluxes."""
import numpy as np
import pytest

import oracle
import workloads as wl
from tests import mp_reference as mpr

SPECS = {"ideal": dict(dim=3, degree=0, n_elem=[1, 1, 1], eos="ideal", gamma_ad=5.0 / 3.0),
         "tm": dict(dim=3, degree=0, n_elem=[1, 1, 1], eos="tm", gamma_ad=5.0 / 3.0)}


@pytest.mark.parametrize("eos", ["ideal", "tm"])
def test_phys_flux_matches_definition(eos):
    W = wl.random_primitive_states(100, seed=21)
    for k in range(W.shape[1]):
        for d in range(3):
            F = oracle.phys_flux(SPECS[eos], W[:, k], d)
            ref = np.array([float(x) for x in mpr.flux(eos, 5.0 / 3.0, W[:, k], d)])
            lor2 = 1.0 / (1.0 - (W[1:4, k] ** 2).sum())
            assert np.allclose(F, ref, rtol=0, atol=1e-14 * lor2 * np.abs(ref).max())


@pytest.mark.parametrize("eos", ["ideal", "tm"])
def test_wavespeeds_are_extreme_eigenvalues(eos):
    """lambda_pm equal the smallest and largest eigenvalues of dF/dU = (dF/dW)(dU/dW)^-1,
    the Jacobians taken by central differences of the (separately pinned) prim->cons map and
    flux."""
    spec = SPECS[eos]
    W = wl.random_primitive_states(40, seed=22, gamma_max=5.0, theta_range=(1e-2, 1e2),
                                   rho_range=(0.1, 10))
    for k in range(W.shape[1]):
        w0 = W[:, k]
        for d in range(3):
            JF = np.zeros((5, 5))
            JU = np.zeros((5, 5))
            for j in range(5):
                h = 1e-6 * (abs(w0[j]) + 1e-3)
                wp, wm = w0.copy(), w0.copy()
                wp[j] += h
                wm[j] -= h
                JF[:, j] = (oracle.phys_flux(spec, wp, d) - oracle.phys_flux(spec, wm, d)) / (2 * h)
                JU[:, j] = (oracle.prim2cons(spec, wp[:, None])[:, 0] -
                            oracle.prim2cons(spec, wm[:, None])[:, 0]) / (2 * h)
            ev = np.linalg.eigvals(JF @ np.linalg.inv(JU)).real
            lm, lp = oracle.wavespeeds(spec, w0, d)
            assert abs(ev.min() - lm) < 1e-6 and abs(ev.max() - lp) < 1e-6
            assert -1.0 < lm < lp < 1.0


@pytest.mark.parametrize("eos", ["ideal", "tm"])
@pytest.mark.parametrize("flux", ["llf", "hll", "hllc"])
def test_numerical_flux_consistency(eos, flux):
    spec = dict(SPECS[eos], flux=flux)
    W = wl.random_primitive_states(50, seed=23)
    for k in range(W.shape[1]):
        for d in range(3):
            F = oracle.phys_flux(spec, W[:, k], d)
            Fs = oracle.numerical_flux(spec, W[:, k], W[:, k], d)
            assert np.allclose(Fs, F, rtol=1e-13, atol=1e-13 * np.abs(F).max())


def test_hll_upwinds_supersonic_flow():
    spec = dict(SPECS["ideal"], flux="hll")
    WL = np.array([1.0, 0.95, 0.0, 0.0, 0.01])
    WR = np.array([0.5, 0.9, 0.1, 0.0, 0.02])
    assert oracle.wavespeeds(spec, WL, 0)[0] > 0 and oracle.wavespeeds(spec, WR, 0)[0] > 0
    assert np.allclose(oracle.numerical_flux(spec, WL, WR, 0), oracle.phys_flux(spec, WL, 0),
                       rtol=1e-14, atol=1e-15)
    WL2, WR2 = WL.copy(), WR.copy()
    WL2[1], WR2[1] = -0.9, -0.95
    assert np.allclose(oracle.numerical_flux(spec, WL2, WR2, 0), oracle.phys_flux(spec, WR2, 0),
                       rtol=1e-14, atol=1e-15)


def test_llf_is_hll_with_symmetric_speeds_for_a_contact():
    """For a pure contact at rest (same P and v = 0) both fluxes keep P continuous; LLF adds
    dissipation -a/2 [D] to the mass flux with a the largest |lambda|, HLL the same with
    S_R = -S_L = a."""
    spec = dict(SPECS["ideal"])
    WL = np.array([1.0, 0.0, 0.0, 0.0, 1.0])
    WR = np.array([0.1, 0.0, 0.0, 0.0, 1.0])
    Fl = oracle.numerical_flux(dict(spec, flux="llf"), WL, WR, 0)
    Fh = oracle.numerical_flux(dict(spec, flux="hll"), WL, WR, 0)
    assert Fl[0] > 0 and Fh[0] > 0          # mass diffuses towards the lighter side
    assert abs(Fl[1] - 1.0) < 1e-15 and abs(Fh[1] - 1.0) < 1e-15
    assert np.allclose(Fl, Fh, rtol=1e-14)


# ---------------------------------------------------------------------------------------
# HLLC: the properties that define it (exact isolated contacts, upwinding, consistency)
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("eos", ["ideal", "tm"])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_hllc_resolves_a_stationary_contact(eos, d):
    """Density jump at rest with equal pressure: HLLC's contact speed is 0 and its flux is the
    exact (0, P e_d, 0); HLL and LLF diffuse mass across it."""
    spec = dict(SPECS[eos], flux="hllc")
    WL = np.array([1.0, 0.0, 0.0, 0.0, 0.7])
    WR = np.array([0.1, 0.0, 0.0, 0.0, 0.7])
    F = oracle.numerical_flux(spec, WL, WR, d)
    want = np.zeros(5)
    want[1 + d] = 0.7
    assert np.allclose(F, want, rtol=0, atol=1e-15), F
    assert oracle.numerical_flux(dict(spec, flux="hll"), WL, WR, d)[0] > 1e-3


@pytest.mark.parametrize("eos", ["ideal", "tm"])
@pytest.mark.parametrize("vn", [0.45, -0.6])
def test_hllc_moving_contact_is_exactly_upwind(eos, vn):
    """A contact moving with v_x = vn (equal v_x and P, jumps in rho and the transverse
    velocities): the flux is the physical flux of the upwind state."""
    spec = dict(SPECS[eos], flux="hllc")
    WL = np.array([1.0, vn, 0.3, -0.1, 0.5])
    WR = np.array([0.2, vn, -0.4, 0.2, 0.5])
    F = oracle.numerical_flux(spec, WL, WR, 0)
    up = WL if vn > 0 else WR
    Fu = oracle.phys_flux(spec, up, 0)
    assert np.allclose(F, Fu, rtol=1e-13, atol=1e-14 * np.abs(Fu).max()), (F, Fu)


def test_hllc_upwinds_supersonic_flow():
    spec = dict(SPECS["ideal"], flux="hllc")
    WL = np.array([1.0, 0.95, 0.0, 0.0, 0.01])
    WR = np.array([0.5, 0.9, 0.1, 0.0, 0.02])
    assert np.array_equal(oracle.numerical_flux(spec, WL, WR, 0), oracle.phys_flux(spec, WL, 0))


@pytest.mark.parametrize("flux", ["llf", "hll", "hllc"])
def test_symmetric_collision_has_no_mass_or_energy_flux(flux):
    """A state against its mirror image (the reflecting-wall ghost): no mass and no energy
    cross the face, only momentum (the wall pressure), for every flux."""
    spec = dict(SPECS["ideal"], flux=flux)
    W = np.array([1.0, 0.6, 0.2, 0.0, 0.3])
    M = W.copy()
    M[1] = -M[1]
    F = oracle.numerical_flux(spec, W, M, 0)
    assert abs(F[0]) < 1e-15 and abs(F[4]) < 1e-15 and abs(F[2]) < 1e-15 and F[1] > 0.3


@pytest.mark.parametrize("flux", ["llf", "hll", "hllc"])
def test_reflecting_walls_conserve_mass_and_energy(flux):
    """1D, reflecting walls at both ends, smooth data with flows into the walls: the quadrature
    sums of D and tau (total mass and energy) are conserved to rounding over 40 steps."""
    spec = dict(dim=1, degree=2, n_elem=[24], lo=[0.0], hi=[1.0], eos="ideal",
                gamma_ad=5.0 / 3.0, c2p="iterative", flux=flux, rk_stages=3,
                bc=[("reflect", "reflect")], enforce=True)
    X = oracle.node_coords(spec)
    x = X[0]
    W = np.stack([1.0 + 0.3 * np.sin(2 * np.pi * x), 0.5 * np.sin(np.pi * x) + 0.2, 0.0 * x,
                  0.0 * x, 1.0 + 0.2 * np.cos(3 * x)])
    U = oracle.prim2cons(spec, W)
    w = np.polynomial.legendre.leggauss(3)[1]
    mass = lambda V: float((V[0] * w).sum())
    energy = lambda V: float((V[4] * w).sum())
    m0, e0 = mass(U), energy(U)
    U1, st = oracle.step(spec, U, oracle.cfl_dt(spec, 0.2), 40)
    assert st["c2p_nonconverged"] == 0
    assert abs(mass(U1) - m0) <= 1e-13 * m0 and abs(energy(U1) - e0) <= 1e-13 * e0
    assert np.abs(U1[1] - U[1]).max() > 1e-3  # the walls do act on the momentum
