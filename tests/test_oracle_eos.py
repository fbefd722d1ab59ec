"""Pins for the oracle's equations of state and prim->cons map (Secs. 2.1, 2.2)."""
import mpmath as mp
import numpy as np
import pytest

import oracle
import workloads as wl
from tests import mp_reference as mpr

IDEAL = dict(dim=1, degree=0, n_elem=[1], eos="ideal", gamma_ad=5.0 / 3.0)
TM = dict(dim=1, degree=0, n_elem=[1], eos="tm", gamma_ad=5.0 / 3.0)


@pytest.mark.parametrize("theta", np.logspace(-6, 6, 25))
def test_taub_matthews_identity(theta):
    """Taub's inequality holds with equality for the TM EOS: (h - Theta)(h - 4 Theta) = 1."""
    h = oracle.enthalpy(TM, 1.0, theta)
    # h - 4 Theta cancels for hot states: the rounding error grows as Theta^2
    assert abs((h - theta) * (h - 4 * theta) - 1.0) < 1e-14 * (1.0 + theta * theta)


def test_equivalent_adiabatic_index_limits():
    """Gamma_eq = (h - 1) / (h - 1 - Theta) runs from 5/3 (cold) to 4/3 (hot) for the TM EOS and
    is Gamma itself for the ideal EOS (Sec. 2.2; the diagnostic of Fig. 9)."""
    th = np.logspace(-4, 4, 30)
    gs = oracle.gamma_eq(TM, 1.0, th)
    assert abs(oracle.gamma_eq(TM, 1.0, 1e-6) - 5.0 / 3.0) < 1e-5
    assert abs(oracle.gamma_eq(TM, 1.0, 1e6) - 4.0 / 3.0) < 1e-5
    assert np.all(np.diff(gs) <= 0.0)
    # depends on Theta alone
    assert np.allclose(oracle.gamma_eq(TM, 7.0, 7.0 * th), gs, rtol=1e-14, atol=0.0)
    for G in (4.0 / 3.0, 5.0 / 3.0):
        assert np.allclose(oracle.gamma_eq(dict(IDEAL, gamma_ad=G), 1.0, th), G, rtol=1e-12)


@pytest.mark.parametrize("spec", [IDEAL, dict(IDEAL, gamma_ad=4.0 / 3.0), TM])
def test_sound_speed_from_general_definition(spec):
    """c_s^2 = -(rho / (n h)) dh/drho with n = rho dh/dP - 1 (Sec. 2.2), by central
    differences of the oracle's h(rho, P)."""
    rng = np.random.default_rng(1)
    for _ in range(40):
        rho = 10 ** rng.uniform(-2, 2)
        P = rho * 10 ** rng.uniform(-3, 3)
        hr, hp = 1e-5 * rho, 1e-5 * P
        dh_drho = (oracle.enthalpy(spec, rho + hr, P) - oracle.enthalpy(spec, rho - hr, P)) / (2 * hr)
        dh_dP = (oracle.enthalpy(spec, rho, P + hp) - oracle.enthalpy(spec, rho, P - hp)) / (2 * hp)
        n = rho * dh_dP - 1.0
        cs2 = -rho / (n * oracle.enthalpy(spec, rho, P)) * dh_drho
        assert abs(oracle.cs2(spec, rho, P) - cs2) < 1e-8 * cs2
        assert 0.0 < oracle.cs2(spec, rho, P) < 1.0


@pytest.mark.parametrize("eos", ["ideal", "tm"])
def test_prim2cons_matches_definition(eos):
    """The oracle's cancellation-free prim->cons equals Eq. primitive_to_conserved evaluated
    at 40 digits, componentwise, including cold states where tau << D."""
    spec = IDEAL if eos == "ideal" else TM
    W = np.concatenate([wl.random_primitive_states(300, seed=3),
                        wl.random_primitive_states(300, seed=4, theta_range=(1e-12, 1e-6),
                                                   gamma_max=100.0)], axis=1)
    U = oracle.prim2cons(spec, W)
    lor2 = 1.0 / (1.0 - (W[1:4] ** 2).sum(0))
    for k in range(W.shape[1]):
        ref = mpr.prim2cons(eos, spec["gamma_ad"], W[:, k])
        for v in range(5):
            r = float(ref[v])
            scale = abs(r) if v in (0, 4) else float(mp.sqrt(ref[1] ** 2 + ref[2] ** 2 + ref[3] ** 2))
            # 1 - v^2 carries a relative rounding error of about eps gamma^2
            assert abs(U[v, k] - r) <= 4e-15 * lor2[k] * scale + 1e-300, (k, v, U[v, k], r)


def test_taub_matthews_approximates_the_synge_gas():
    """Sec. 2.2 and Fig. 1: the Taub-Matthews EOS approximates the Synge gas,
    h = K_3(1/Theta) / K_2(1/Theta) (modified Bessel functions, here exponentially scaled:
    the scale cancels in the ratio).  It agrees with it to a few per cent across Theta and
    exactly in both limits (h -> 1 + 5/2 Theta cold, h -> 4 Theta hot)."""
    from scipy.special import kve
    th = np.logspace(-3, 3, 601)
    synge = kve(3, 1.0 / th) / kve(2, 1.0 / th)
    tm = np.array([oracle.enthalpy(TM, 1.0, t) for t in th])
    rel = np.abs(tm - synge) / synge
    assert rel.max() < 0.025
    assert 0.3 < th[np.argmax(rel)] < 1.0        # the largest gap sits at Theta of order 1
    assert rel[0] < 1e-5 and rel[-1] < 1e-5
