"""Pins for the oracle's four conserved->primitive solvers (Sec. 3): round trips against the
exact prim->cons map, the paper's accuracy study on its (gamma, P) grid (Sec. 3.3), iteration
counts, the zero-momentum case and invalid input."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as wl
from tests import mp_reference as mpr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "con2prim_accuracy_envelope.json")


def spec_for(eos, c2p, max_iter=0, gamma_ad=5.0 / 3.0):
    return dict(dim=1, degree=0, n_elem=[1], eos=eos, gamma_ad=gamma_ad, c2p=c2p,
                c2p_max_iter=max_iter)


def exact_cons(eos, gamma_ad, W):
    """Conserved states from Eq. primitive_to_conserved at 40 digits, rounded once."""
    return np.array([[float(x) for x in mpr.prim2cons(eos, gamma_ad, W[:, k])]
                     for k in range(W.shape[1])]).T


def vel_err(Wr, W):
    v = np.linalg.norm(W[1:4], axis=0)
    return np.linalg.norm(Wr[1:4] - W[1:4], axis=0) / np.where(v > 0, v, 1.0)


@pytest.fixture(scope="module")
def moderate_box():
    """gamma in [1, 10], Theta in [1e-3, 1e3], rho in [1e-3, 1e3]."""
    W = wl.random_primitive_states(400, seed=11)
    return W, {"ideal": exact_cons("ideal", 5.0 / 3.0, W), "tm": exact_cons("tm", 5.0 / 3.0, W)}


@pytest.mark.parametrize("eos,c2p", [("ideal", "iterative"), ("tm", "analytic"), ("tm", "iterative")])
def test_round_trip_well_conditioned_solvers(moderate_box, eos, c2p):
    W, U = moderate_box
    Wr, it, st = oracle.con2prim(spec_for(eos, c2p), U[eos])
    assert st["c2p_nonconverged"] == 0 and st["c2p_invalid_input"] == 0
    assert vel_err(Wr, W).max() < 2e-13
    assert (np.abs(Wr[0] - W[0]) / W[0]).max() < 5e-13
    # pressure: conditioning of E - S.v - rho for cold, fast states (P / (tau + |S|) small)
    kappa = (U[eos][4] + np.linalg.norm(U[eos][1:4], axis=0)) / W[4]
    assert (np.abs(Wr[4] - W[4]) / W[4] / kappa).max() < 1e-14


@pytest.mark.parametrize("eos,c2p", [("ideal", "analytic"), ("ideal", "iterative"),
                                     ("tm", "analytic"), ("tm", "iterative")])
def test_backward_error(moderate_box, eos, c2p):
    """The recovered primitive reproduces the conserved state (exact prim->cons at 40 digits)."""
    W, U = moderate_box
    Wr, _, _ = oracle.con2prim(spec_for(eos, c2p), U[eos])
    # the closed-form quartic route loses digits on hot, fast states (Sec. 3.3 reports its
    # error growing with gamma); on this machine its backward error stays below 1e-7
    tol = 1e-7 if c2p == "analytic" and eos == "ideal" else 1e-13
    Ur = exact_cons(eos, 5.0 / 3.0, Wr)
    scale = U[eos][0] + U[eos][4] + np.linalg.norm(U[eos][1:4], axis=0)
    assert (np.abs(Ur - U[eos]).max(axis=0) / scale).max() < tol


@pytest.mark.parametrize("eos,G", [("ideal", 4.0 / 3.0), ("ideal", 5.0 / 3.0), ("tm", 5.0 / 3.0)])
def test_hot_ultrarelativistic_round_trip(eos, G):
    """Hot states near |v| = 1, gamma up to 100 and Theta from 10 to 1e3 (the states behind the
    Taub-Matthews blast of Sec. 4.3): the iterative solver converges and recovers the primitive
    from its exact conserved state.  rho = D / gamma is the ill-conditioned output: the root
    w < 1 has a partner 1/w about 2/gamma away, so its rounding grows as gamma, and gamma's
    sensitivity to w adds another factor gamma (about 20 eps gamma^2)."""
    rng = np.random.default_rng(3)
    n = 300
    gam = np.exp(rng.uniform(np.log(5.0), np.log(100.0), n))
    th = np.exp(rng.uniform(np.log(10.0), np.log(1e3), n))
    rho = np.exp(rng.uniform(np.log(1e-2), np.log(1e2), n))
    v = np.sqrt(1.0 - 1.0 / gam ** 2)
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    W = np.stack([rho, v * np.cos(phi), v * np.sin(phi), np.zeros(n), rho * th])
    U = exact_cons(eos, G, W)
    Wr, it, st = oracle.con2prim(spec_for(eos, "iterative", gamma_ad=G), U)
    assert st["c2p_nonconverged"] == 0 and st["c2p_invalid_input"] == 0
    assert vel_err(Wr, W).max() < 1e-14
    assert (np.abs(Wr[0] - W[0]) / W[0] / gam ** 2).max() < 1e-14
    kappa = (U[4] + np.linalg.norm(U[1:4], axis=0)) / W[4]
    assert (np.abs(Wr[4] - W[4]) / W[4] / kappa).max() < 1e-14


def test_solvers_agree(moderate_box):
    W, U = moderate_box
    a, _, _ = oracle.con2prim(spec_for("ideal", "analytic"), U["ideal"])
    i, _, _ = oracle.con2prim(spec_for("ideal", "iterative"), U["ideal"])
    assert vel_err(a, i).max() < 1e-8
    a, _, _ = oracle.con2prim(spec_for("tm", "analytic"), U["tm"])
    i, _, _ = oracle.con2prim(spec_for("tm", "iterative"), U["tm"])
    assert vel_err(a, i).max() < 1e-13


@pytest.fixture(scope="module")
def e2():
    W, lor, P_si = wl.e2_grid()
    Wf = W.reshape(5, -1)
    G = np.tile(lor, 25)
    return Wf, G, {"ideal": exact_cons("ideal", 5.0 / 3.0, Wf), "tm": exact_cons("tm", 5.0 / 3.0, Wf)}


def _v_err(Wr, Wf):
    v = Wf[1]
    return np.where(v > 0, np.abs(Wr[1] - v) / np.where(v > 0, v, 1.0), np.abs(Wr[1]))


def test_e2_grid_ideal_analytic_envelope(e2):
    """Sec. 3.3: the analytic ideal solver recovers v to ~1e-15 below gamma = 3, losing
    accuracy roughly as a power law to ~1e-10 at gamma = 100."""
    claims = json.load(open(GOLDEN))["claims"]
    Wf, G, U = e2
    Wr, _, st = oracle.con2prim(spec_for("ideal", "analytic"), U["ideal"])
    err = _v_err(Wr, Wf)
    assert st["c2p_nonconverged"] == 0
    assert err[G < 3].max() < 100 * claims["ideal_analytic_gamma_below_3_max_rel_err_v"]
    assert err[G == 100].max() < 10 * claims["ideal_analytic_gamma_100_rel_err_v_order"]
    assert err[G == 100].max() > 1e-3 * claims["ideal_analytic_gamma_100_rel_err_v_order"]


def test_e2_grid_ideal_iterative_iteration_claims(e2):
    """Sec. 3.3: 6 Newton iterations reach machine precision for gamma < 10; 12 reach it for
    every gamma <= 100."""
    Wf, G, U = e2
    W6, _, _ = oracle.con2prim(spec_for("ideal", "iterative", 6), U["ideal"])
    W12, it, _ = oracle.con2prim(spec_for("ideal", "iterative", 12), U["ideal"])
    assert _v_err(W6, Wf)[G < 10].max() < 4e-15
    assert _v_err(W12, Wf).max() < 4e-15
    assert it.max() <= 12


def test_e2_grid_taub_matthews(e2):
    """Sec. 3.3: the TM analytic solver is near machine precision everywhere; Brent's method
    needs tens of iterations (the paper tests 25 and 50)."""
    Wf, G, U = e2
    Wa, _, _ = oracle.con2prim(spec_for("tm", "analytic"), U["tm"])
    Wi, it, st = oracle.con2prim(spec_for("tm", "iterative"), U["tm"])
    assert _v_err(Wa, Wf).max() < 1e-14
    assert _v_err(Wi, Wf).max() < 1e-14
    assert st["c2p_nonconverged"] == 0
    assert 10 <= it.mean() <= 50 and it.max() <= 60


@pytest.mark.parametrize("eos,c2p", [("ideal", "analytic"), ("ideal", "iterative"),
                                     ("tm", "analytic"), ("tm", "iterative")])
def test_zero_momentum(eos, c2p):
    W = np.array([[2.0], [0.0], [0.0], [0.0], [0.3]])
    U = exact_cons(eos, 5.0 / 3.0, W)
    Wr, _, st = oracle.con2prim(spec_for(eos, c2p), U)
    assert np.all(Wr[1:4] == 0.0)
    assert abs(Wr[0, 0] - 2.0) < 1e-15 and abs(Wr[4, 0] - 0.3) < 1e-14
    assert st["c2p_nonconverged"] == 0


@pytest.mark.parametrize("eos,c2p", [("ideal", "iterative"), ("tm", "iterative")])
def test_small_momentum_series(eos, c2p):
    """xi below the series threshold: the small-xi series of Eq. iterative_cubic_approximation
    (ideal) and Brent (TM) still recover v to machine precision."""
    W = np.array([[1.0, 1.0], [1e-7, 3e-6], [0.0, 0.0], [0.0, 0.0], [1.0, 1e-6]])
    U = exact_cons(eos, 5.0 / 3.0, W)
    Wr, _, _ = oracle.con2prim(spec_for(eos, c2p), U)
    assert vel_err(Wr, W).max() < 1e-12


def test_invalid_input_is_counted():
    U = np.array([[-1.0, 1.0, 1.0, np.nan, 1.0],
                  [0.0, 0.0, 2.0, 0.0, 0.0],
                  [0.0, 0.0, 0.0, 0.0, 0.0],
                  [0.0, 0.0, 0.0, 0.0, 0.0],
                  [1.0, -0.5, 0.5, 1.0, 0.1]])
    for eos in ("ideal", "tm"):
        for c2p in ("analytic", "iterative"):
            Wr, _, st = oracle.con2prim(spec_for(eos, c2p), U)
            assert st["c2p_invalid_input"] == 4
            assert np.all(np.isnan(Wr[:, :4]))
            assert np.all(np.isfinite(Wr[:, 4]))


def test_iteration_cap_counts_nonconvergence():
    W = wl.random_primitive_states(50, seed=5, gamma_max=50.0)
    U = exact_cons("tm", 5.0 / 3.0, W)
    _, it, st = oracle.con2prim(spec_for("tm", "iterative", 3), U)
    assert st["c2p_nonconverged"] > 0 and it.max() == 3


@pytest.mark.parametrize("eos,rtol", [("ideal", 1e-6), ("tm", 1e-6), ("tm", 1e-9)])
def test_relative_tolerance_stops_earlier_within_it(moderate_box, eos, rtol):
    """c2p_rtol > 0: the iterative solvers stop once Newton's step or Brent's bracket is within
    rtol of the iterate, in fewer iterations, and the recovered velocity stays within rtol of
    the exact one (Newton's last step squares its error; Brent's bracket holds the root)."""
    W, U = moderate_box
    spec = spec_for(eos, "iterative")
    Wr0, it0, _ = oracle.con2prim(spec, U[eos])
    Wr, it, st = oracle.con2prim(dict(spec, c2p_rtol=rtol), U[eos])
    assert st["c2p_nonconverged"] == 0
    assert np.all(it <= it0) and it.mean() < it0.mean()
    # W = gamma^2 - 1 (TM) or w (ideal) within rtol: |v| within rtol (times gamma^2 for TM)
    g2 = 1.0 / (1.0 - (W[1:4] ** 2).sum(0))
    assert (vel_err(Wr, W) / g2).max() < 10.0 * rtol
    assert vel_err(Wr0, W).max() < 2e-13


@pytest.mark.parametrize("theta", [1e16, 1e18, 1e20, 1e22])
@pytest.mark.parametrize("gam", [1.5, 10.0])
def test_extreme_pressure_closed_form_fails_newton_does_not(theta, gam):
    """Sec. 3.3: at very high pressures the ideal closed form runs into negative radicands and
    loses the velocity, while the iterative solver does not.  Here from P/rho = 1e16 on, the
    closed form returns NaN (flagged as not converged) or a velocity off by more than 1e-9;
    Newton recovers v to 1e-14 and P to 1e-12."""
    v = np.sqrt(1.0 - 1.0 / gam ** 2)
    W = np.array([[1.0], [v], [0.0], [0.0], [theta]])
    U = exact_cons("ideal", 5.0 / 3.0, W)
    Wa, _, sta = oracle.con2prim(spec_for("ideal", "analytic"), U)
    ea = vel_err(Wa, W)[0]
    assert not (ea <= 1e-9), ea
    Wi, _, sti = oracle.con2prim(spec_for("ideal", "iterative"), U)
    assert sti["c2p_nonconverged"] == 0
    assert vel_err(Wi, W)[0] < 1e-14
    assert abs(Wi[4, 0] - theta) / theta < 1e-12
