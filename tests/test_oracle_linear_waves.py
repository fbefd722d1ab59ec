"""Linear waves (Sec. 4.1) in the oracle: the eigenpairs are eigenpairs of the oracle's own
flux Jacobian, and the DG solution converges at order p + 1 with the SSP-RK of p + 1 stages,
in 1D and in an oblique 2D box."""
import numpy as np
import pytest

import oracle
import workloads as wl
from tests.linear_wave_support import WAVES, eigenpair, l1_errors, make, order


@pytest.mark.parametrize("wave", WAVES)
def test_eigenpairs_of_the_flux_jacobian(wave):
    """dF/dW r = lambda dU/dW r at the base state, by central differences of the oracle's
    prim->cons and flux along x."""
    spec = dict(dim=1, degree=0, n_elem=[1], eos="ideal", gamma_ad=5.0 / 3.0)
    r, lam = eigenpair(wave)
    W0 = np.array([1.0, 0.0, 0.0, 0.0, 1.0])
    h = 1e-6
    Wp, Wm = W0 + h * np.array(r), W0 - h * np.array(r)
    dF = (oracle.phys_flux(spec, Wp, 0) - oracle.phys_flux(spec, Wm, 0)) / (2 * h)
    U = lambda W: oracle.prim2cons(spec, W.reshape(5, 1, 1))[:, 0, 0]
    dU = (U(Wp) - U(Wm)) / (2 * h)
    assert np.allclose(dF, lam * dU, rtol=0, atol=1e-8 * np.abs(dU).max()), (dF, lam * dU)


def run(frame, wave, degree, n_base, refine):
    spec = make(frame, wave, degree, n_base, refine)
    X = oracle.node_coords(spec)
    U = oracle.prim2cons(spec, wl.linear_wave_ic(spec, X))
    T = spec["t_final"]
    nsteps = int(np.ceil(T / oracle.cfl_dt(spec, spec["cfl"])))
    U, st = oracle.step(spec, U, T / nsteps, nsteps)
    assert st["enforced_cells"] == 0 and st["c2p_nonconverged"] == 0
    return l1_errors(spec, U, T), (spec["hi"][0] - spec["lo"][0]) / spec["n_elem"][0]


@pytest.mark.parametrize("frame,degree,n_base", [("1d", 1, 8), ("1d", 2, 8), ("2d_oblique", 1, 4)])
@pytest.mark.parametrize("wave", ["-", "0(1)", "0(2)", "+"])
def test_linear_wave_converges_at_order_p_plus_one(frame, degree, n_base, wave):
    e1, h1 = run(frame, wave, degree, n_base, 1)
    e2, h2 = run(frame, wave, degree, n_base, 2)
    # D, or for a shear wave the momentum component it perturbs (S_y in 1D, S_x in the oblique
    # box, where the transverse direction (-sin, cos) has an x component)
    k = 0 if wave != "0(2)" else (2 if frame == "1d" else 1)
    q = order(e1[k], e2[k], h1, h2)
    assert q > degree + 1 - 0.35, (q, e1, e2)
