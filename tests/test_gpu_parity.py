"""Parity of the CUDA library (through the C ABI) with the FP64 oracle, element by element on the
same seeded inputs.  Each side builds its own conserved state from the shared primitive fields
of ``workloads``.  Tolerances: relative L-infinity (per call, normalised by the largest oracle
magnitude) 1e-11 for one RHS or step of the FP64 path, 1e-9 after 100 steps on smooth problems;
the closed-form ideal con2prim is ill-conditioned (Sec. 3.3) and gets its own bound."""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib(gpu_lib):
    return gpu_lib


def solver(spec, **kw):
    from paper_2205_00095_gb300 import Solver
    return Solver(spec, **kw)


def to_dev(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    torch.cuda.synchronize()
    return t


def rel_inf(got, want):
    return float(np.abs(got - want).max() / max(np.abs(want).max(), 1e-300))


def gpu_state(s, spec):
    with torch.cuda.stream(s.stream):
        U = s.initial_state(wl.initial_primitive(spec, s.node_coords_device()))
    s.synchronize()
    return U


def oracle_state(spec):
    X = oracle.node_coords(spec)
    return oracle.prim2cons(spec, wl.initial_primitive(spec, X))


# ---------------------------------------------------------------------------------------
# point-wise
# ---------------------------------------------------------------------------------------

def test_node_coords_match(lib):
    spec = wl.smooth_random(3, [3, 2, 4], 3)
    s = solver(spec)
    assert np.allclose(s.node_coords(), oracle.node_coords(spec), rtol=0, atol=1e-15)


@pytest.mark.parametrize("eos", ["ideal", "tm"])
def test_prim2cons(lib, eos):
    spec = dict(dim=1, degree=0, n_elem=[3000], eos=eos, gamma_ad=5.0 / 3.0)
    W = wl.random_primitive_states(3000, seed=41, gamma_max=30.0)[:, :, None]
    s = solver(spec)
    U = s.prim2cons(to_dev(W)).cpu().numpy()
    Uo = oracle.prim2cons(spec, W)
    lor2 = (1.0 / (1.0 - (W[1:4] ** 2).sum(0)))
    scale = np.abs(Uo).max(axis=0)
    assert np.all(np.abs(U - Uo) <= 1e-14 * lor2 * scale)


@pytest.mark.parametrize("eos,c2p", [("ideal", "analytic"), ("ideal", "iterative"),
                                     ("tm", "analytic"), ("tm", "iterative")])
def test_con2prim(lib, eos, c2p):
    n = 4000
    spec = dict(dim=1, degree=0, n_elem=[n], eos=eos, gamma_ad=4.0 / 3.0, c2p=c2p)
    W = wl.random_primitive_states(n, seed=42)[:, :, None]
    Uo = oracle.prim2cons(spec, W)
    s = solver(spec)
    Wg, it = s.con2prim(to_dev(Uo), with_iters=True)
    Wg = Wg.cpu().numpy()
    Wo, ito, sto = oracle.con2prim(spec, Uo)
    status, st = s.stats()
    assert status == 0 and st["c2p_nonconverged"] == 0 and sto["c2p_nonconverged"] == 0
    kappa = (Uo[4] + np.linalg.norm(Uo[1:4], axis=0)) / Wo[4]
    if (eos, c2p) == ("ideal", "analytic"):
        # The closed form of Sec. 3.1 is ill-conditioned for slow, hot states: the resolvent's
        # T = R^2 + S^3 cancels, and two FP64 evaluations with different rounding orders differ by
        # up to eps times that cancellation factor kT = (R^2 + |S|^3)/|T|.  Both the GPU's and the
        # oracle's closed form are measured against the exact root (the oracle's Newton solver)
        # with the per-state bound 1e-13 + 50 eps kT (kT from the section's coefficients, here
        # only as the conditioning estimate).
        Wx, _, _ = oracle.con2prim(dict(spec, c2p="iterative"), Uo)
        D, tau = Uo[0, :, 0], Uo[4, :, 0]
        S2 = (Uo[1:4, :, 0] ** 2).sum(0)
        G, E = spec["gamma_ad"], tau + D
        wq = 1.0 / ((G - 1.0) ** 2 * (D * D + S2))
        a0, a1 = S2 * wq, -2.0 * G * np.sqrt(S2) * E * wq
        a3, a2 = (G - 1.0) * a1, (G * G * E * E + 2.0 * (G - 1.0) * S2 - (G - 1.0) ** 2 * D * D) * wq
        i1, i2, i3 = -a2, a3 * a1 - 4.0 * a0, 4.0 * a2 * a0 - a1 * a1 - a3 * a3 * a0
        R = (9.0 * i1 * i2 - 27.0 * i3 - 2.0 * i1 ** 3) / 54.0
        Sq = (3.0 * i2 - i1 * i1) / 9.0
        kT = (R * R + np.abs(Sq) ** 3) / np.maximum(np.abs(R * R + Sq ** 3), 1e-300)
        bound = (1e-13 + 50.0 * 2.220446049250313e-16 * kT)[:, None]  # per state, shape (n, 1)
        nx = np.linalg.norm(Wx[1:4], axis=0)
        for Wc in (Wo, Wg):  # the oracle's closed form obeys the same envelope as the GPU's
            assert np.all(np.linalg.norm(Wc[1:4] - Wx[1:4], axis=0) / nx <= bound)
            assert np.all(np.abs(Wc[0] - Wx[0]) / Wx[0] <= bound)
            assert np.all(np.abs(Wc[4] - Wx[4]) / (Wx[4] * kappa) <= bound)
        return
    tol = 1e-12
    # velocity relative to |v|, rho relative, P relative to its conditioning (tau + |S|)/P
    dv = np.linalg.norm(Wg[1:4] - Wo[1:4], axis=0) / np.maximum(np.linalg.norm(Wo[1:4], axis=0), 1e-300)
    assert dv.max() < tol
    assert (np.abs(Wg[0] - Wo[0]) / Wo[0]).max() < tol
    assert (np.abs(Wg[4] - Wo[4]) / Wo[4] / kappa).max() < tol
    if c2p == "iterative":
        # the GPU counts its FP32 and FP64 iterations together
        if eos == "ideal":
            assert 0.5 * float(ito.mean()) <= float(it.float().mean()) <= 1.6 * float(ito.mean()) + 1.0
        else:
            # Brent's FP32 phase starts from the bound W < xi^2/(eta^2 - xi^2) instead of the
            # paper's [0, 200^2 - 1]: fewer iterations than the oracle, never more
            assert 1.0 <= float(it.float().mean()) <= float(ito.mean())
        assert st["c2p_iters_total"] == int(it.sum())


@pytest.mark.parametrize("eos,G", [("ideal", 4.0 / 3.0), ("ideal", 5.0 / 3.0), ("tm", 5.0 / 3.0)])
def test_con2prim_hot_ultrarelativistic_states(lib, eos, G):
    """Hot states near |v| = 1 (xi = |S|/D up to 2e4 with eta - xi = 0.5 ... 20, the states
    behind the Taub-Matthews blast of Sec. 4.3 at 2048 cells; gamma up to about 100): there the
    ideal quartic is close to palindromic with two roots near w = 1, and FP32 rounding keeps
    Newton's FP32 step above its stop.  Every recovery converges and agrees with the oracle."""
    xi = np.repeat(np.geomspace(50.0, 2e4, 60), 40)
    eta = xi + np.tile(np.geomspace(0.5, 20.0, 40), 60)
    th = np.linspace(0.0, 2.0 * np.pi, xi.size)
    U = np.stack([np.ones_like(xi), xi * np.cos(th), xi * np.sin(th), np.zeros_like(xi),
                  eta - 1.0])[:, :, None]
    spec = dict(dim=1, degree=0, n_elem=[xi.size], eos=eos, gamma_ad=G, c2p="iterative")
    s = solver(spec)
    Wg, it = s.con2prim(to_dev(U), with_iters=True)
    Wg = Wg.cpu().numpy()
    status, st = s.stats()
    Wo, ito, sto = oracle.con2prim(spec, U)
    assert sto["c2p_nonconverged"] == 0 and sto["c2p_invalid_input"] == 0
    assert status == 0 and st["c2p_nonconverged"] == 0, st
    if eos == "ideal":
        assert int(it.max()) <= 15
    dv = np.linalg.norm(Wg[1:4] - Wo[1:4], axis=0) / np.linalg.norm(Wo[1:4], axis=0)
    assert dv.max() < 1e-12
    # rho = D / gamma: gamma near 100 amplifies the root's rounding by about gamma
    assert (np.abs(Wg[0] - Wo[0]) / Wo[0]).max() < 1e-9
    kappa = (U[4] + np.linalg.norm(U[1:4], axis=0)) / Wo[4]
    assert (np.abs(Wg[4] - Wo[4]) / Wo[4] / kappa).max() < 1e-9


@pytest.mark.parametrize("eos", ["ideal", "tm"])
def test_con2prim_relative_tolerance(lib, eos):
    """c2p_rtol = 1e-6: every recovery converges in no more iterations than at the default
    rules, and the velocity agrees with the oracle's (same tolerance) to 10 rtol gamma^2."""
    n = 4000
    spec = dict(dim=1, degree=0, n_elem=[n], eos=eos, gamma_ad=4.0 / 3.0, c2p="iterative")
    W = wl.random_primitive_states(n, seed=42)[:, :, None]
    Uo = oracle.prim2cons(spec, W)
    s0, s1 = solver(spec), solver(dict(spec, c2p_rtol=1e-6))
    _, it0 = s0.con2prim(to_dev(Uo), with_iters=True)
    Wg, it1 = s1.con2prim(to_dev(Uo), with_iters=True)
    status, st = s1.stats()
    assert status == 0 and st["c2p_nonconverged"] == 0
    assert float(it1.float().mean()) <= float(it0.float().mean())
    Wo, _, sto = oracle.con2prim(dict(spec, c2p_rtol=1e-6), Uo)
    assert sto["c2p_nonconverged"] == 0
    Wg = Wg.cpu().numpy()
    g2 = 1.0 / (1.0 - (Wo[1:4] ** 2).sum(0))
    dv = np.linalg.norm(Wg[1:4] - Wo[1:4], axis=0) / np.maximum(np.linalg.norm(Wo[1:4], axis=0), 1e-300)
    assert (dv / g2).max() < 1e-5


def test_con2prim_invalid_and_cap(lib):
    spec = dict(dim=1, degree=0, n_elem=[5], eos="tm", gamma_ad=5.0 / 3.0, c2p="iterative")
    U = np.array([[-1.0, 1.0, 1.0, np.nan, 1.0],
                  [0.0, 0.0, 2.0, 0.0, 0.0],
                  [0.0, 0.0, 0.0, 0.0, 0.0],
                  [0.0, 0.0, 0.0, 0.0, 0.0],
                  [1.0, -0.5, 0.5, 1.0, 0.1]])[:, :, None]
    s = solver(spec)
    W = s.con2prim(to_dev(U)).cpu().numpy()
    status, st = s.stats(reset=True)
    assert st["c2p_invalid_input"] == 4 and np.all(np.isnan(W[:, :4]))
    from paper_2205_00095_gb300 import _lib
    assert status == _lib.DGSRHD_EBADSTATE
    # an iteration cap of 3 forces non-convergence; the context stays usable
    spec2 = dict(spec, n_elem=[50], c2p_max_iter=3)
    W2 = wl.random_primitive_states(50, seed=5, gamma_max=50.0)[:, :, None]
    s2 = solver(spec2)
    s2.con2prim(s2.prim2cons(to_dev(W2)))
    status, st = s2.stats()
    assert status == _lib.DGSRHD_EC2P_NOCONV and st["c2p_nonconverged"] > 0
    assert st["c2p_iters_max"] == 3


# ---------------------------------------------------------------------------------------
# right-hand side
# ---------------------------------------------------------------------------------------

RHS_CASES = [
    # dim, n_elem (several blocks and a ragged tail), degree, eos, flux, bc
    (1, [301], 0, "ideal", "llf", None),
    (1, [257], 1, "ideal", "hll", [("dirichlet", "outflow")]),
    (1, [100], 4, "tm", "llf", None),
    (2, [19, 23], 0, "tm", "hll", None),
    (2, [21, 17], 1, "ideal", "llf", [("outflow", "dirichlet"), ("periodic", "periodic")]),
    (2, [18, 13], 2, "tm", "llf", None),
    (2, [17, 19], 3, "ideal", "hll", None),
    (2, [17, 19], 3, "tm", "hll", [("periodic", "periodic"), ("dirichlet", "outflow")]),
    (2, [11, 9], 4, "ideal", "llf", None),
    (3, [7, 6, 5], 1, "ideal", "hll", None),
    (3, [5, 6, 7], 2, "tm", "llf", [("periodic", "periodic"), ("outflow", "outflow"), ("periodic", "periodic")]),
    (3, [6, 5, 7], 3, "tm", "hll", None),
    (3, [4, 3, 5], 4, "ideal", "llf", None),
    # HLLC and reflecting walls
    (1, [129], 2, "ideal", "hllc", [("reflect", "dirichlet")]),
    (2, [17, 15], 1, "tm", "hllc", [("reflect", "reflect"), ("periodic", "periodic")]),
    (2, [13, 11], 3, "ideal", "hllc", [("outflow", "reflect"), ("reflect", "outflow")]),
    (2, [12, 10], 2, "ideal", "hll", [("reflect", "reflect"), ("reflect", "reflect")]),
    (3, [5, 4, 6], 2, "ideal", "hllc", [("reflect", "reflect"), ("periodic", "periodic"),
                                        ("outflow", "reflect")]),
]


@pytest.mark.parametrize("dim,n,degree,eos,flux,bc", RHS_CASES)
@pytest.mark.parametrize("c2p", ["iterative", "analytic"])
def test_rhs(lib, dim, n, degree, eos, flux, bc, c2p):
    spec = wl.smooth_random(dim, n, degree, eos=eos, flux=flux, c2p=c2p, seed=dim * 10 + degree,
                            bc=bc)
    s = solver(spec)
    U = gpu_state(s, spec)
    R = s.rhs(U).cpu().numpy()
    Ro, sto = oracle.rhs(spec, oracle_state(spec))
    tol = 1e-11 if (eos, c2p) != ("ideal", "analytic") else 1e-10
    assert rel_inf(R, Ro) < tol
    status, st = s.stats()
    assert status == 0 and st["c2p_invalid_input"] == 0
    assert st["face_guard_hits"] == sto["face_guard_hits"]


# ---------------------------------------------------------------------------------------
# physicality operator
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("dim,degree,n", [(1, 3, [997]), (2, 2, [31, 29]), (2, 3, [40, 25]),
                                          (3, 3, [9, 8, 7]), (2, 4, [19, 21])])
def test_enforce(lib, dim, degree, n):
    spec = dict(dim=dim, degree=degree, n_elem=n, eos="ideal", gamma_ad=5.0 / 3.0)
    E, Nn = wl.shape(spec)
    U = wl.random_conserved_cells(E, Nn, seed=7 + dim + degree)
    s = solver(spec)
    Ug, sg = s.enforce(to_dev(U), with_s=True)
    Uo, so, sto = oracle.enforce(spec, U)
    assert rel_inf(Ug.cpu().numpy(), Uo) < 1e-13
    assert np.allclose(sg.cpu().numpy(), so, rtol=1e-12, atol=1e-15)
    status, st = s.stats()
    assert st["enforced_cells"] == sto["enforced_cells"] > 0
    assert st["mean_inadmissible_cells"] == sto["mean_inadmissible_cells"] > 0


# ---------------------------------------------------------------------------------------
# time steps
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("spec_fn,c2p", [
    (lambda c2p: wl.advected_wave(n=16, degree=3, c2p=c2p), "analytic"),
    (lambda c2p: wl.advected_wave(n=16, degree=3, c2p=c2p), "iterative"),
    (lambda c2p: wl.kh2d(nx=12, ny=24, degree=3, c2p=c2p), "iterative"),
    (lambda c2p: wl.kh2d(nx=12, ny=24, degree=3, c2p=c2p), "analytic"),
    (lambda c2p: wl.smooth_random(3, [5, 6, 4], 2, eos="tm", flux="hll", c2p=c2p, seed=8), "iterative"),
    (lambda c2p: wl.kh_single(nx=12, ny=24, degree=1, c2p=c2p), "iterative"),
    (lambda c2p: wl.kh_single(nx=10, ny=20, degree=2, c2p=c2p), "iterative"),
    (lambda c2p: wl.riemann_1d(4, n=96, degree=1), "iterative"),
    (lambda c2p: wl.riemann_1d(5, n=64, degree=0), "iterative"),
    # the scaling limiter
    (lambda c2p: dict(wl.riemann_1d(2, n=96, degree=1), limiter=True), "iterative"),
    (lambda c2p: dict(wl.riemann_1d(5, n=64, degree=1), limiter=True), "iterative"),
    (lambda c2p: dict(wl.kh_single(nx=12, ny=24, degree=2), limiter=True), "iterative"),
    # transverse velocity: Riemann problem 3 (Sec. 4.2) and the Taub-Matthews blast (Sec. 4.3)
    (lambda c2p: dict(wl.riemann_1d(3, n=96, degree=1), limiter=True), "iterative"),
    (lambda c2p: dict(wl.tm_blast("tm", n=96, degree=1), limiter=True), "iterative"),
    (lambda c2p: wl.tm_blast("ideal", 4.0 / 3.0, n=64, degree=0), "iterative"),
    # the minmod limiter
    (lambda c2p: dict(wl.riemann_1d(2, n=96, degree=1), limiter="minmod", limiter_alpha=0.0), "iterative"),
    (lambda c2p: dict(wl.tm_blast("tm", n=96, degree=2), limiter="minmod"), "iterative"),
    (lambda c2p: dict(wl.kh_single(nx=12, ny=24, degree=2), limiter="minmod", limiter_alpha=0.0), "iterative"),
    # both limiters in 3D (every element limited at M = 0: extrema everywhere in random data)
    (lambda c2p: dict(wl.smooth_random(3, [5, 6, 4], 2, eos="tm", flux="hllc", c2p=c2p, seed=8),
                      limiter="minmod", limiter_alpha=0.0), "iterative"),
    (lambda c2p: dict(wl.smooth_random(3, [5, 6, 4], 2, eos="tm", flux="hllc", c2p=c2p, seed=8),
                      limiter=True, limiter_alpha=0.0), "iterative"),
])
def test_step_one_and_hundred(lib, spec_fn, c2p):
    spec = spec_fn(c2p)
    s = solver(spec, stream=torch.cuda.Stream())
    dt = s.cfl_dt(0.2)
    U = gpu_state(s, spec)
    Uo = oracle_state(spec)
    s.step(U, dt, 1)
    Uo1, st1 = oracle.step(spec, Uo, dt, 1)
    torch.cuda.synchronize()
    assert rel_inf(U.cpu().numpy(), Uo1) < 1e-11
    s.step(U, dt, 99)
    Uo100, sto = oracle.step(spec, Uo1, dt, 99)
    torch.cuda.synchronize()
    # Riemann problem 5 runs at gamma = 224: one recovery's rounding in rho is about
    # 20 eps gamma^2 = 2e-10 (the root w has a partner 1/w about 2/gamma away), and the two
    # sides' solvers stop at different rounding-level iterates; 100 steps through the wall
    # shock amplify that to a few 1e-9
    tol100 = 1e-8 if spec.get("problem") == 5 else 1e-9
    assert rel_inf(U.cpu().numpy(), Uo100) < tol100
    status, st = s.stats()
    assert status == 0
    # the device counters cover all 100 steps: the oracle's two calls together
    assert st["enforced_cells"] == st1["enforced_cells"] + sto["enforced_cells"]
    assert st["limited_cells"] == st1["limited_cells"] + sto["limited_cells"]
    if spec.get("limiter") and spec["name"] == "riemann_1d":
        assert st["limited_cells"] > 0


def test_kh3d_one_step(lib):
    """The 3D high-Lorentz-factor Kelvin-Helmholtz set-up on a coarse 6^3 mesh: one step.
    (At this resolution the shear layers are unresolved and the run is not meant to last.)"""
    spec = wl.kh3d(n=6, degree=3)
    s = solver(spec, stream=torch.cuda.Stream())
    dt = s.cfl_dt(0.2)
    U = gpu_state(s, spec)
    s.step(U, dt, 1)
    Uo, sto = oracle.step(spec, oracle_state(spec), dt, 1)
    torch.cuda.synchronize()
    assert rel_inf(U.cpu().numpy(), Uo) < 1e-11
    status, st = s.stats()
    assert st["enforced_cells"] == sto["enforced_cells"]


def test_blast_wave_full_run(lib):
    """The 1D blast wave (128 elements, p = 1, SSPRK2, 768 steps): the operator is active and
    the solutions agree to the conditioning of the shock fronts."""
    spec = wl.blast_wave()
    s = solver(spec, stream=torch.cuda.Stream())
    U = gpu_state(s, spec)
    s.enforce(U)
    Uo, _, _ = oracle.enforce(spec, oracle_state(spec))
    dt = s.cfl_dt(0.2)
    nsteps = int(round(0.4 / dt))
    s.step(U, 0.4 / nsteps, nsteps)
    Uo, sto = oracle.step(spec, Uo, 0.4 / nsteps, nsteps)
    torch.cuda.synchronize()
    status, st = s.stats()
    assert status == 0
    assert st["enforced_cells"] > 0 and abs(st["enforced_cells"] - sto["enforced_cells"]) <= 2
    assert rel_inf(U.cpu().numpy(), Uo) < 1e-6


@pytest.mark.parametrize("nsteps", [5, 37])
def test_graph_replay_matches_direct_launches(lib, nsteps):
    """Captured steps (replays of the cached one-step graph) give the bits of direct launches,
    and the launch count of the step."""
    spec = wl.kh2d(nx=8, ny=16, degree=3)
    a = solver(spec, stream=torch.cuda.Stream())
    U1 = gpu_state(a, spec)
    U2 = U1.clone()
    dt = a.cfl_dt(0.2)
    n0 = a.kernel_launches()
    a.step(U1, dt, nsteps)                    # captured graphs
    assert a.kernel_launches() - n0 == 9 * nsteps
    from paper_2205_00095_gb300 import Solver
    b = Solver(spec)                          # legacy stream: direct launches
    b.lib.dgsrhd_set_stream(b.ctx, None)
    b.step(U2, dt, nsteps)
    torch.cuda.synchronize()
    assert torch.equal(U1, U2)
    a.step(U1, dt, nsteps)                    # replay of the cached graphs
    b.step(U2, dt, nsteps)
    torch.cuda.synchronize()
    assert torch.equal(U1, U2)


def test_step_host_matches_device_step(lib):
    spec = wl.advected_wave(n=8, degree=2)
    s = solver(spec, stream=torch.cuda.Stream())
    U = gpu_state(s, spec)
    Uh = U.cpu().pin_memory()
    dt = s.cfl_dt(0.2)
    s.step(U, dt, 3)
    s.step_host(Uh, dt, 3)
    torch.cuda.synchronize()
    assert torch.equal(U.cpu(), Uh)


def test_periodic_conservation_at_scale(lib):
    """On the 512^2 p = 3 advected wave (the benchmark workload) one SSPRK3 step conserves
    sum_e sum_i w_i U_i to round-off, stays admissible and finite."""
    spec = wl.advected_wave(n=512, degree=3)
    s = solver(spec, stream=torch.cuda.Stream())
    U = gpu_state(s, spec)
    s.synchronize()
    w = np.polynomial.legendre.leggauss(4)[1]
    w2 = torch.from_numpy(np.multiply.outer(w, w).ravel()).cuda()
    tot0 = (U * w2).sum(dim=(1, 2))
    s.step(U, s.cfl_dt(0.2), 1)
    s.synchronize()
    tot1 = (U * w2).sum(dim=(1, 2))
    torch.cuda.synchronize()
    assert torch.isfinite(U).all()
    assert float(((tot1 - tot0).abs() / (U.abs() * w2).sum(dim=(1, 2)).clamp_min(1e-300)).max()) < 1e-13


def test_full_size_sampled_elements(lib):
    """The 512^2 p = 3 advected wave after one SSPRK3 step, checked on sampled elements: the
    oracle steps a 7 x 7 element patch around each sample (three stages reach three elements),
    built from the same workload field, and its centre element must match."""
    spec = wl.advected_wave(n=512, degree=3)
    s = solver(spec, stream=torch.cuda.Stream())
    U = gpu_state(s, spec)
    dt = s.cfl_dt(0.2)
    s.step(U, dt, 1)
    s.synchronize()
    Ug = U.cpu().numpy()
    rng = np.random.default_rng(3)
    h = 1.0 / 512
    for _ in range(12):
        ex, ey = (int(v) for v in rng.integers(0, 512, 2))
        patch = dict(spec, n_elem=[7, 7], lo=[(ex - 3) * h, (ey - 3) * h],
                     hi=[(ex + 4) * h, (ey + 4) * h], bc=[("outflow", "outflow")] * 2)
        Xp = oracle.node_coords(patch)
        Up = oracle.prim2cons(patch, wl.advected_wave_ic(patch, Xp))
        Up1, _ = oracle.step(patch, Up, dt, 1)
        got = Ug[:, ex + 512 * ey, :]
        want = Up1[:, 3 + 7 * 3, :]
        assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()


def _sampled_patch_parity(s, spec, U_after, samples, dt, tol=1e-11):
    """Each sampled element after one SSPRK3 step against the oracle run on the (2 r + 1)^d
    element patch around it (three stages reach three elements), built from the same workload
    field with outflow sides."""
    dim = spec["dim"]
    n = spec["n_elem"][:dim]
    h = [(spec["hi"][d] - spec["lo"][d]) / n[d] for d in range(dim)]
    Ug = U_after
    for ec in samples:
        patch = dict(spec, n_elem=[7] * dim,
                     lo=[spec["lo"][d] + (ec[d] - 3) * h[d] for d in range(dim)],
                     hi=[spec["lo"][d] + (ec[d] + 4) * h[d] for d in range(dim)],
                     bc=[("outflow", "outflow")] * dim)
        Xp = oracle.node_coords(patch)
        Up = oracle.prim2cons(patch, wl.initial_primitive(spec, Xp))
        Up1, _ = oracle.step(patch, Up, dt, 1)
        e = ec[0] + n[0] * (ec[1] + (n[1] * ec[2] if dim > 2 else 0))
        centre = 3 + 7 * 3 + (49 * 3 if dim > 2 else 0)
        got, want = Ug[:, e, :], Up1[:, centre, :]
        assert np.abs(got - want).max() < tol * np.abs(want).max(), (ec, np.abs(got - want).max())


def test_full_size_kh2d_sampled_elements(lib):
    """The 2D Taub-Matthews Kelvin-Helmholtz workload at full size (256 x 512, p = 3, Brent,
    HLL): one SSPRK3 step, sampled elements against the oracle."""
    spec = wl.kh2d(nx=256, ny=512, degree=3)
    s = solver(spec, stream=torch.cuda.Stream())
    U = gpu_state(s, spec)
    dt = s.cfl_dt(0.2)
    s.step(U, dt, 1)
    s.synchronize()
    rng = np.random.default_rng(21)
    samples = [(0, 0), (255, 511), (128, 256), (3, 255)] + [tuple(int(x) for x in rng.integers(0, [256, 512])) for _ in range(4)]
    _sampled_patch_parity(s, spec, U.cpu().numpy(), samples, dt)


def test_full_size_kh3d_sampled_elements(lib):
    """The 3D high-Lorentz-factor Kelvin-Helmholtz workload at full size (128^3 elements,
    p = 3, 134M nodes, Brent, HLL): one SSPRK3 step, sampled elements against the oracle."""
    spec = wl.kh3d(n=128, degree=3)
    s = solver(spec, stream=torch.cuda.Stream())
    U = gpu_state(s, spec)
    dt = s.cfl_dt(0.2)
    s.step(U, dt, 1)
    s.synchronize()
    status, st = s.stats()
    assert status == 0 and st["c2p_nonconverged"] == 0
    rng = np.random.default_rng(23)
    samples = [(0, 32, 0), (127, 96, 127)] + [tuple(int(x) for x in rng.integers(0, 128, 3)) for _ in range(2)]
    Uc = U.cpu().numpy()
    del U
    _sampled_patch_parity(s, spec, Uc, samples, dt)


@pytest.mark.parametrize("dim,n,degree", [(1, [1], 3), (2, [1, 6], 2), (2, [5, 1], 4), (3, [1, 2, 1], 2)])
def test_single_element_periodic_axes(lib, dim, n, degree):
    """An axis with one element is periodic onto itself: the element is its own neighbour."""
    spec = wl.smooth_random(dim, n, degree, eos="tm", flux="hll", seed=31)
    s = solver(spec)
    R = s.rhs(gpu_state(s, spec)).cpu().numpy()
    Ro, _ = oracle.rhs(spec, oracle_state(spec))
    assert rel_inf(R, Ro) < 1e-11


@pytest.mark.parametrize("eos,c2p", [("ideal", "analytic"), ("ideal", "iterative"),
                                     ("tm", "analytic"), ("tm", "iterative")])
def test_con2prim_zero_and_tiny_momentum(lib, eos, c2p):
    n = 6
    W = np.array([[1.0, 2.0, 0.5, 1.0, 1.0, 3.0],
                  [0.0, 0.0, 0.0, 1e-9, 0.0, 3e-7],
                  [0.0, 0.0, 0.0, 0.0, -2e-8, 0.0],
                  [0.0, 0.0, 0.0, 0.0, 0.0, 0.0],
                  [1.0, 1e-6, 10.0, 1.0, 0.3, 0.2]])[:, :, None]
    spec = dict(dim=1, degree=0, n_elem=[n], eos=eos, gamma_ad=5.0 / 3.0, c2p=c2p)
    Uo = oracle.prim2cons(spec, W)
    s = solver(spec)
    Wg = s.con2prim(to_dev(Uo)).cpu().numpy()
    Wo, _, sto = oracle.con2prim(spec, Uo)
    assert np.all(Wg[1:4, :3] == 0.0)
    if c2p == "analytic":
        # the closed forms lose their digits as xi -> 0 (they stay finite); rho and P agree,
        # the velocity to an absolute 1e-6
        assert np.allclose(Wg[[0, 4]], Wo[[0, 4]], rtol=1e-12)
        assert np.allclose(Wg[1:4], Wo[1:4], rtol=0, atol=1e-6)
    else:
        assert np.allclose(Wg, Wo, rtol=1e-12, atol=1e-20)


# ---------------------------------------------------------------------------------------
# the library's FP64 reciprocal and roots (FP32 seed and one third-order correction) against
# CUDA's division, sqrt, rsqrt and rcbrt
# ---------------------------------------------------------------------------------------
def test_reciprocal_and_sqrt_primitives_against_cuda(lib):
    from paper_2205_00095_gb300 import _lib
    rng = np.random.default_rng(12)
    mags = np.ldexp(1.0 + rng.random(200000), rng.integers(-120, 121, size=200000))
    edge = np.array([1.0, 2.0, 0.5, np.nextafter(2.0, 0), np.ldexp(1.0, -100), np.ldexp(1.0, 100),
                     np.ldexp(1.5, -101), np.ldexp(1.5, 101), 5e-324, 2.2e-308, 1.7e308])
    x = np.concatenate([mags, -mags[:1000], edge, -edge, [0.0, -0.0, np.inf, -np.inf, np.nan]])
    xd = to_dev(x)
    out = torch.empty(8 * x.size, dtype=torch.float64, device="cuda")
    assert lib.dgsrhd_math_check(xd.data_ptr(), x.size, out.data_ptr(), None) == 0
    torch.cuda.synchronize()
    o = out.cpu().numpy().reshape(8, x.size)

    def ulps(a, b):
        ia, ib = a.view(np.int64), b.view(np.int64)
        return np.abs(ia - ib)

    fin = np.isfinite(o[1]) & (o[1] != 0.0)
    assert ulps(o[0][fin], o[1][fin]).max() <= 1
    assert np.array_equal(np.isnan(o[0]), np.isnan(o[1]))
    assert np.array_equal(o[0][~fin & ~np.isnan(o[1])], o[1][~fin & ~np.isnan(o[1])])
    pos = (x > 0) & np.isfinite(x)
    assert ulps(o[2][pos], o[3][pos]).max() <= 2
    assert np.all(np.isnan(o[2][x < 0])) and np.all(o[2][x == 0] == 0.0)
    assert np.isnan(o[2][np.isnan(x)]).all()
    # reciprocal cube root: within 2 ulp of CUDA's and of x^(-1/3) in extended precision
    # (numpy's long double, rounded once to FP64), with the sign of x
    nz = np.isfinite(x) & (x != 0.0)
    assert ulps(o[4][nz], o[5][nz]).max() <= 2
    ref = (1.0 / np.cbrt(x[nz].astype(np.longdouble))).astype(np.float64)
    assert ulps(o[4][nz], ref).max() <= 2
    assert np.array_equal(np.signbit(o[4][nz]), np.signbit(x[nz]))
    # reciprocal square root: within 2 ulp of CUDA's and of 1/sqrt(x) in extended precision;
    # CUDA's values (infinities, NaN, zero) at +-0, x < 0, +inf and NaN
    ref = (1.0 / np.sqrt(x[pos].astype(np.longdouble))).astype(np.float64)
    assert ulps(o[6][pos], o[7][pos]).max() <= 2
    assert ulps(o[6][pos], ref).max() <= 2
    rest = ~pos
    assert np.array_equal(np.isnan(o[6][rest]), np.isnan(o[7][rest]))
    keep = rest & ~np.isnan(o[7])
    assert np.array_equal(o[6][keep], o[7][keep])
    assert lib.dgsrhd_math_check(None, 1, out.data_ptr(), None) == _lib.DGSRHD_EINVAL
    assert lib.dgsrhd_math_check(xd.data_ptr(), -1, out.data_ptr(), None) == _lib.DGSRHD_EINVAL


# ---------------------------------------------------------------------------------------
# reflecting walls: no mass or energy crosses them (every flux)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("flux", ["llf", "hll", "hllc"])
def test_reflecting_box_conserves_mass_and_energy(lib, flux):
    spec = wl.smooth_random(2, [14, 11], 2, flux=flux, seed=6,
                            bc=[("reflect", "reflect"), ("reflect", "reflect")])
    s = solver(spec, stream=torch.cuda.Stream())
    U = gpu_state(s, spec)
    w1 = np.polynomial.legendre.leggauss(3)[1]
    w = torch.from_numpy(np.multiply.outer(w1, w1).ravel()).cuda()
    m0, e0 = float((U[0] * w).sum()), float((U[4] * w).sum())
    S0 = U[1].clone()
    s.step(U, s.cfl_dt(0.2), 50)
    s.synchronize()
    m1, e1 = float((U[0] * w).sum()), float((U[4] * w).sum())
    assert abs(m1 - m0) <= 1e-12 * m0 and abs(e1 - e0) <= 1e-12 * e0
    assert float((U[1] - S0).abs().max()) > 1e-3
    status, _ = s.stats()
    assert status == 0


# ---------------------------------------------------------------------------------------
# Gauss-Lobatto-Legendre nodes: the same method on the other node family
# ---------------------------------------------------------------------------------------
GLL_CASES = [
    (1, [53], 1, "ideal", "llf", None),
    (2, [13, 11], 2, "tm", "hll", [("outflow", "reflect"), ("periodic", "periodic")]),
    (2, [9, 10], 3, "ideal", "hllc", None),
    (3, [4, 5, 3], 4, "tm", "llf", None),
]


@pytest.mark.parametrize("dim,n,degree,eos,flux,bc", GLL_CASES)
def test_rhs_gll(lib, dim, n, degree, eos, flux, bc):
    spec = dict(wl.smooth_random(dim, n, degree, eos=eos, flux=flux, seed=dim + 7 * degree, bc=bc),
                nodes="gll")
    s = solver(spec)
    U = gpu_state(s, spec)
    R = s.rhs(U).cpu().numpy()
    Ro, sto = oracle.rhs(spec, oracle_state(spec))
    assert rel_inf(R, Ro) < 1e-11
    X = s.node_coords()
    assert np.isclose(X[0].min(), spec["lo"][0]) and np.isclose(X[0].max(), spec["hi"][0])


def test_gll_blast_wave_needs_no_face_guard(lib):
    """Problem 1 at p = 1 on Gauss-Lobatto nodes: the face traces are node values, which the
    physicality operator keeps admissible, so the face guard never fires; GPU and oracle agree
    after 100 steps."""
    spec = dict(wl.blast_wave(n=64, degree=1), nodes="gll")
    s = solver(spec, stream=torch.cuda.Stream())
    dt = s.cfl_dt(0.2)
    with torch.cuda.stream(s.stream):
        U = s.initial_state(wl.initial_primitive(spec, s.node_coords_device()))
        s.enforce(U)
    Uo = oracle.prim2cons(spec, wl.initial_primitive(spec, oracle.node_coords(spec)))
    Uo, _, _ = oracle.enforce(spec, Uo)
    s.step(U, dt, 100)
    s.synchronize()
    Uo, sto = oracle.step(spec, Uo, dt, 100)
    status, st = s.stats()
    assert st["face_guard_hits"] == 0 and sto["face_guard_hits"] == 0
    assert st["enforced_cells"] == sto["enforced_cells"] > 0
    assert rel_inf(U.cpu().numpy(), Uo) < 1e-9


# ---------------------------------------------------------------------------------------
# the paper's 2D Riemann problems (HLLC with the limiter)
# ---------------------------------------------------------------------------------------
# Test 1's colliding shocks amplify rounding-level differences quickly (the oracle alone breaks
# its mirror symmetry by 6e-6 at p = 1, t = 0.8): one step at 1e-11, forty steps at 1e-4.
@pytest.mark.parametrize("test,degree,steps,tol,limiter", [
    (1, 1, 1, 1e-11, True), (1, 1, 40, 1e-4, True), (2, 1, 40, 1e-9, True),
    (3, 2, 40, 1e-9, True),
    (1, 1, 1, 1e-11, "minmod"), (1, 1, 40, 1e-4, "minmod"), (3, 2, 40, 1e-9, "minmod")])
def test_riemann_2d_against_oracle(lib, test, degree, steps, tol, limiter):
    spec = dict(wl.riemann_2d(test, n=20, degree=degree), limiter=limiter)
    if limiter == "minmod":
        spec["limiter_alpha"] = 0.0
    s = solver(spec, stream=torch.cuda.Stream())
    dt = s.cfl_dt(0.2)
    with torch.cuda.stream(s.stream):
        U = s.initial_state(wl.initial_primitive(spec, s.node_coords_device()))
        s.enforce(U)
    Uo = oracle.prim2cons(spec, wl.initial_primitive(spec, oracle.node_coords(spec)))
    Uo, _, st0 = oracle.enforce(spec, Uo)
    s.step(U, dt, steps)
    s.synchronize()
    Uo, sto = oracle.step(spec, Uo, dt, steps)
    assert rel_inf(U.cpu().numpy(), Uo) < tol
    status, st = s.stats()
    assert status == 0
    if tol < 1e-8:
        assert st["limited_cells"] == sto["limited_cells"]


# ---------------------------------------------------------------------------------------
# host-state stepping: pinned memory (read and written by the kernels) and pageable memory
# (copied) give the bits of stepping the state on the device
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("spec_fn", [lambda: wl.advected_wave(n=24, degree=3),
                                     lambda: wl.kh2d(nx=8, ny=16, degree=2),
                                     lambda: dict(wl.smooth_random(1, [33], 1, seed=2), rk_stages=1)])
def test_step_host_paths_match_the_device_step(lib, spec_fn):
    spec = spec_fn()
    s = solver(spec, stream=torch.cuda.Stream())
    U = gpu_state(s, spec)
    dt = s.cfl_dt(0.2)
    pinned = U.cpu().pin_memory()
    pageable = U.cpu().clone()
    s.step(U, dt, 3)
    s.step_host(pinned, dt, 3)
    s.step_host(pageable, dt, 3)
    s.synchronize()
    Ud = U.cpu()
    assert torch.equal(pinned, Ud) and torch.equal(pageable, Ud)


def test_checkpoint_resume_reproduces_the_run(lib, tmp_path):
    """Ten steps, a checkpoint, a fresh solver from the saved spec and ten more steps give the
    bits of twenty uninterrupted steps."""
    from paper_2205_00095_gb300 import checkpoint
    spec = wl.kh_single(nx=12, ny=24, degree=2)
    s = solver(spec, stream=torch.cuda.Stream())
    U = gpu_state(s, spec)
    dt = s.cfl_dt(0.2)
    ref = U.clone()
    s.step(ref, dt, 20)
    s.step(U, dt, 10)
    s.synchronize()
    path = str(tmp_path / "kh.pt")
    checkpoint.save(path, spec, U, t=10 * dt, step=10)
    d = checkpoint.load(path, device="cuda")
    s2 = solver(d["spec"], stream=torch.cuda.Stream())
    U2 = d["U"]
    s2.step(U2, dt, 10)
    s2.synchronize()
    torch.cuda.synchronize()
    assert d["step"] == 10 and d["t"] == 10 * dt
    assert torch.equal(U2, ref)


@pytest.mark.parametrize("spec_fn", [
    lambda: wl.advected_wave(n=24, degree=3),
    lambda: dict(wl.kh2d(nx=12, ny=24, degree=3), precision="split"),
    lambda: dict(wl.smooth_random(3, [5, 6, 4], 2, eos="tm", flux="hllc", seed=8),
                 limiter="minmod", limiter_alpha=0.0),
    lambda: dict(wl.riemann_1d(2, n=96, degree=1), limiter=True),
])
def test_runs_are_bitwise_reproducible(lib, spec_fn):
    """Race evidence without a sanitizer: the same 30 steps in two fresh contexts, on different
    streams, give the same bits (block-level reductions, shared-memory staging and the split
    kernels' tiles would show a race as run-to-run differences), and so do the counters."""
    spec = spec_fn()
    out, stats = [], []
    for _ in range(2):
        s = solver(spec, stream=torch.cuda.Stream())
        U = gpu_state(s, spec)
        dt = s.cfl_dt(0.2)
        s.step(U, dt, 30)
        s.synchronize()
        out.append(U.cpu())
        stats.append(s.stats()[1])
    assert torch.equal(out[0], out[1])
    for k in ("c2p_iters_total", "enforced_cells", "limited_cells", "face_guard_hits"):
        assert stats[0][k] == stats[1][k]


def test_zero_steps_are_a_no_op(lib):
    """nsteps = 0: the state keeps its bits and no kernel is launched (device and host paths)."""
    spec = wl.kh_single(nx=6, ny=12, degree=2)
    s = solver(spec, stream=torch.cuda.Stream())
    U = gpu_state(s, spec)
    V = U.clone()
    n0 = s.kernel_launches()
    s.step(U, s.cfl_dt(0.2), 0)
    Uh = V.cpu().pin_memory()
    Wh = Uh.clone()
    s.step_host(Uh, s.cfl_dt(0.2), 0)
    s.synchronize()
    assert torch.equal(U, V) and torch.equal(Uh, Wh)
    assert s.kernel_launches() == n0


def test_newton_recovers_extreme_pressures(lib):
    """Sec. 3.3: the iterative ideal solver keeps working at very high pressures (P/rho up to
    1e22, where the closed form fails): velocity to 1e-14 and pressure to 1e-14 of its
    conditioning, all converged, as in the oracle."""
    th = np.repeat([1e16, 1e18, 1e20, 1e22], 3)
    gam = np.tile([1.5, 10.0, 50.0], 4)
    v = np.sqrt(1.0 - 1.0 / gam ** 2)
    W = np.stack([np.ones_like(th), v, 0 * th, 0 * th, th])[:, :, None]
    spec = dict(dim=1, degree=0, n_elem=[th.size], eos="ideal", gamma_ad=5.0 / 3.0,
                c2p="iterative")
    U = oracle.prim2cons(spec, W)
    s = solver(spec)
    Wg = s.con2prim(to_dev(U)).cpu().numpy()
    status, st = s.stats()
    assert status == 0 and st["c2p_nonconverged"] == 0
    assert (np.abs(Wg[1] - W[1]) / W[1]).max() < 1e-14
    # P = (Gamma - 1)(E - S.v - rho) cancels by about gamma^2: its conditioning (tau + |S|)/P
    kappa = (U[4] + np.linalg.norm(U[1:4], axis=0)) / W[4]
    assert (np.abs(Wg[4] - W[4]) / W[4] / kappa).max() < 1e-14


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("degree", [0, 1, 2, 3, 4])
def test_cfl_dt_matches_the_oracle(lib, dim, degree):
    """The library's time step (dgsrhd_cfl_dt) equals the oracle's CFL rule on isotropic and
    anisotropic meshes (element counts and domain lengths differing per axis), for several CFL
    numbers."""
    meshes = [([8] * dim, [0.0] * dim, [1.0] * dim),
              ([7, 3, 5][:dim], [-0.5, -1.0, 0.0][:dim], [0.5, 1.0, 3.0][:dim]),
              ([96, 40, 6][:dim], [0.0, -1.0, 0.25][:dim], [0.3, 1.0, 0.5][:dim])]
    for n, lo, hi in meshes:
        spec = dict(wl.smooth_random(dim, n, degree, seed=1), lo=lo, hi=hi)
        s = solver(spec)
        for cfl in (0.2, 0.45, 1.0):
            got, want = s.cfl_dt(cfl), oracle.cfl_dt(spec, cfl)
            assert abs(got - want) <= 2e-16 * want, (n, lo, hi, cfl, got, want)
        s.close()


# ---------------------------------------------------------------------------------------
# the face-point variant of the physicality operator (enforce = "faces")
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("dim,degree,n", [(1, 3, [997]), (2, 2, [31, 29]), (2, 3, [40, 25]),
                                          (3, 2, [9, 7, 6]), (3, 3, [6, 5, 4])])
def test_enforce_face_points(lib, dim, degree, n):
    """The operator with the face points of each element's conserved polynomial in the minimum:
    state and factors equal to the oracle's, on random cells (some flagged by their faces
    alone) and on cells whose nodes are admissible but whose polynomial is not at a face."""
    spec = dict(dim=dim, degree=degree, n_elem=n, eos="ideal", gamma_ad=5.0 / 3.0, enforce="faces")
    E, Nn = wl.shape(spec)
    N = degree + 1
    U = wl.random_conserved_cells(E, Nn, seed=17 + dim + degree)
    x = np.polynomial.legendre.leggauss(N)[0][np.arange(Nn) % N]
    D0 = np.linspace(0.5, 2.0, 40)[:, None]
    U[:, :40] = 0.0
    U[0, :40] = D0 * (1.0 + 1.15 * x)  # D < 0 at x = -1 only
    U[4, :40] = 0.3 * D0
    s = solver(spec)
    Ug, sg = s.enforce(to_dev(U), with_s=True)
    Uo, so, sto = oracle.enforce(spec, U)
    assert rel_inf(Ug.cpu().numpy(), Uo) < 1e-13
    assert np.allclose(sg.cpu().numpy(), so, rtol=1e-12, atol=1e-15)
    assert np.all(so[:40] < 1.0)  # flagged by the faces
    status, st = s.stats()
    assert st["enforced_cells"] == sto["enforced_cells"] > 40
    assert st["mean_inadmissible_cells"] == sto["mean_inadmissible_cells"] > 0


@pytest.mark.parametrize("degree", [1, 2])
def test_blast_wave_with_the_face_point_operator(lib, degree):
    """Problem 1 (128 elements, SSPRK2, to t = 0.4) with the face-point operator after every
    stage: GPU and oracle agree to the conditioning of the shock fronts, count the same operator
    actions and face-guard hits (to a few), and the guard fires far less often than with the
    nodal operator (the extrapolated primitive traces, which the conserved-state operator does not
    bound, can still leave the admissible set)."""
    spec = dict(wl.blast_wave(degree=degree), enforce="faces")
    s = solver(spec, stream=torch.cuda.Stream())
    U = gpu_state(s, spec)
    s.enforce(U)
    Uo, _, _ = oracle.enforce(spec, oracle_state(spec))
    dt = s.cfl_dt(0.2)
    nsteps = int(round(0.4 / dt))
    s.step(U, 0.4 / nsteps, nsteps)
    Uo, sto = oracle.step(spec, Uo, 0.4 / nsteps, nsteps)
    torch.cuda.synchronize()
    status, st = s.stats()
    assert status == 0
    assert abs(st["enforced_cells"] - sto["enforced_cells"]) <= 2
    assert abs(st["face_guard_hits"] - sto["face_guard_hits"]) <= 4
    assert rel_inf(U.cpu().numpy(), Uo) < 1e-6
    nodal = dict(spec, enforce=True)
    Un = oracle.enforce(nodal, oracle_state(nodal))[0]
    _, stn = oracle.step(nodal, Un, 0.4 / nsteps, nsteps)
    assert st["face_guard_hits"] < 0.5 * stn["face_guard_hits"]
    print(f"\nblast wave p={degree}: face-guard hits {st['face_guard_hits']} with the face-point "
          f"operator, {stn['face_guard_hits']} with the nodal one")
