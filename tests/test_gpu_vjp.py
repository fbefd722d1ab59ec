"""The hand-written vector-Jacobian products (through the C ABI) against central finite
differences of the FP64 oracle: the RHS, con2prim, the frozen-factor physicality operator, and
the gradient of the transverse kinetic energy after a checkpointed SSPRK3 rollout of the
Kelvin-Helmholtz set-up with respect to the perturbation amplitude and the nodal initial v_x.
Tolerance: 1e-6 relative (central differences with h = 1e-6)."""
import os

import numpy as np
import pytest
import torch

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu


def dev(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    torch.cuda.synchronize()
    return t


def solver(spec):
    from paper_2205_00095_gb300 import Solver
    return Solver(spec)  # default stream


VJP_CASES = [
    (1, [9], 2, "ideal", "llf", [("dirichlet", "outflow")], "iterative"),
    (1, [7], 3, "tm", "hll", None, "analytic"),
    (2, [5, 4], 3, "tm", "hll", None, "iterative"),
    (2, [4, 5], 1, "ideal", "llf", [("outflow", "outflow"), ("periodic", "periodic")], "analytic"),
    (2, [4, 3], 4, "ideal", "hll", None, "iterative"),
    (3, [3, 3, 2], 2, "tm", "llf", None, "iterative"),
    (2, [5, 4], 2, "ideal", "hll", [("reflect", "outflow"), ("periodic", "periodic")], "iterative"),
    (1, [8], 3, "tm", "llf", [("reflect", "reflect")], "iterative"),
    (1, [9], 2, "ideal", "hllc", [("dirichlet", "reflect")], "iterative"),
    (2, [5, 4], 3, "tm", "hllc", None, "iterative"),
    (3, [3, 2, 3], 2, "ideal", "hllc", None, "iterative"),
]


@pytest.mark.parametrize("dim,n,degree,eos,flux,bc,c2p", VJP_CASES)
def test_rhs_vjp_against_oracle_differences(gpu_lib, dim, n, degree, eos, flux, bc, c2p):
    spec = wl.smooth_random(dim, n, degree, eos=eos, flux=flux, c2p=c2p, seed=3, bc=bc)
    X = oracle.node_coords(spec)
    W = wl.smooth_random_ic(spec, X)
    Uo = oracle.prim2cons(spec, W)
    rng = np.random.default_rng(7)
    V = rng.normal(size=Uo.shape) * np.abs(Uo).mean(axis=(1, 2), keepdims=True)
    Rb = rng.normal(size=Uo.shape)
    h = 1e-6
    Rp, _ = oracle.rhs(spec, Uo + h * V)
    Rm, _ = oracle.rhs(spec, Uo - h * V)
    fd = float((Rb * (Rp - Rm) / (2 * h)).sum())
    s = solver(spec)
    U = s.initial_state(W)
    Ub = s.rhs_vjp(U, dev(Rb))
    torch.cuda.synchronize()
    got = float((Ub.cpu().numpy() * V).sum())
    assert abs(got - fd) <= 1e-6 * abs(fd), (got, fd)


@pytest.mark.parametrize("dim,n,degree,eos,flux", [(2, [6, 5], 3, "tm", "hll"),
                                                    (3, [3, 3, 2], 3, "ideal", "llf")])
def test_rhs_vjp_is_homogeneous_in_r_bar_over_the_fp64_range(gpu_lib, dim, n, degree, eos, flux):
    """The VJP is linear in R_bar.  Its transposed volume term runs in FP32 pair arithmetic on
    R_bar scaled per element by a power of two, so scaling R_bar by 2^k, far outside FP32's
    range, must scale U_bar by exactly 2^k, bit for bit, with elements of very different
    magnitudes side by side."""
    spec = wl.smooth_random(dim, n, degree, eos=eos, flux=flux, c2p="iterative", seed=5)
    W = wl.smooth_random_ic(spec, oracle.node_coords(spec))
    s = solver(spec)
    U = s.initial_state(W)
    rng = np.random.default_rng(11)
    E = int(np.prod(n))
    Rb = rng.normal(size=(5, E, (degree + 1) ** dim))
    # elements whose R_bar differs by 2^300 from its neighbours'
    Rb[:, ::2] *= 2.0 ** 300
    base = s.rhs_vjp(U, dev(Rb)).cpu().numpy()
    assert np.all(np.isfinite(base)) and np.abs(base).max() > 0.0
    for k in (-600, -300, 200, 400):
        got = s.rhs_vjp(U, dev(Rb * 2.0 ** k)).cpu().numpy()
        assert np.array_equal(got, base * 2.0 ** k), k
    # R_bar of moderate size everywhere takes the unscaled pairs; scaled far down, the rescaled
    # ones: the same bits either way
    Rm = Rb.copy()
    Rm[:, ::2] *= 2.0 ** -300
    assert np.abs(Rm).min() > 2.0 ** -90 and np.abs(Rm).max() < 2.0 ** 90
    mid = s.rhs_vjp(U, dev(Rm)).cpu().numpy()
    low = s.rhs_vjp(U, dev(Rm * 2.0 ** -500)).cpu().numpy()
    assert np.array_equal(low, mid * 2.0 ** -500)


@pytest.mark.parametrize("eos,c2p", [("ideal", "analytic"), ("ideal", "iterative"),
                                     ("tm", "analytic"), ("tm", "iterative")])
def test_con2prim_vjp_against_oracle_differences(gpu_lib, eos, c2p):
    n = 200
    spec = dict(dim=1, degree=0, n_elem=[n], eos=eos, gamma_ad=4.0 / 3.0, c2p=c2p)
    W = wl.random_primitive_states(n, seed=9, gamma_max=5.0, theta_range=(1e-2, 1e2),
                                   rho_range=(0.1, 10.0))[:, :, None]
    Uo = oracle.prim2cons(spec, W)
    rng = np.random.default_rng(2)
    V = rng.normal(size=Uo.shape) * np.abs(Uo)
    Wb = rng.normal(size=Uo.shape)
    h = 1e-6
    # The adjoint is the derivative of the exact inverse of prim->cons, whichever solver finds
    # it; differences of the closed-form ideal solver are dominated by its rounding (Sec. 3.3:
    # up to 1e-10 relative), so the ideal case is differenced with the Newton solver.
    fd_spec = dict(spec, c2p="iterative") if eos == "ideal" else spec
    Wp, _, _ = oracle.con2prim(fd_spec, Uo + h * V)
    Wm, _, _ = oracle.con2prim(fd_spec, Uo - h * V)
    fd = (Wb * (Wp - Wm) / (2 * h)).sum(axis=0)[:, 0]
    s = solver(spec)
    Ub = s.con2prim_vjp(dev(Uo), dev(Wb)).cpu().numpy()
    got = (Ub * V).sum(axis=0)[:, 0]
    assert np.all(np.abs(got - fd) <= 1e-6 * np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max())), \
        np.abs(got - fd).max()


def test_enforce_vjp_is_the_transpose_of_the_frozen_operator(gpu_lib):
    """With each element's factor s frozen the operator is the linear map
    V -> s V + (1 - s) mean(V) (Eq. smoothed_states); its transpose must satisfy
    <Z, L_s V> = <L_s^T Z, V>."""
    spec = dict(dim=2, degree=3, n_elem=[12, 10], eos="ideal", gamma_ad=5.0 / 3.0)
    E, Nn = wl.shape(spec)
    U = wl.random_conserved_cells(E, Nn, seed=4)
    s = solver(spec)
    _, sf = s.enforce(dev(U), with_s=True)
    sf_np = sf.cpu().numpy()
    assert np.any(sf_np < 1.0) and np.any(sf_np == 1.0)
    rng = np.random.default_rng(5)
    V = rng.normal(size=U.shape)
    Z = rng.normal(size=U.shape)
    w1 = np.polynomial.legendre.leggauss(4)[1]
    w = np.multiply.outer(w1, w1).ravel()
    mean = (V * w).sum(-1, keepdims=True) / w.sum()
    LV = sf_np[None, :, None] * V + (1 - sf_np[None, :, None]) * mean
    LTZ = s.enforce_vjp(sf, dev(Z)).cpu().numpy()
    lhs, rhs = float((Z * LV).sum()), float((LTZ * V).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def oracle_objective(spec, A, vx_dir=None, eps=0.0, nsteps=10):
    X = oracle.node_coords(spec)
    W = wl.kh2d_ic(spec, X, amplitude=A)
    if vx_dir is not None:
        W[1] += eps * vx_dir
    U = oracle.prim2cons(spec, W)
    U, st = oracle.step(spec, U, spec["dt"], nsteps)
    assert st["enforced_cells"] == 0 and st["c2p_invalid_input"] == 0
    Wf, _, _ = oracle.con2prim(spec, U)
    g2 = 1.0 / (1.0 - (Wf[1:4] ** 2).sum(0))
    N = spec["degree"] + 1
    w1 = np.polynomial.legendre.leggauss(N)[1]
    w = np.multiply.outer(w1, w1).ravel()
    jac = (spec["hi"][0] - spec["lo"][0]) / spec["n_elem"][0] / 2 * (spec["hi"][1] - spec["lo"][1]) / spec["n_elem"][1] / 2
    return float((w * jac * Wf[0] * g2 * Wf[2] ** 2).sum())


def test_checkpointed_rollout_gradient_against_oracle_differences(gpu_lib):
    from paper_2205_00095_gb300 import adjoint

    spec = wl.kh2d(nx=8, ny=16, degree=3)
    s = solver(spec)
    spec["dt"] = s.cfl_dt(0.2)
    nsteps, every, A = 10, 4, 0.01
    X = s.node_coords()
    W0 = wl.kh2d_ic(spec, X, amplitude=A)
    U0 = s.initial_state(W0).requires_grad_(True)
    UT = adjoint.rollout(s, U0, spec["dt"], nsteps, every)
    J = adjoint.transverse_kinetic_energy(s, UT)
    J.backward()
    torch.cuda.synchronize()
    Ubar0 = U0.grad.cpu().numpy()
    status, st = s.stats()
    assert st["enforced_cells"] == 0

    # forward objective agrees with the oracle
    assert abs(float(J.detach()) - oracle_objective(spec, A, nsteps=nsteps)) <= 1e-11 * abs(float(J.detach()))

    def tangent(dW):
        h = 1e-6
        Up = s.initial_state(W0 + h * dW).cpu().numpy()
        Um = s.initial_state(W0 - h * dW).cpu().numpy()
        return (Up - Um) / (2 * h)

    # d J / d A: the amplitude enters through v_y only
    dW = np.zeros_like(W0)
    dW[2] = wl.kh2d_ic(spec, X, amplitude=1.0)[2]
    g_adj = float((Ubar0 * tangent(dW)).sum())
    hA = 1e-6 * A
    g_fd = (oracle_objective(spec, A + hA, nsteps=nsteps) - oracle_objective(spec, A - hA, nsteps=nsteps)) / (2 * hA)
    assert abs(g_adj - g_fd) <= 1e-6 * abs(g_fd), (g_adj, g_fd)

    # nodal initial v_x: individual nodes and random directions.  The nodes are those with the
    # largest direct sensitivity 2 rho gamma^4 |v_x| v_y^2 w at t = 0, one per element, where the
    # gradient stands far above the rounding of J / (2 eps); no absolute floor is needed.
    rng = np.random.default_rng(11)
    E, Nn = s.n_elem, s.n_node
    w1 = np.polynomial.legendre.leggauss(spec["degree"] + 1)[1]
    wn = np.multiply.outer(w1, w1).ravel()
    g2 = 1.0 / (1.0 - (W0[1:4] ** 2).sum(0))
    score = 2.0 * W0[0] * g2 * g2 * np.abs(W0[1]) * W0[2] ** 2 * wn
    dirs = []
    for e in np.argsort(-score.max(axis=1))[:6]:
        d = np.zeros((E, Nn))
        d[e, score[e].argmax()] = 1.0
        dirs.append(d)
    dirs += [rng.normal(size=(E, Nn)) for _ in range(2)]
    for d in dirs:
        dWx = np.zeros_like(W0)
        dWx[1] = d
        g_adj = float((Ubar0 * tangent(dWx)).sum())
        eps = 1e-6
        g_fd = (oracle_objective(spec, A, d, eps, nsteps) - oracle_objective(spec, A, d, -eps, nsteps)) / (2 * eps)
        assert abs(g_adj - g_fd) <= 1e-6 * abs(g_fd), (g_adj, g_fd)


def test_stage_vjp_with_saved_forward_equals_recompute(gpu_lib):
    """dgsrhd_stage_vjp on the quantities kept by dgsrhd_step_stage gives the same adjoint as the
    version that re-runs the forward volume kernel, and the stages compose to dgsrhd_step."""
    spec = wl.kh2d(nx=8, ny=8, degree=2)
    s = solver(spec)
    U = s.initial_state(wl.kh2d_ic(spec, s.node_coords()))
    dt = s.cfl_dt(0.2)
    ref = U.clone()
    s.step(ref, dt, 1)
    X1 = torch.empty_like(U)
    X2 = torch.empty_like(U)
    out = torch.empty_like(U)
    saves = [torch.empty(s.stage_save_size(), dtype=torch.float64, device="cuda") for _ in range(3)]
    ss = [torch.empty(s.n_elem, dtype=torch.float64, device="cuda") for _ in range(3)]
    s.step_stage(U, U, X1, 0, dt, ss[0], saves[0])
    s.step_stage(U, X1, X2, 1, dt, ss[1], saves[1])
    s.step_stage(U, X2, out, 2, dt, ss[2], saves[2])
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    Z = torch.from_numpy(np.random.default_rng(1).normal(size=U.shape)).cuda()
    for k, Xk in enumerate((U, X1, X2)):
        a_un, a_uk = torch.zeros_like(U), torch.zeros_like(U)
        b_un, b_uk = torch.zeros_like(U), torch.zeros_like(U)
        s.stage_vjp(Xk, ss[k], Z, a_un, a_uk, k, dt, saves[k])
        s.stage_vjp(Xk, ss[k], Z, b_un, b_uk, k, dt, None)
        torch.cuda.synchronize()
        assert torch.equal(a_un, b_un) and torch.equal(a_uk, b_uk)


@pytest.mark.parametrize("flux", ["llf", "hll", "hllc"])
@pytest.mark.parametrize("eos", ["ideal", "tm"])
def test_stages_that_keep_the_tape_give_the_bits_of_a_step(gpu_lib, flux, eos):
    """The face kernel that writes the reverse sweep's tape and the one that does not give the
    same numerical fluxes bit for bit: LLF reaches its dissipation speed by different but
    bit-identical routes in the two, and both fold the normal fluxes into the same sums."""
    if eos == "ideal":
        spec = wl.advected_wave(n=12, degree=3, flux=flux)
        s = solver(spec)
        U = s.initial_state(wl.advected_wave_ic(spec, s.node_coords()))
    else:
        spec = dict(wl.kh2d(nx=8, ny=8, degree=2), flux=flux)
        s = solver(spec)
        U = s.initial_state(wl.kh2d_ic(spec, s.node_coords()))
    dt = s.cfl_dt(0.2)
    ref = U.clone()
    s.step(ref, dt, 1)
    X1, X2, out = torch.empty_like(U), torch.empty_like(U), torch.empty_like(U)
    saves = [torch.empty(s.stage_save_size(), dtype=torch.float64, device="cuda") for _ in range(3)]
    ss = [torch.empty(s.n_elem, dtype=torch.float64, device="cuda") for _ in range(3)]
    s.step_stage(U, U, X1, 0, dt, ss[0], saves[0])
    s.step_stage(U, X1, X2, 1, dt, ss[1], saves[1])
    s.step_stage(U, X2, out, 2, dt, ss[2], saves[2])
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    assert s.stats()[0] == 0


def test_stage_vjp_of_a_limited_stage_needs_the_saved_forward(gpu_lib):
    """The limiter's factors exist only in the saved forward quantities (recomputing them would
    need U^n): without saved, dgsrhd_stage_vjp returns DGSRHD_EINVAL for a limited stage."""
    from paper_2205_00095_gb300 import _lib
    spec = dict(wl.kh2d(nx=4, ny=8, degree=2), limiter=True)
    s = solver(spec)
    U = s.initial_state(wl.kh2d_ic(spec, s.node_coords()))
    Z = torch.zeros_like(U)
    a, b = torch.zeros_like(U), torch.zeros_like(U)
    torch.cuda.synchronize()
    st = s.lib.dgsrhd_stage_vjp(s.ctx, U.data_ptr(), None, None, Z.data_ptr(), a.data_ptr(),
                                b.data_ptr(), 0, 1e-3)
    assert st == _lib.DGSRHD_EINVAL


def frozen_scale(U, f, w):
    """V -> mean + f (V - mean) per element (the limiter and the operator with frozen f)."""
    mean = (U * w).sum(-1, keepdims=True) / w.sum()
    return mean + f[None, :, None] * (U - mean)


LIMITED_STAGES = [
    (dict(wl.riemann_1d(4, n=24, degree=1), limiter=True, limiter_alpha=0.0), 1),
    (dict(wl.riemann_1d(2, n=24, degree=2), limiter="minmod", limiter_alpha=0.0), 2),
    (dict(wl.kh_single(nx=6, ny=12, degree=2), limiter="minmod", limiter_alpha=0.0), 2),
]


@pytest.mark.parametrize("spec,stage", LIMITED_STAGES)
def test_limited_stage_vjp_is_the_transpose_of_the_frozen_stage(gpu_lib, spec, stage):
    """With the limiter's theta and the operator's s frozen at their forward values a stage is
    Z = L_s(L_theta(a Un + b (Uk + dt R(Uk)))); <Zbar, dZ/dUk V> by central differences of the
    oracle's R (h = 1e-6) equals <Ukbar, V> from dgsrhd_stage_vjp, and Unbar = a L^T Zbar."""
    s = solver(spec)
    E, Nn = s.n_elem, s.shape[2]
    U0 = s.initial_state(wl.initial_primitive(spec, s.node_coords()))
    s.enforce(U0)
    dt = s.cfl_dt(0.2)
    s.step(U0, dt, 6)           # a few limited steps: structure near the discontinuities
    Un = U0.clone()
    X = [Un]
    for k in range(stage):      # the inputs of stages 0..stage
        out = torch.empty_like(Un)
        s.step_stage(Un, X[k], out, k, dt)
        X.append(out)
    Uk = X[stage]
    out = torch.empty_like(Un)
    sf = torch.empty(E, dtype=torch.float64, device="cuda")
    save = torch.empty(s.stage_save_size(), dtype=torch.float64, device="cuda")
    s.step_stage(Un, Uk, out, stage, dt, sf, save)
    torch.cuda.synchronize()
    theta = save[-E:].cpu().numpy()
    sfn = sf.cpu().numpy() if spec.get("enforce", True) else np.ones(E)
    assert np.any(theta < 1.0), "the stage should be limited somewhere"
    rng = np.random.default_rng(11)
    Zb = rng.normal(size=tuple(U0.shape))
    Ua = np.abs(Uk.cpu().numpy())
    V = rng.normal(size=tuple(U0.shape)) * (Ua + 1e-3 * Ua.max(axis=(1, 2), keepdims=True))
    Unb, Ukb = torch.zeros_like(Un), torch.zeros_like(Un)
    s.stage_vjp(Uk, sf, torch.from_numpy(Zb).cuda(), Unb, Ukb, stage, dt, save)
    torch.cuda.synchronize()
    ns = spec["rk_stages"]
    a_n = [[0.0], [0.0, 0.5], [0.0, 0.75, 1.0 / 3.0]][ns - 1][stage]
    b_k = [[1.0], [1.0, 0.5], [1.0, 0.25, 2.0 / 3.0]][ns - 1][stage]
    N = spec["degree"] + 1
    w1 = np.polynomial.legendre.leggauss(N)[1]
    w = w1
    for _ in range(spec["dim"] - 1):
        w = np.multiply.outer(w1, w).ravel()
    Unp, Ukp = Un.cpu().numpy(), Uk.cpu().numpy()

    def stage_map(Ukx):
        R, _ = oracle.rhs(spec, Ukx)
        Y = a_n * Unp + b_k * (Ukx + dt * R)
        return frozen_scale(frozen_scale(Y, theta, w), sfn, w)

    h = 1e-6
    dZ = (stage_map(Ukp + h * V) - stage_map(Ukp - h * V)) / (2 * h)
    lhs = float((Zb * dZ).sum())
    rhs = float((Ukb.cpu().numpy() * V).sum())
    assert abs(lhs - rhs) <= 1e-6 * max(abs(lhs), abs(rhs))
    # Un enters linearly: Unbar = a_n L_theta^T L_s^T Zbar
    Ln = frozen_scale(frozen_scale(Unp + V, theta, w), sfn, w) - frozen_scale(frozen_scale(Unp, theta, w), sfn, w)
    if a_n != 0.0:
        lhs_n = float((Zb * a_n * Ln).sum())
        rhs_n = float((Unb.cpu().numpy() * V).sum())
        assert abs(lhs_n - rhs_n) <= 1e-10 * max(abs(lhs_n), abs(rhs_n))


GOLDEN_C4 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "kh_adjoint_c4.json")


def test_full_size_rollout_gradient_against_stored_oracle_differences(gpu_lib):
    """The adjoint's own benchmark configuration: KH 128 x 256, p = 3, 200 SSPRK3 steps with a
    checkpoint every 20.  The objective, dJ/dA, the derivative along three seeded fields of
    initial v_x and dJ/dv_x at single nodes from the checkpointed adjoint against the FP64
    oracle's central differences stored by tests/golden/make_kh_adjoint_c4.py, at 1e-6 relative
    with no absolute floor: h = 1e-6 for dJ/dA and the fields (their h and 2h differences agree
    to 1e-8), the Richardson value of h = 1e-4 and 2e-4 for single nodes (at h = 1e-6 a single
    node moves J by a few units of its last place).  The step is the library's dgsrhd_cfl_dt,
    which must equal the oracle's CFL step that the stored runs used."""
    import json
    from paper_2205_00095_gb300 import adjoint

    g = json.load(open(GOLDEN_C4))
    cfg = g["configuration"]
    spec = wl.kh2d(nx=cfg["n_elem"][0], ny=cfg["n_elem"][1], degree=cfg["degree"])
    s = solver(spec)
    dt = s.cfl_dt(cfg["cfl"])
    assert dt == cfg["dt"], (dt, cfg["dt"])
    A, h = cfg["amplitude"], cfg["h"]
    X = s.node_coords()
    W0 = wl.kh2d_ic(spec, X, amplitude=A)
    U0 = s.initial_state(W0).requires_grad_(True)
    J = adjoint.transverse_kinetic_energy(s, adjoint.rollout(s, U0, dt, cfg["nsteps"], cfg["checkpoint_every"]))
    J.backward()
    torch.cuda.synchronize()
    status, st = s.stats()
    assert status == 0 and st["enforced_cells"] == 0
    Ubar0 = U0.grad.cpu().numpy()
    Jv = float(J.detach())
    assert abs(Jv - g["J"]) <= 1e-9 * abs(g["J"]), (Jv, g["J"])

    def directional(dW):
        """<U_bar0, dU0/dW . dW> with the tangent of the library's prim -> cons by differences."""
        scale = 1.0 / np.abs(dW).max()
        tang = (s.initial_state(W0 + h * scale * dW).cpu().numpy()
                - s.initial_state(W0 - h * scale * dW).cpu().numpy()) / (2 * h * scale)
        return float((Ubar0 * tang).sum())

    report = []
    dW = np.zeros_like(W0)
    dW[2] = wl.kh2d_ic(spec, X, amplitude=1.0)[2]  # the amplitude enters through v_y only
    report.append(("dJ/dA", directional(dW), g["dJ_dA"]["fd_h"]))
    for r in g["dJ_dvx_directions"]:
        d = np.zeros_like(W0)
        rnd = np.random.RandomState(r["seed"]).standard_normal(W0.shape[1:])
        d[1] = W0[1] * np.sin(2.0 * np.pi * X[0]) ** 2 * np.exp(-2.0 * X[1] ** 2 / 0.01) * (1.0 + 0.5 * rnd)
        report.append((f"field {r['seed']}", directional(d), r["fd_h"]))
    assert len(g["dJ_dvx_nodes"]) >= 8
    for n in g["dJ_dvx_nodes"]:
        d = np.zeros_like(W0)
        d[1, n["elem"], n["node"]] = 1.0
        report.append((f"node {n['elem']}/{n['node']}", directional(d), n["richardson"]))
    worst = max(abs(a - b) / abs(b) for _, a, b in report)
    print(f"\nC4 adjoint vs oracle differences: worst relative error {worst:.2e} over {len(report)} checks")
    for name, a, b in report:
        assert abs(a - b) <= 1e-6 * abs(b), (name, a, b)
