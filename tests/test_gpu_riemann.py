"""The paper's Riemann problems on the GPU at the paper's resolutions (Sec. 4.2, 4.4), HLLC
with the limiter: the 1D problems 2-5 and the Taub-Matthews blast with the three EOS of Fig. 9 at
p = 1 from 256 to 2048 cells against the exact solution (L1 errors fall; the table is printed
with -s), the ordering Fig. 9 shows between the three EOS, and the three 2D problems at 256^2
to t = 0.8 (admissible throughout; the mirror-symmetric test 3 stays symmetric)."""
import time

import numpy as np
import pytest
import torch

import oracle
import workloads as wl
from oracle.exact_riemann import ExactRiemann
from oracle.exact_riemann_general import GeneralExactRiemann

pytestmark = pytest.mark.gpu


def exact(spec):
    L, R, G = spec["left"], spec["right"], spec["gamma_ad"]
    if spec["eos"] != "ideal" or L[2] != 0.0 or R[2] != 0.0:
        return GeneralExactRiemann((L[0], L[1], L[2], L[4]), (R[0], R[1], R[2], R[4]),
                                   spec["eos"], G, 0.5)
    if spec["bc"][0][1] == "reflect":
        return ExactRiemann((L[0], L[1], L[4]), (L[0], -L[1], L[4]), G, 1.0)
    return ExactRiemann((L[0], L[1], L[4]), (R[0], R[1], R[4]), G, 0.5)


def run(spec):
    from paper_2205_00095_gb300 import Solver
    s = Solver(spec, stream=torch.cuda.Stream())
    with torch.cuda.stream(s.stream):
        U = s.initial_state(wl.initial_primitive(spec, s.node_coords_device()))
        s.enforce(U)
    T = spec["t_final"]
    nsteps = int(np.ceil(T / s.cfl_dt(spec["cfl"])))
    s.synchronize()
    t0 = time.perf_counter()
    s.step(U, T / nsteps, nsteps)
    s.synchronize()
    el = time.perf_counter() - t0
    status, st = s.stats()
    return s, U, st, status, nsteps, el


BLAST_EOS = {"tm": ("tm", 4.0 / 3.0), "ideal4/3": ("ideal", 4.0 / 3.0),
             "ideal5/3": ("ideal", 5.0 / 3.0)}


def spec_of(problem, n, degree):
    if problem in BLAST_EOS:
        return wl.tm_blast(*BLAST_EOS[problem], n=n, degree=degree)
    return wl.riemann_1d(problem, n=n, degree=degree)


@pytest.mark.parametrize("problem", [2, 3, 4, 5, "tm", "ideal4/3", "ideal5/3"])
def test_1d_riemann_problem_converges_on_the_gpu(gpu_lib, problem):
    rows = []
    for n in (256, 512, 1024, 2048):
        spec = dict(spec_of(problem, n, 1), limiter=True)
        s, U, st, status, nsteps, el = run(spec)
        assert st["mean_inadmissible_cells"] == 0 and st["c2p_invalid_input"] == 0
        X = s.node_coords()
        from paper_2205_00095_gb300.solver import quadrature_weights_1d
        w = quadrature_weights_1d(2)
        Ue = s.initial_state(exact(spec).sample(X[0], spec["t_final"])).cpu().numpy()
        l1 = (np.abs(U.cpu().numpy() - Ue) * w).sum(axis=(1, 2)) / (2 * n)
        rows.append((n, l1[0], l1[1], l1[2], l1[4], nsteps, el))
    print(f"\nRiemann problem {problem}, p = 1, HLLC + limiter "
          "(n, L1 D, L1 S_x, L1 S_y, L1 tau, steps, s)")
    for r in rows:
        print("  %5d  %.4e  %.4e  %.4e  %.4e  %6d  %.2f" % r)
    e = np.array([[r[1], r[2], r[3], r[4]] for r in rows])
    if problem in (2, 4, 5):
        e = e[:, [0, 1, 3]]
    assert np.all(e[1:] < e[:-1])


@pytest.mark.parametrize("problem,degree", [(2, 1), (3, 1), (4, 1), ("tm", 1), (5, 2)])
def test_1d_riemann_problem_converges_with_minmod_on_the_gpu(gpu_lib, problem, degree):
    """The same runs with the minmod limiter (limiter_alpha = 0: the TVD form); with it the
    wall problem 5 also runs at p = 2, where the scaling limiter loses admissible means."""
    rows = []
    for n in (256, 512, 1024, 2048):
        spec = dict(spec_of(problem, n, degree), limiter="minmod", limiter_alpha=0.0)
        s, U, st, status, nsteps, el = run(spec)
        assert status == 0 and st["mean_inadmissible_cells"] == 0 and st["limited_cells"] > 0
        X = s.node_coords()
        from paper_2205_00095_gb300.solver import quadrature_weights_1d
        w = quadrature_weights_1d(degree + 1)
        Ue = s.initial_state(exact(spec).sample(X[0], spec["t_final"])).cpu().numpy()
        l1 = (np.abs(U.cpu().numpy() - Ue) * w).sum(axis=(1, 2)) / (2 * n)
        rows.append((n, l1[0], l1[1], l1[2], l1[4], nsteps, el))
    print(f"\nRiemann problem {problem}, p = {degree}, HLLC + minmod "
          "(n, L1 D, L1 S_x, L1 S_y, L1 tau, steps, s)")
    for r in rows:
        print("  %5d  %.4e  %.4e  %.4e  %.4e  %6d  %.2f" % r)
    e = np.array([[r[1], r[2], r[3], r[4]] for r in rows])
    if problem in (2, 4, 5):
        e = e[:, [0, 1, 3]]
    assert np.all(e[1:] < e[:-1])


def test_tm_blast_ordering_of_fig9(gpu_lib):
    """Fig. 9 at t = 0.7 on 2048 cells: the Taub-Matthews blast front lies ahead of both ideal
    gases' (the front: the right-most node whose density exceeds twice the right state's), near
    the exact shock, and its minimum transverse four-velocity is the lowest of the three; its
    equivalent adiabatic index is 4/3 on the hot side and 5/3 on the cold side."""
    front, umin = {}, {}
    for k in BLAST_EOS:
        spec = dict(spec_of(k, 2048, 1), limiter=True)
        s, U, st, status, nsteps, el = run(spec)
        assert status == 0 and st["mean_inadmissible_cells"] == 0
        W = s.con2prim(U)
        s.synchronize()
        W = W.cpu().numpy()
        x = s.node_coords()[0]
        rho = W[0].reshape(-1)
        front[k] = x.reshape(-1)[np.nonzero(rho > 2.0)[0].max()]
        lor = 1.0 / np.sqrt(1.0 - (W[1:4] ** 2).sum(axis=0))
        umin[k] = (lor * W[2]).min()
        if k == "tm":
            # Gamma_eq: 4/3 in the hot left state, 5/3 in the cold right one, between across
            g = oracle.gamma_eq(spec, W[0].reshape(-1), W[4].reshape(-1))
            xs = x.reshape(-1)
            assert np.all((g > 4.0 / 3.0 - 1e-12) & (g < 5.0 / 3.0 + 1e-12))
            assert np.all(np.abs(g[xs < 0.1] - 4.0 / 3.0) < 1e-3)
            assert np.all(np.abs(g[xs > 0.95] - 5.0 / 3.0) < 1e-2)
        # the thin shell behind the blast converges at first order in position: the front lies
        # ahead of the exact shock by about 0.010 (5/3) and 0.007 (TM) at 2048 cells
        ex = exact(spec)
        assert -0.002 < front[k] - (0.5 + ex.Vs_R * spec["t_final"]) < 0.015
    print("\nTM blast fronts at t = 0.7:", front, "min u_y:", umin)
    assert front["tm"] > front["ideal4/3"] > front["ideal5/3"]
    assert umin["tm"] < umin["ideal4/3"] and umin["tm"] < umin["ideal5/3"]


@pytest.mark.parametrize("test,degree", [(1, 1), (2, 1), (3, 1), (3, 2)])
def test_2d_riemann_problem_at_256(gpu_lib, test, degree):
    spec = wl.riemann_2d(test, n=256, degree=degree)
    s, U, st, status, nsteps, el = run(spec)
    assert status == 0 and st["mean_inadmissible_cells"] == 0
    N = degree + 1
    dof = 256 * 256 * N * N
    print(f"\n2D Riemann test {test}, p = {degree}: {nsteps} steps, {el:.2f} s, "
          f"{dof * nsteps * spec['rk_stages'] / el:.3e} DOF-updates/s, "
          f"limited {st['limited_cells']}, smoothed {st['enforced_cells']}")
    if test == 3:
        V = U.cpu().numpy().reshape(5, 256, 256, N, N)
        M = V.transpose(0, 2, 1, 4, 3).copy()
        M[[1, 2]] = M[[2, 1]]
        # the problem is symmetric under x <-> y (Sec. 4.4); the x-then-y summation order breaks
        # the symmetry at rounding level, and the limiter's decisions amplify it over the run
        # (5120 steps at p = 2: a few 1e-9 here, moving with any change of rounding; at 1024^2
        # it reaches 3e-3), while a mistake in one axis's arithmetic shows at O(dx)
        assert np.abs(M - V).max() / np.abs(V).max() < 1e-8
