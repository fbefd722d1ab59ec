"""The paper's Riemann problems on the GPU at the paper's resolutions (Sec. 4.2, 4.3), HLLC
with the limiter: the 1D problems 2, 4 and 5 at p = 1 from 256 to 2048 cells against the exact
solution (L1 errors fall; the table is printed with -s), and the three 2D problems at 256^2
to t = 0.8 (admissible throughout; the mirror-symmetric test 3 stays symmetric)."""
import time

import numpy as np
import pytest
import torch

import workloads as wl
from oracle.exact_riemann import ExactRiemann

pytestmark = pytest.mark.gpu


def exact(spec):
    L, R, G = spec["left"], spec["right"], spec["gamma_ad"]
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


@pytest.mark.parametrize("problem", [2, 4, 5])
def test_1d_riemann_problem_converges_on_the_gpu(gpu_lib, problem):
    rows = []
    for n in (256, 512, 1024, 2048):
        spec = dict(wl.riemann_1d(problem, n=n, degree=1), limiter=True)
        s, U, st, status, nsteps, el = run(spec)
        assert st["mean_inadmissible_cells"] == 0 and st["c2p_invalid_input"] == 0
        X = s.node_coords()
        from paper_2205_00095_gb300.solver import quadrature_weights_1d
        w = quadrature_weights_1d(2)
        Ue = s.initial_state(exact(spec).sample(X[0], spec["t_final"])).cpu().numpy()
        l1 = (np.abs(U.cpu().numpy() - Ue) * w).sum(axis=(1, 2)) / (2 * n)
        rows.append((n, l1[0], l1[1], l1[4], nsteps, el))
    print(f"\nRiemann problem {problem}, p = 1, HLLC + limiter (n, L1 D, L1 S_x, L1 tau, steps, s)")
    for r in rows:
        print("  %5d  %.4e  %.4e  %.4e  %6d  %.2f" % r)
    e = np.array([[r[1], r[2], r[3]] for r in rows])
    assert np.all(e[1:] < e[:-1])


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
        assert np.abs(M - V).max() / np.abs(V).max() < 1e-10
