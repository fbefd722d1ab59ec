"""The Kelvin-Helmholtz diagnostic <v_y^2> (Sec. 4.5) through the C ABI against the oracle and
a closed form, and the growth of the instability in the paper's set-up."""
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


def test_mean_square_velocity_against_oracle_and_closed_form(gpu_lib):
    from paper_2205_00095_gb300 import Solver
    spec = wl.kh_single(nx=16, ny=32, degree=2)
    X = oracle.node_coords(spec)
    U = oracle.prim2cons(spec, wl.kh_single_ic(spec, X))
    s = Solver(spec)
    for axis in (0, 1, 2):
        got, want = s.mean_square_velocity(dev(U), axis), oracle.mean_square_velocity(spec, U, axis)
        assert abs(got - want) <= 1e-12 * max(abs(want), 1e-300), (axis, got, want)
    # v_y = 0.3 sin(2 pi x) on the periodic unit square: exactly 0.3^2 / 2 (see the oracle pin)
    spec2 = dict(dim=2, degree=3, n_elem=[8, 8], lo=[0.0, 0.0], hi=[1.0, 1.0], eos="ideal",
                 gamma_ad=4.0 / 3.0, c2p="iterative", bc=[("periodic", "periodic")] * 2)
    X2 = oracle.node_coords(spec2)
    W2 = np.stack([np.ones_like(X2[0]), 0.2 + 0.0 * X2[0], 0.3 * np.sin(2 * np.pi * X2[0]),
                   0.0 * X2[0], np.ones_like(X2[0])])
    s2 = Solver(spec2)
    assert abs(s2.mean_square_velocity(dev(oracle.prim2cons(spec2, W2)), 1) - 0.045) < 1e-14
    from paper_2205_00095_gb300 import _lib
    assert s2.lib.dgsrhd_mean_square_velocity(s2.ctx, None, 1, None) == _lib.DGSRHD_EINVAL


def test_kh_single_grows_exponentially(gpu_lib):
    """64 x 128 elements, p = 1, HLL, to t = 3: <v_y^2> grows, and log <v_y^2> is close to a
    line over the paper's fitting window t in [1.5, 3]."""
    from paper_2205_00095_gb300 import kh_growth
    r = kh_growth.run(nx=64, degree=1, flux="hll", t_end=3.0)
    t, m = np.array(r["t"]), np.array(r["mean_vy2"])
    assert r["device_status"] == 0 and np.all(np.isfinite(m))
    assert m[t >= 3.0 - 1e-9][0] > m[np.argmin(np.abs(t - 1.5))]
    assert r["growth_rate_fit_1p5_to_3"] > 0.0 and r["fit_r2"] > 0.9, r["fit_r2"]



def test_kh_throughput_points(gpu_lib):
    """The throughput study of Sec. 4.6 on two points: runs clean, and the paper's smallest mesh
    updates more DOF per second than a 32 x 64 mesh (the small one cannot fill the GPU)."""
    from paper_2205_00095_gb300 import kh_perf
    small = kh_perf.measure(32, 64, 1, "hll", steps=20)
    paper = kh_perf.measure(256, 512, 1, "hll", steps=20)
    for r in (small, paper):
        assert r["status"] == 0 and r["dof_updates_per_s"] > 0.0
        assert r["rk_stages"] == 2 and r["dof"] == r["n_x"] * r["n_y"] * 4
    assert paper["dof_updates_per_s"] > small["dof_updates_per_s"]
