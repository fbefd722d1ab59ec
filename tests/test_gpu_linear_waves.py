"""Linear waves (Sec. 4.1) through the C ABI: parity with the oracle in an oblique box, and
order p + 1 convergence of the GPU solution in the oblique 3D box of the paper's table."""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl
from tests.linear_wave_support import make

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("frame,wave,degree", [("2d_oblique", "+", 2), ("3d_oblique", "0(2)", 1),
                                               ("2d", "-", 3)])
def test_linear_wave_twenty_steps_against_oracle(gpu_lib, frame, wave, degree):
    from paper_2205_00095_gb300 import Solver
    spec = make(frame, wave, degree, 4, 0)
    s = Solver(spec, stream=torch.cuda.Stream())
    X = oracle.node_coords(spec)
    Uo = oracle.prim2cons(spec, wl.linear_wave_ic(spec, X))
    dt = s.cfl_dt(0.2)
    U = torch.from_numpy(Uo.copy()).cuda()
    torch.cuda.synchronize()
    s.step(U, dt, 20)
    s.synchronize()
    Uo20, _ = oracle.step(spec, Uo, dt, 20)
    # the perturbation is 1e-6 of the state: measure the difference against the size of the
    # deviation from the base state (1e-7 of it is 1e-13 of the state)
    dev = np.abs(Uo20 - Uo.mean(axis=(1, 2), keepdims=True)).max()
    assert np.abs(U.cpu().numpy() - Uo20).max() <= 1e-7 * dev


def test_oblique_3d_acoustic_wave_converges_at_third_order(gpu_lib):
    from paper_2205_00095_gb300 import linear_waves
    r = linear_waves.run_wave("3d_oblique", "+", 2, 4, 3, wl)
    q = r["variables"]["D"]["order_finest_pair"]
    assert q > 2.5, r["variables"]["D"]
    assert r["variables"]["u_y"] is not None and r["variables"]["P"] is not None
