"""Split-precision form: the volume term and trace extrapolation on tensor cores (3xTF32, FP32
accumulation), the lift as FP32 FMAs, all on deviations from a per-element reference;
everything else FP64.  Checked
against the FP64 oracle: the RHS to 1e-5 of its largest magnitude, and the state after 100
SSPRK3 steps to an L1 difference below 1e-6 relative."""
import numpy as np
import pytest
import torch

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu


def solver(spec, **kw):
    from paper_2205_00095_gb300 import Solver
    return Solver(dict(spec, precision="split"), **kw)


def gpu_state(s, spec):
    with torch.cuda.stream(s.stream):
        U = s.initial_state(wl.initial_primitive(spec, s.node_coords_device()))
    s.synchronize()
    return U


def oracle_state(spec):
    X = oracle.node_coords(spec)
    return oracle.prim2cons(spec, wl.initial_primitive(spec, X))


def l1_rel(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


CASES = [
    (1, [203], 1, "ideal", "hll", None),
    (1, [64], 4, "tm", "llf", [("dirichlet", "outflow")]),
    (2, [19, 17], 2, "tm", "llf", None),
    (2, [17, 19], 3, "ideal", "hll", None),
    (2, [11, 9], 4, "ideal", "llf", [("outflow", "dirichlet"), ("periodic", "periodic")]),
    (3, [6, 5, 7], 3, "tm", "hll", None),
    (3, [4, 3, 5], 4, "ideal", "llf", None),
    (2, [20, 13], 0, "ideal", "llf", None),
    (2, [9, 8], 2, "ideal", "hllc", [("reflect", "outflow"), ("periodic", "periodic")]),
    (1, [33], 3, "tm", "hllc", [("reflect", "reflect")]),
]


@pytest.mark.parametrize("dim,n,degree,eos,flux,bc", CASES)
@pytest.mark.parametrize("nodes", ["gl", "gll"])
def test_split_rhs_against_oracle(gpu_lib, dim, n, degree, eos, flux, bc, nodes):
    if nodes == "gll" and degree == 0:
        pytest.skip("Gauss-Lobatto-Legendre needs degree >= 1")
    spec = dict(wl.smooth_random(dim, n, degree, eos=eos, flux=flux, c2p="iterative", seed=5,
                                 bc=bc), nodes=nodes)
    s = solver(spec)
    R = s.rhs(gpu_state(s, spec)).cpu().numpy()
    Ro, _ = oracle.rhs(spec, oracle_state(spec))
    err = float(np.abs(R - Ro).max() / np.abs(Ro).max())
    assert err < 1e-5, err


@pytest.mark.parametrize("spec_fn", [
    lambda: wl.advected_wave(n=16, degree=3, c2p="analytic"),
    lambda: wl.kh2d(nx=12, ny=24, degree=3),
    lambda: wl.smooth_random(3, [5, 6, 4], 2, eos="tm", flux="hll", seed=8),
    # limiters after the split update, HLLC
    lambda: dict(wl.riemann_1d(4, n=96, degree=1), limiter=True),
    lambda: dict(wl.tm_blast("tm", n=96, degree=2), limiter="minmod"),
    lambda: dict(wl.kh_single(nx=12, ny=24, degree=2, flux="hllc"), limiter="minmod"),
])
def test_split_hundred_steps_l1(gpu_lib, spec_fn):
    spec = spec_fn()
    s = solver(spec, stream=torch.cuda.Stream())
    dt = s.cfl_dt(0.2)
    U = gpu_state(s, spec)
    s.step(U, dt, 100)
    s.synchronize()
    Uo, sto = oracle.step(spec, oracle_state(spec), dt, 100)
    err = l1_rel(U.cpu().numpy(), Uo)
    assert err < 1e-6, err
    status, st = s.stats()
    assert status == 0


def test_split_matches_fp64_at_benchmark_size(gpu_lib):
    """512^2, p = 3 advected wave, 20 SSPRK3 steps: split vs FP64 GPU paths (the FP64 path
    matches the oracle to 1e-11), L1 difference below 1e-6 relative."""
    from paper_2205_00095_gb300 import Solver
    spec = wl.advected_wave(n=512, degree=3, c2p="analytic")
    st = torch.cuda.Stream()
    a = Solver(spec, stream=st)
    b = Solver(dict(spec, precision="split"), stream=st)
    U = gpu_state(a, spec)
    V = U.clone()
    dt = a.cfl_dt(0.2)
    a.step(U, dt, 20)
    b.step(V, dt, 20)
    st.synchronize()
    err = float((U - V).abs().sum() / U.abs().sum())
    assert err < 1e-6, err


def test_split_error_against_the_exact_wave_equals_fp64(gpu_lib):
    """Advected wave 64^2, p = 3, 100 SSPRK3 steps: the relative L1 errors of the FP64 and the
    split-precision states against the exact translated wave agree to 1e-6."""
    from paper_2205_00095_gb300 import Solver
    spec = wl.advected_wave(n=64, degree=3, c2p="analytic")
    st = torch.cuda.Stream()
    a = Solver(spec, stream=st)
    b = Solver(dict(spec, precision="split"), stream=st)
    U = gpu_state(a, spec)
    V = U.clone()
    dt = a.cfl_dt(0.2)
    a.step(U, dt, 100)
    b.step(V, dt, 100)
    with torch.cuda.stream(st):
        Ue = a.initial_state(wl.advected_wave_ic(spec, a.node_coords_device(), 100 * dt))
    st.synchronize()
    nrm = float(Ue.abs().sum())
    e64 = float((U - Ue).abs().sum()) / nrm
    esp = float((V - Ue).abs().sum()) / nrm
    assert e64 < 1e-6  # the wave is resolved
    assert abs(esp - e64) <= 1e-6, (esp, e64)
