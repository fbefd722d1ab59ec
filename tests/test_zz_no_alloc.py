"""dgsrhd_rhs_noalloc: the right-hand side for callers that cannot allocate device memory.

It must give the same R as the context-based dgsrhd_rhs (same kernels, scratch in the library's
fixed device array instead of context buffers), on consecutive calls that reuse the shared
scratch, and refuse a mesh larger than that scratch before touching the GPU.  This file is
collected last so that a failure here comes after every other test has run."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_rhs_matches_context_rhs_on_two_consecutive_calls(gpu_lib):
    from paper_2205_00095_gb300 import Solver, _lib

    lib = gpu_lib
    spec = wl.kh2d(nx=16, ny=32, degree=3)          # Taub-Matthews, Brent, HLL, periodic
    s = Solver(spec)                                 # default stream
    X = s.node_coords()
    U1 = s.initial_state(wl.kh2d_ic(spec, X))
    U2 = s.initial_state(wl.kh2d_ic(spec, X, amplitude=0.05))
    cfg = _lib.make_config(spec)
    for U in (U1, U2):
        R_ref = s.rhs(U)
        R = torch.full_like(U, float("nan"))
        st = _lib.dgsrhd_stats()
        status = lib.dgsrhd_rhs_noalloc(ctypes.byref(cfg), None, _ptr(U), _ptr(R), ctypes.byref(st))
        torch.cuda.synchronize()
        assert status == _lib.DGSRHD_OK, status
        assert st.c2p_invalid_input == 0 and st.c2p_calls == U.shape[1] * U.shape[2]
        assert st.c2p_iters_total > 0
        got, want = R.cpu().numpy(), R_ref.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max()
    # the two states differ, so the second call did not return stale scratch
    assert not torch.equal(s.rhs(U1), s.rhs(U2))


def test_noalloc_rhs_without_stats_and_other_dimensions(gpu_lib):
    from paper_2205_00095_gb300 import Solver, _lib

    lib = gpu_lib
    for spec in (wl.smooth_random(1, [257], 4, seed=2), wl.smooth_random(3, [6, 5, 4], 3, eos="tm", seed=3)):
        s = Solver(spec)
        U = s.initial_state(wl.initial_primitive(spec, s.node_coords()))
        R_ref = s.rhs(U)
        R = torch.empty_like(U)
        cfg = _lib.make_config(spec)
        for _ in range(2):
            R.fill_(float("nan"))
            assert lib.dgsrhd_rhs_noalloc(ctypes.byref(cfg), None, _ptr(U), _ptr(R), None) == _lib.DGSRHD_OK
            torch.cuda.synchronize()
            assert np.abs(R.cpu().numpy() - R_ref.cpu().numpy()).max() <= 1e-11 * R_ref.abs().max().item()


def test_noalloc_rhs_rejects_meshes_beyond_the_fixed_scratch(gpu_lib):
    from paper_2205_00095_gb300 import _lib

    lib = gpu_lib
    spec = wl.advected_wave(n=512, degree=3)         # needs about 3.4e8 bytes > 64 MiB
    cfg = _lib.make_config(spec)
    U = torch.zeros(16, dtype=torch.float64, device="cuda")
    R = torch.zeros(16, dtype=torch.float64, device="cuda")
    assert lib.dgsrhd_rhs_noalloc(ctypes.byref(cfg), None, _ptr(U), _ptr(R), None) == _lib.DGSRHD_EINVAL
    assert lib.dgsrhd_rhs_noalloc(ctypes.byref(cfg), None, _ptr(U), _ptr(U), None) == _lib.DGSRHD_EINVAL
    assert lib.dgsrhd_rhs_noalloc(None, None, _ptr(U), _ptr(R), None) == _lib.DGSRHD_EINVAL


def test_noalloc_rhs_runs_the_split_kernels_for_a_split_configuration(gpu_lib):
    """precision = split: the same split-precision kernels as the context's dgsrhd_rhs (the
    per-element reference fluxes live in the fixed scratch too), so the two R agree bit for bit,
    and they differ from the FP64 R at the split form's rounding level."""
    from paper_2205_00095_gb300 import Solver, _lib

    lib = gpu_lib
    spec = dict(wl.kh2d(nx=16, ny=32, degree=3), precision="split")
    s = Solver(spec)
    s64 = Solver(dict(spec, precision="fp64"))
    U = s.initial_state(wl.kh2d_ic(spec, s.node_coords()))
    cfg = _lib.make_config(spec)
    for _ in range(2):
        R_ref = s.rhs(U)
        R = torch.full_like(U, float("nan"))
        assert lib.dgsrhd_rhs_noalloc(ctypes.byref(cfg), None, _ptr(U), _ptr(R), None) == _lib.DGSRHD_OK
        torch.cuda.synchronize()
        assert torch.equal(R, R_ref)
    R64 = s64.rhs(U)
    torch.cuda.synchronize()
    d = (R - R64).abs().max().item() / R64.abs().max().item()
    assert 0.0 < d < 1e-4, d
