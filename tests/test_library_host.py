"""CPU tests of the library boundary: it builds, loads, exports every symbol include/dgsrhd.h
declares, and rejects invalid configurations before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2205_00095_gb300 import _lib, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "dgsrhd.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dgsrhd_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dgsrhd_create", "dgsrhd_con2prim", "dgsrhd_rhs", "dgsrhd_enforce",
                     "dgsrhd_step", "dgsrhd_rhs_vjp"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(_lib.exported_symbols()) <= set(declared_functions())


def test_status_strings(lib):
    for code in range(7):
        assert lib.dgsrhd_status_string(code).decode()


def base_spec():
    return dict(dim=2, degree=3, n_elem=[4, 4], eos="ideal", gamma_ad=5.0 / 3.0, rk_stages=3)


@pytest.mark.parametrize("bad", [
    dict(dim=4), dict(dim=0), dict(degree=5), dict(degree=-1), dict(n_elem=[0, 4]),
    dict(gamma_ad=1.0), dict(rk_stages=4), dict(rk_stages=0), dict(flux=7), dict(eos=3),
    dict(bc=[("periodic", "outflow"), ("periodic", "periodic")]),
    dict(bc=[("dirichlet", "outflow"), ("periodic", "periodic")],
         bc_state=[[(1.0, 1.2, 0.0, 0.0, 1.0), (1.0, 0.0, 0.0, 0.0, 1.0)]] * 2),
    dict(lo=[1.0, 0.0], hi=[0.0, 1.0]),
    # 2^30 elements or more: the kernels divide element and face indices in 32 bits
    dict(n_elem=[1 << 15, 1 << 15]), dict(dim=1, n_elem=[1 << 30]),
    dict(dim=3, n_elem=[1 << 10, 1 << 10, 1 << 10]),
    dict(c2p_rtol=-1e-6), dict(c2p_rtol=1.0), dict(c2p_rtol=float("nan")),
])
def test_invalid_configuration_rejected_on_host(lib, bad):
    spec = base_spec()
    spec.update(bad)
    cfg = _lib.make_config(spec)
    ctx = ctypes.c_void_p(1)
    assert lib.dgsrhd_create(ctypes.byref(cfg), None, ctypes.byref(ctx)) == _lib.DGSRHD_EINVAL
    assert not ctx.value


def test_null_arguments_rejected(lib):
    assert lib.dgsrhd_create(None, None, None) == _lib.DGSRHD_EINVAL
    assert lib.dgsrhd_rhs(None, None, None) == _lib.DGSRHD_EINVAL
    assert lib.dgsrhd_step(None, None, 0.1, 1) == _lib.DGSRHD_EINVAL
    lib.dgsrhd_destroy(None)


def test_fit_growth_recovers_a_known_rate():
    """Host-side fit: exp(0.7 + 2.5 t) sampled on [0, 4] gives rate 2.5, intercept 0.7."""
    from paper_2205_00095_gb300 import kh_growth
    t = np.linspace(0.0, 4.0, 81)
    r, a, r2 = kh_growth.fit_growth(t, np.exp(0.7 + 2.5 * t))
    assert abs(r - 2.5) < 1e-12 and abs(a - 0.7) < 1e-12 and r2 > 1.0 - 1e-12


def test_linear_wave_order_fit_recovers_a_known_order():
    """L1(dx) = 3e-9 + 2 dx^3 sampled at four resolutions: the fitted p2 is 3."""
    from paper_2205_00095_gb300 import linear_waves
    dx = np.array([0.2, 0.1, 0.05, 0.025])
    p2, slope = linear_waves.fit_order(dx, 3e-9 + 2.0 * dx ** 3)
    assert abs(p2 - 3.0) < 1e-3 and slope > 2.8


def test_checkpoint_round_trip(tmp_path):
    """save/load keep the state's bits, the spec, the time and the step count; a file that is
    not a checkpoint is refused."""
    import torch

    import workloads as wl
    from paper_2205_00095_gb300 import checkpoint
    spec = wl.kh_single(nx=4, ny=8, degree=2)
    E, Nn = wl.shape(spec)
    U = torch.from_numpy(wl.random_conserved_cells(E, Nn, seed=3))
    p = tmp_path / "state.pt"
    checkpoint.save(str(p), spec, U, t=0.125, step=7)
    d = checkpoint.load(str(p))
    assert torch.equal(d["U"], U) and d["U"].dtype == torch.float64
    assert d["t"] == 0.125 and d["step"] == 7
    assert d["spec"]["n_elem"] == spec["n_elem"] and d["spec"]["name"] == "kh_single"
    torch.save({"not": "a checkpoint"}, str(tmp_path / "other.pt"))
    with pytest.raises(ValueError):
        checkpoint.load(str(tmp_path / "other.pt"))
    with pytest.raises(ValueError):
        checkpoint.save(str(p), spec, U.float())


def test_parity_summary_statistics():
    """Host logic of the con2prim study: per-Lorentz-factor median and quartiles over the states
    that reached parity, extremes, and the counts of exact and unreached states."""
    from paper_2205_00095_gb300 import c2p_study
    lor = np.repeat([1.0, 10.0, 100.0], 4)
    need = np.array([-2, -2, -2, -2, 3, 4, 5, 6, 8, 8, -1, 9])
    s = c2p_study.parity_summary(need, lor)
    assert s["by_gamma_median_q1_q3"][0] == [1.0, None, None, None]
    assert s["by_gamma_median_q1_q3"][1] == [10.0, 4.5, 3.75, 5.25]
    assert s["by_gamma_median_q1_q3"][2][:2] == [100.0, 8.0]
    assert (s["min"], s["max"], s["analytic_exact_states"], s["unreached"]) == (3, 9, 4, 1)


def test_make_config_maps_every_field():
    """The binding's spec -> dgsrhd_config map: names of the enumerations, defaults, and the
    fields added over time (nodes, limiter, limiter_alpha, c2p_rtol)."""
    spec = dict(dim=2, degree=2, n_elem=[3, 5], lo=[-1.0, 0.0], hi=[1.0, 2.0], eos="tm",
                c2p="iterative", c2p_max_iter=17, c2p_rtol=1e-9, flux="hllc", rk_stages=2,
                bc=[("reflect", "outflow"), ("periodic", "periodic")],
                bc_state=[[(1.0, 0.1, 0.0, 0.0, 1.0), (0.5, 0.0, 0.0, 0.0, 0.4)]] * 2,
                enforce=False, precision="3xtf32", nodes="gll", limiter="minmod",
                limiter_alpha=2.5)
    c = _lib.make_config(spec)
    assert (c.dim, c.degree, c.n_elem[0], c.n_elem[1], c.n_elem[2]) == (2, 2, 3, 5, 1)
    assert (c.lo[0], c.hi[1], c.eos, c.c2p, c.c2p_max_iter) == (-1.0, 2.0, 1, 1, 17)
    assert (c.c2p_rtol, c.flux, c.rk_stages) == (1e-9, 2, 2)
    assert (c.bc[0][0], c.bc[0][1], c.bc[1][0]) == (3, 2, 0)
    assert (c.bc_state[0][1][4], c.enforce, c.precision, c.nodes) == (0.4, 0, 1, 1)
    assert (c.limiter, c.limiter_alpha) == (2, 2.5)
    d = _lib.make_config(dict(dim=1, degree=0, n_elem=[4]))
    assert (d.eos, d.c2p, d.flux, d.rk_stages, d.enforce, d.precision) == (0, 2, 0, 3, 1, 0)
    assert (d.limiter, d.c2p_rtol, d.nodes) == (0, 0.0, 0)
    for name, code in (("moe", 1), ("scaling", 1), (True, 1), (False, 0), (None, 0)):
        assert _lib.make_config(dict(dim=1, degree=1, n_elem=[4], limiter=name)).limiter == code


@pytest.mark.parametrize("spec", [
    dict(dim=2, degree=2, n_elem=[3, 5], eos="tm", c2p="iterative", c2p_rtol=1e-9, flux="hllc",
         rk_stages=2, bc=[("reflect", "outflow"), ("periodic", "periodic")],
         bc_state=[[(1.0, 0.1, 0.0, 0.0, 1.0), (0.5, 0.0, 0.0, 0.0, 0.4)]] * 2,
         nodes="gll", limiter="minmod", limiter_alpha=2.5),
    dict(dim=1, degree=0, n_elem=[4]),
    dict(dim=3, degree=1, n_elem=[2, 3, 4], eos="ideal", gamma_ad=1.4, c2p="analytic",
         flux="hll", limiter=True, enforce=False),
])
def test_oracle_and_library_read_a_spec_alike(spec):
    """The two bindings (they share no code) turn one problem description into the same
    configuration, so every parity test compares the same problem."""
    import oracle
    a, b = _lib.make_config(spec), oracle.make_config(spec)
    for f in ("dim", "degree", "eos", "gamma_ad", "c2p", "c2p_max_iter", "c2p_rtol", "flux",
              "rk_stages", "enforce", "nodes", "limiter", "limiter_alpha"):
        assert getattr(a, f) == getattr(b, f), f
    for k in range(3):
        assert a.n_elem[k] == b.n_elem[k] and a.lo[k] == b.lo[k] and a.hi[k] == b.hi[k]
        for s in range(2):
            assert a.bc[k][s] == b.bc[k][s]
            assert list(a.bc_state[k][s]) == list(b.bc_state[k][s])


class _FakeTensor:
    """Stands in for a tensor in the binding's pointer checks (no GPU needed)."""

    def __init__(self, shape, dtype=None, cuda=True, contiguous=True, index=0):
        import torch
        self.shape = tuple(shape)
        self.dtype = torch.float64 if dtype is None else dtype
        self.is_cuda = cuda
        self._contiguous = contiguous
        self.device = torch.device("cuda", index) if cuda else torch.device("cpu")

    def is_contiguous(self):
        return self._contiguous

    def numel(self):
        return int(np.prod(self.shape))

    def data_ptr(self):
        return 4096


def test_binding_checks_every_pointer_it_hands_the_kernels():
    """A host tensor, another dtype, a strided view, another shape or size, or a tensor on
    another GPU is refused before any library call."""
    import torch
    from paper_2205_00095_gb300.solver import _dev_ptr, _vec_ptr
    dev = torch.device("cuda", 0)
    shape = (5, 12, 4)
    assert _dev_ptr(_FakeTensor(shape), "U", shape, dev) == 4096
    for bad in (_FakeTensor(shape, cuda=False), _FakeTensor(shape, dtype=torch.float32),
                _FakeTensor(shape, contiguous=False), _FakeTensor((5, 12, 3)),
                _FakeTensor(shape, index=1)):
        with pytest.raises(ValueError):
            _dev_ptr(bad, "U", shape, dev)
    assert _vec_ptr(None, "s", 12, dev) is None
    assert _vec_ptr(_FakeTensor((12,)), "s", 12, dev) == 4096
    assert _vec_ptr(_FakeTensor((20,)), "save", 12, dev, at_least=True) == 4096
    for bad, at_least in ((_FakeTensor((11,)), False), (_FakeTensor((13,)), False),
                          (_FakeTensor((11,)), True), (_FakeTensor((12,), cuda=False), False),
                          (_FakeTensor((12,), dtype=torch.int64), False),
                          (_FakeTensor((12,), index=1), False)):
        with pytest.raises(ValueError):
            _vec_ptr(bad, "s", 12, dev, at_least=at_least)
