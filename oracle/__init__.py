"""Oracle for the DG special-relativistic hydrodynamics hot path (arXiv 2205.00095).

TEST INFRASTRUCTURE ONLY.  This package is the plain FP64 CPU restatement of the
method that the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it.
It shares no code with the CUDA library and never imports it.

The arithmetic lives in ``dgsrhd_oracle.c`` (plain loops, one routine per
equation of the paper); this module compiles it with gcc on first use and wraps
it with ctypes.  ``exact_riemann.py`` holds the exact 1D Riemann solution used
to check the blast-wave problem, ``exact_riemann_general.py`` the one with
transverse velocity and either equation of state (Riemann problem 3 and the
Taub-Matthews blast wave).

Parity status per function (each is pinned by a ``-m "not gpu"`` test):
  basis (Gauss-Legendre and Gauss-Lobatto-Legendre), EOS, prim2cons, the four
  con2prim solvers, wavespeeds, the LLF, HLL and HLLC fluxes, rhs (periodic,
  Dirichlet, outflow and reflecting boundaries), enforce, the scaling and minmod
  limiters, step, cfl_dt, mean_square_velocity, gamma_eq and both exact Riemann
  solutions: pinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dgsrhd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIBPATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIBPATH) or os.path.getmtime(_LIBPATH) < os.path.getmtime(_SRC):
        tmp = _LIBPATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIBPATH)
    return _LIBPATH


class Config(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("degree", ctypes.c_int32),
        ("n_elem", ctypes.c_int64 * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("eos", ctypes.c_int32),
        ("gamma_ad", ctypes.c_double),
        ("c2p", ctypes.c_int32),
        ("c2p_max_iter", ctypes.c_int32),
        ("c2p_rtol", ctypes.c_double),
        ("flux", ctypes.c_int32),
        ("rk_stages", ctypes.c_int32),
        ("bc", (ctypes.c_int32 * 2) * 3),
        ("bc_state", ((ctypes.c_double * 5) * 2) * 3),
        ("enforce", ctypes.c_int32),
        ("nodes", ctypes.c_int32),
        ("limiter", ctypes.c_int32),
        ("limiter_alpha", ctypes.c_double),
    ]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "c2p_calls", "c2p_iters_total", "c2p_iters_max", "c2p_nonconverged",
        "c2p_invalid_input", "face_guard_hits", "enforced_cells", "mean_inadmissible_cells",
        "limited_cells")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


_EOS = {"ideal": 0, "tm": 1, "taub_matthews": 1}
_C2P = {"analytic": 0, "iterative": 1, "default": 2}
_NODES = {"gl": 0, "gll": 1}
_FLUX = {"llf": 0, "hll": 1, "hllc": 2}
_BC = {"periodic": 0, "dirichlet": 1, "outflow": 2, "reflect": 3}


def _enum(table, v):
    return v if isinstance(v, (int, np.integer)) else table[v]


def _limiter(v) -> int:
    """False / None: none; True or "moe": the scaling limiter; "minmod": the minmod limiter."""
    if v is None:
        return 0
    if isinstance(v, str):
        return {"none": 0, "moe": 1, "scaling": 1, "minmod": 2}[v]
    return int(v)


def _enforce(v) -> int:
    """Physicality operator: False/0 off, True/1 on the nodes, "faces"/2 on the nodes and the
    face points of the element's conserved polynomial."""
    if v == "faces" or v == 2:
        return 2
    return int(bool(v))


def make_config(spec: dict) -> Config:
    """Problem description (plain dict, see ``workloads``) -> oracle struct."""
    c = Config()
    c.dim = int(spec["dim"])
    c.degree = int(spec["degree"])
    n = list(spec["n_elem"]) + [1] * (3 - len(spec["n_elem"]))
    lo = list(spec.get("lo", [0.0] * c.dim)) + [0.0] * (3 - c.dim)
    hi = list(spec.get("hi", [1.0] * c.dim)) + [1.0] * (3 - c.dim)
    for d in range(3):
        c.n_elem[d] = int(n[d])
        c.lo[d] = float(lo[d])
        c.hi[d] = float(hi[d])
    c.eos = _enum(_EOS, spec.get("eos", "ideal"))
    c.gamma_ad = float(spec.get("gamma_ad", 5.0 / 3.0))
    c.c2p = _enum(_C2P, spec.get("c2p", "default"))
    c.c2p_max_iter = int(spec.get("c2p_max_iter", 0))
    c.c2p_rtol = float(spec.get("c2p_rtol", 0.0))
    c.flux = _enum(_FLUX, spec.get("flux", "llf"))
    c.rk_stages = int(spec.get("rk_stages", 3))
    bc = spec.get("bc", [("periodic", "periodic")] * c.dim)
    for d in range(3):
        for s in range(2):
            c.bc[d][s] = _enum(_BC, bc[d][s]) if d < len(bc) else 0
    bcs = spec.get("bc_state")
    if bcs is not None:
        for d in range(len(bcs)):
            for s in range(2):
                for v in range(5):
                    c.bc_state[d][s][v] = float(bcs[d][s][v])
    c.enforce = _enforce(spec.get("enforce", True))
    c.nodes = _enum(_NODES, spec.get("nodes", "gl"))
    c.limiter = _limiter(spec.get("limiter", False))
    c.limiter_alpha = float(spec.get("limiter_alpha", 50.0))
    return c


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            d = ctypes.c_double
            cfg = P(Config)
            st = P(Stats)
            dp = P(d)
            lib.or_gauss_legendre.argtypes = [ctypes.c_int, dp, dp]
            lib.or_basis.argtypes = [ctypes.c_int, dp, dp, dp, dp, dp]
            lib.or_basis_family.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp]
            lib.or_prim2cons.argtypes = [cfg, ctypes.c_int64, dp, dp]
            lib.or_con2prim.argtypes = [cfg, ctypes.c_int64, dp, dp, P(ctypes.c_int32), st]
            lib.or_rhs.argtypes = [cfg, dp, dp, st]
            lib.or_enforce.argtypes = [cfg, dp, dp, st]
            lib.or_step.argtypes = [cfg, dp, d, ctypes.c_int, st]
            lib.or_cfl_dt.argtypes = [cfg, d]
            lib.or_cfl_dt.restype = d
            lib.or_node_coords.argtypes = [cfg, dp]
            lib.or_wavespeeds.argtypes = [cfg, dp, ctypes.c_int, dp, dp]
            lib.or_numerical_flux.argtypes = [cfg, dp, dp, ctypes.c_int, dp]
            lib.or_phys_flux.argtypes = [cfg, dp, ctypes.c_int, dp]
            lib.or_enthalpy.argtypes = [cfg, d, d]
            lib.or_enthalpy.restype = d
            lib.or_cs2.argtypes = [cfg, d, d]
            lib.or_cs2.restype = d
            lib.or_mean_square_velocity.argtypes = [cfg, dp, ctypes.c_int]
            lib.or_mean_square_velocity.restype = d
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def shape(spec: dict):
    """(n_elem_total, nodes_per_element)."""
    dim = int(spec["dim"])
    N = int(spec["degree"]) + 1
    E = int(np.prod([int(x) for x in spec["n_elem"][:dim]]))
    return E, N ** dim


def gauss_legendre(N: int):
    x = np.zeros(N)
    w = np.zeros(N)
    if _load().or_gauss_legendre(N, _ptr(x), _ptr(w)):
        raise ValueError("bad N")
    return x, w


def basis(N: int, nodes: str = "gl") -> dict:
    """Nodes, weights and the tables of the collocated scheme for N Gauss-Legendre ('gl') or
    Gauss-Lobatto-Legendre ('gll', N >= 2) nodes."""
    x, w, em, ep = (np.zeros(N) for _ in range(4))
    Dhat = np.zeros(N * N)
    if _load().or_basis_family(N, _NODES[nodes], _ptr(x), _ptr(w), _ptr(Dhat), _ptr(em), _ptr(ep)):
        raise ValueError("bad N")
    return {"x": x, "w": w, "Dhat": Dhat.reshape(N, N), "em": em, "ep": ep}


def node_coords(spec: dict) -> np.ndarray:
    """Node coordinates, shape (dim, E, Nn)."""
    E, Nn = shape(spec)
    X = np.zeros((int(spec["dim"]), E, Nn))
    if _load().or_node_coords(ctypes.byref(make_config(spec)), _ptr(X)):
        raise ValueError("bad config")
    return X


def prim2cons(spec: dict, W: np.ndarray) -> np.ndarray:
    """W (5, ...) = (rho, vx, vy, vz, P) -> U (5, ...) = (D, Sx, Sy, Sz, tau)."""
    W = _f64(W)
    n = W.size // 5
    U = np.zeros_like(W)
    _load().or_prim2cons(ctypes.byref(make_config(spec)), n, _ptr(W), _ptr(U))
    return U


def con2prim(spec: dict, U: np.ndarray):
    """U (5, ...) -> (W (5, ...), iterations (...), stats dict)."""
    U = _f64(U)
    n = U.size // 5
    W = np.zeros_like(U)
    it = np.zeros(U.shape[1:], dtype=np.int32)
    st = Stats()
    _load().or_con2prim(ctypes.byref(make_config(spec)), n, _ptr(U), _ptr(W),
                        it.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(st))
    return W, it, st.as_dict()


def rhs(spec: dict, U: np.ndarray):
    """dU/dt of the DG semi-discretisation (no physicality operator)."""
    U = _f64(U)
    R = np.zeros_like(U)
    st = Stats()
    rc = _load().or_rhs(ctypes.byref(make_config(spec)), _ptr(U), _ptr(R), ctypes.byref(st))
    if rc:
        raise RuntimeError(f"or_rhs failed ({rc})")
    return R, st.as_dict()


def enforce(spec: dict, U: np.ndarray):
    """Physicality operator on every element; returns (U_new, s per element, stats)."""
    U = _f64(U).copy()
    E, _ = shape(spec)
    s = np.zeros(E)
    st = Stats()
    rc = _load().or_enforce(ctypes.byref(make_config(spec)), _ptr(U), _ptr(s), ctypes.byref(st))
    if rc:
        raise RuntimeError(f"or_enforce failed ({rc})")
    return U, s, st.as_dict()


def step(spec: dict, U: np.ndarray, dt: float, nsteps: int = 1):
    """nsteps SSP-RK steps (with the operator after each stage if enabled)."""
    U = _f64(U).copy()
    st = Stats()
    rc = _load().or_step(ctypes.byref(make_config(spec)), _ptr(U), float(dt), int(nsteps),
                         ctypes.byref(st))
    if rc:
        raise RuntimeError(f"or_step failed ({rc})")
    return U, st.as_dict()


def cfl_dt(spec: dict, cfl: float) -> float:
    return float(_load().or_cfl_dt(ctypes.byref(make_config(spec)), float(cfl)))


def mean_square_velocity(spec: dict, U: np.ndarray, axis: int = 1) -> float:
    """<v_axis^2> = (1/|Omega|) int v_axis^2 dV by the nodal quadrature (Sec. 4.5)."""
    U = _f64(U)
    return float(_load().or_mean_square_velocity(ctypes.byref(make_config(spec)), _ptr(U), int(axis)))


def wavespeeds(spec: dict, Wv, d: int):
    Wv = _f64(Wv)
    lm = ctypes.c_double()
    lp = ctypes.c_double()
    _load().or_wavespeeds(ctypes.byref(make_config(spec)), _ptr(Wv), int(d), ctypes.byref(lm),
                          ctypes.byref(lp))
    return lm.value, lp.value


def numerical_flux(spec: dict, WvL, WvR, d: int) -> np.ndarray:
    WvL, WvR = _f64(WvL), _f64(WvR)
    F = np.zeros(5)
    _load().or_numerical_flux(ctypes.byref(make_config(spec)), _ptr(WvL), _ptr(WvR), int(d), _ptr(F))
    return F


def phys_flux(spec: dict, Wv, d: int) -> np.ndarray:
    Wv = _f64(Wv)
    F = np.zeros(5)
    _load().or_phys_flux(ctypes.byref(make_config(spec)), _ptr(Wv), int(d), _ptr(F))
    return F


def enthalpy(spec: dict, rho: float, P: float) -> float:
    return float(_load().or_enthalpy(ctypes.byref(make_config(spec)), rho, P))


def cs2(spec: dict, rho: float, P: float) -> float:
    return float(_load().or_cs2(ctypes.byref(make_config(spec)), rho, P))


def gamma_eq(spec: dict, rho, P):
    """Equivalent adiabatic index Gamma_eq = (h - 1) / (h - 1 - Theta), Theta = P / rho, c = 1
    (Sec. 2.2 and the Taub-Matthews test of Sec. 4.3, Fig. 9): Gamma for the ideal EOS; between
    4/3 (hot) and 5/3 (cold) for Taub-Matthews.  A diagnostic; rho and P may be arrays."""
    rho, P = np.broadcast_arrays(np.asarray(rho, dtype=np.float64), np.asarray(P, dtype=np.float64))
    hm1 = np.vectorize(lambda r, p: enthalpy(spec, r, p) - 1.0)(rho, P)
    return hm1 / (hm1 - P / rho)
