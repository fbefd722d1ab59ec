"""ctypes binding of libdgsrhd.so (include/dgsrhd.h): argument marshalling only.

Every function of the C ABI is exposed under its own name.  Device arrays are passed as
integer addresses (``tensor.data_ptr()``); streams as ``cudaStream_t`` integers.  The library
must have been built (``paper_2205_00095_gb300.build.build()``); loading fails loudly if it
is missing.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

DGSRHD_OK = 0
DGSRHD_EINVAL = 1
DGSRHD_ECUDA = 2
DGSRHD_ENOMEM = 3
DGSRHD_EC2P_NOCONV = 4
DGSRHD_EUNPHYS_MEAN = 5
DGSRHD_EBADSTATE = 6

EOS = {"ideal": 0, "tm": 1, "taub_matthews": 1}
C2P = {"analytic": 0, "iterative": 1, "default": 2}
FLUX = {"llf": 0, "hll": 1, "hllc": 2}
BC = {"periodic": 0, "dirichlet": 1, "outflow": 2, "reflect": 3}
PRECISION = {"fp64": 0, "split": 1, "3xtf32": 1}
NODES = {"gl": 0, "gll": 1}
KERNEL_KINDS = ("volume", "face", "update", "enforce", "pointwise", "vjp")
PROBE = {"dfma": 0, "ddiv": 1, "dsqrt": 2, "drsqrt": 3, "drcbrt": 4, "recip": 5, "sqrt": 6,
         "rcbrt": 7, "ffma": 8, "rsqrt": 9}


class dgsrhd_config(ctypes.Structure):
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
        ("precision", ctypes.c_int32),
        ("nodes", ctypes.c_int32),
        ("limiter", ctypes.c_int32),
        ("limiter_alpha", ctypes.c_double),
    ]


STAT_FIELDS = ("c2p_calls", "c2p_iters_total", "c2p_iters_max", "c2p_nonconverged",
               "c2p_invalid_input", "face_guard_hits", "enforced_cells", "mean_inadmissible_cells",
               "limited_cells")


class dgsrhd_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in STAT_FIELDS]

    def as_dict(self):
        """The counters as {name: int}."""
        return {n: int(getattr(self, n)) for n in STAT_FIELDS}


_lib = None
LIB_PATH = _build.LIB


def load() -> ctypes.CDLL:
    """Load libdgsrhd.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "dgsrhd_create": (i32, [P(dgsrhd_config), vp, P(vp)]),
        "dgsrhd_destroy": (None, [vp]),
        "dgsrhd_set_stream": (i32, [vp, vp]),
        "dgsrhd_state_shape": (i32, [vp, P(i64), P(i64), P(i64)]),
        "dgsrhd_node_coords": (i32, [vp, vp]),
        "dgsrhd_prim2cons": (i32, [vp, vp, vp]),
        "dgsrhd_con2prim": (i32, [vp, vp, vp, vp]),
        "dgsrhd_rhs": (i32, [vp, vp, vp]),
        "dgsrhd_enforce": (i32, [vp, vp, vp]),
        "dgsrhd_step": (i32, [vp, vp, d, i32]),
        "dgsrhd_step_host": (i32, [vp, vp, d, i32]),
        "dgsrhd_rhs_vjp": (i32, [vp, vp, vp, vp]),
        "dgsrhd_enforce_vjp": (i32, [vp, vp, vp, vp]),
        "dgsrhd_cfl_dt": (i32, [vp, d, P(d)]),
        "dgsrhd_get_stats": (i32, [vp, P(dgsrhd_stats), i32]),
        "dgsrhd_kernel_launches": (i64, [vp]),
        "dgsrhd_set_profiling": (i32, [vp, i32]),
        "dgsrhd_kernel_times": (i32, [vp, P(d), P(i64), i32]),
        "dgsrhd_status_string": (ctypes.c_char_p, [i32]),
        "dgsrhd_rhs_noalloc": (i32, [P(dgsrhd_config), vp, vp, vp, P(dgsrhd_stats)]),
        "dgsrhd_step_stage": (i32, [vp, vp, vp, vp, i32, d, vp, vp]),
        "dgsrhd_stage_save_size": (i32, [vp, P(i64)]),
        "dgsrhd_stage_vjp": (i32, [vp, vp, vp, vp, vp, vp, vp, i32, d]),
        "dgsrhd_con2prim_vjp": (i32, [vp, vp, vp, vp]),
        "dgsrhd_math_check": (i32, [vp, i64, vp, vp]),
        "dgsrhd_mean_square_velocity": (i32, [vp, vp, i32, P(d)]),
        "dgsrhd_arith_probe": (i32, [i32, i64, vp, i64, vp, P(i64)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names declared in include/dgsrhd.h that the binding expects the library to export."""
    return [
        "dgsrhd_create", "dgsrhd_destroy", "dgsrhd_set_stream", "dgsrhd_state_shape",
        "dgsrhd_node_coords", "dgsrhd_prim2cons", "dgsrhd_con2prim", "dgsrhd_rhs",
        "dgsrhd_enforce", "dgsrhd_step", "dgsrhd_step_host", "dgsrhd_rhs_vjp",
        "dgsrhd_enforce_vjp", "dgsrhd_cfl_dt", "dgsrhd_get_stats", "dgsrhd_kernel_launches",
        "dgsrhd_set_profiling", "dgsrhd_kernel_times", "dgsrhd_status_string",
        "dgsrhd_rhs_noalloc", "dgsrhd_step_stage", "dgsrhd_stage_save_size", "dgsrhd_stage_vjp",
        "dgsrhd_con2prim_vjp", "dgsrhd_math_check", "dgsrhd_mean_square_velocity",
        "dgsrhd_arith_probe",
    ]


def _enum(table, v):
    return int(v) if isinstance(v, int) else table[v]


LIMITER = {"none": 0, "moe": 1, "scaling": 1, "minmod": 2}
ENFORCE = {"off": 0, "nodes": 1, "faces": 2}


def _enforce(v) -> int:
    """Physicality operator of a spec: False/0 off, True/1 on the nodes, "faces"/2 on the nodes
    and the face points of the element's conserved polynomial."""
    if isinstance(v, str):
        return ENFORCE[v]
    return 2 if v == 2 else int(bool(v))


def _limiter(v) -> int:
    """False / None: none; True or "moe": the scaling limiter; "minmod": the minmod limiter."""
    if v is None:
        return 0
    if isinstance(v, str):
        return LIMITER[v]
    return int(v)


def make_config(spec: dict) -> dgsrhd_config:
    """Problem description (plain dict) -> dgsrhd_config."""
    c = dgsrhd_config()
    c.dim = int(spec["dim"])
    c.degree = int(spec["degree"])
    n = list(spec["n_elem"]) + [1] * (3 - len(spec["n_elem"]))
    lo = list(spec.get("lo", [0.0] * c.dim)) + [0.0] * (3 - c.dim)
    hi = list(spec.get("hi", [1.0] * c.dim)) + [1.0] * (3 - c.dim)
    for k in range(3):
        c.n_elem[k] = int(n[k])
        c.lo[k] = float(lo[k])
        c.hi[k] = float(hi[k])
    c.eos = _enum(EOS, spec.get("eos", "ideal"))
    c.gamma_ad = float(spec.get("gamma_ad", 5.0 / 3.0))
    c.c2p = _enum(C2P, spec.get("c2p", "default"))
    c.c2p_max_iter = int(spec.get("c2p_max_iter", 0))
    c.c2p_rtol = float(spec.get("c2p_rtol", 0.0))
    c.flux = _enum(FLUX, spec.get("flux", "llf"))
    c.rk_stages = int(spec.get("rk_stages", 3))
    bc = spec.get("bc", [("periodic", "periodic")] * c.dim)
    for k in range(3):
        for s in range(2):
            c.bc[k][s] = _enum(BC, bc[k][s]) if k < len(bc) else 0
    bcs = spec.get("bc_state")
    if bcs is not None:
        for k in range(len(bcs)):
            for s in range(2):
                for v in range(5):
                    c.bc_state[k][s][v] = float(bcs[k][s][v])
    c.enforce = _enforce(spec.get("enforce", True))
    c.precision = _enum(PRECISION, spec.get("precision", "fp64"))
    c.nodes = _enum(NODES, spec.get("nodes", "gl"))
    c.limiter = _limiter(spec.get("limiter", False))
    c.limiter_alpha = float(spec.get("limiter_alpha", 50.0))
    return c


class DGSRHDError(RuntimeError):
    def __init__(self, fn, status):
        msg = load().dgsrhd_status_string(int(status)).decode()
        super().__init__(f"{fn} returned {status} ({msg})")
        self.status = status


def check(fn: str, status: int) -> int:
    """Raise DGSRHDError unless status is DGSRHD_OK."""
    if status != DGSRHD_OK:
        raise DGSRHDError(fn, status)
    return status
