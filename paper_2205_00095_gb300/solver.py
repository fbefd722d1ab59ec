"""Thin torch-facing wrapper of the dgsrhd C ABI.

torch supplies device memory and streams; every step of the method runs in the library's CUDA
kernels.  State tensors are float64, contiguous, shape (5, n_elem, n_node) on the context's
device (layout of include/dgsrhd.h).

Stream contract: every call is ordered on ``Solver.stream``.  Outputs are allocated on that
stream; inputs must be ready on it (create them under ``torch.cuda.stream(solver.stream)`` or
synchronise first), and results must be synchronised (``solver.stream.synchronize()``) before
they are read on another stream or on the host."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dev_ptr(t: torch.Tensor, name: str, shape=None, device: torch.device | None = None) -> int:
    """The device address of t after checking it is a contiguous float64 CUDA tensor of the
    given shape on the given device: the library dereferences it in its kernels."""
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, the solver on {device}")
    return t.data_ptr()


def _vec_ptr(t: torch.Tensor | None, name: str, n: int, device: torch.device | None = None,
             at_least: bool = False) -> int | None:
    """As _dev_ptr for a flat buffer of n doubles (at least n when at_least); None stays None."""
    if t is None:
        return None
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    if t.numel() < n or (t.numel() != n and not at_least):
        raise ValueError(f"{name} holds {t.numel()} doubles, expected {'at least ' if at_least else ''}{n}")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, the solver on {device}")
    return t.data_ptr()


def quadrature_weights_1d(N: int, nodes: str = "gl") -> np.ndarray:
    """The N one-dimensional quadrature weights of the collocated basis on [-1, 1]:
    Gauss-Legendre ('gl'), or Gauss-Lobatto-Legendre ('gll', N >= 2: the end points and the
    roots of P'_{N-1}, weights 2 / (N (N - 1) P_{N-1}(x)^2))."""
    if nodes == "gl":
        return np.polynomial.legendre.leggauss(N)[1]
    P = np.polynomial.legendre.Legendre.basis(N - 1)
    x = np.concatenate([[-1.0], np.sort(P.deriv().roots().real), [1.0]]) if N > 2 else np.array([-1.0, 1.0])
    return 2.0 / (N * (N - 1) * P(x) ** 2)


def node_weights_nd(spec: dict) -> np.ndarray:
    """Tensor-product quadrature weight of every node of an element (x fastest), without the
    (dx/2) Jacobians."""
    dim, N = int(spec["dim"]), int(spec["degree"]) + 1
    w1 = quadrature_weights_1d(N, spec.get("nodes", "gl"))
    w = w1
    for _ in range(dim - 1):
        w = np.multiply.outer(w1, w).ravel()
    return w


class Solver:
    """One mesh and method choice (a dgsrhd context) bound to a CUDA stream."""

    def __init__(self, spec: dict, stream: torch.cuda.Stream | None = None,
                 device: torch.device | str | None = None):
        self.lib = _lib.load()
        self.spec = dict(spec)
        self.device = torch.device(device or "cuda")
        if self.device.type != "cuda":
            raise ValueError(f"the solver runs on a CUDA device, not {self.device}")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.cfg = _lib.make_config(spec)
        ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check("dgsrhd_create", self.lib.dgsrhd_create(ctypes.byref(self.cfg),
                                                          _stream_handle(self.stream),
                                                          ctypes.byref(ctx)))
        self.ctx = ctx
        nv, ne, nn = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        check("dgsrhd_state_shape", self.lib.dgsrhd_state_shape(self.ctx, ctypes.byref(nv),
                                                                ctypes.byref(ne), ctypes.byref(nn)))
        self.shape = (nv.value, ne.value, nn.value)
        self.n_elem, self.n_node = ne.value, nn.value

    def close(self):
        """Free the library context (its scratch and cached graphs); later calls are invalid."""
        if getattr(self, "ctx", None):
            self.lib.dgsrhd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers -----------------------------------------------------------------------
    def _ptr(self, t: torch.Tensor, name: str) -> int:
        return _dev_ptr(t, name, self.shape, self.device)

    def _elem_ptr(self, t: torch.Tensor | None, name: str) -> int | None:
        return _vec_ptr(t, name, self.n_elem, self.device)

    def _save_ptr(self, t: torch.Tensor | None, name: str) -> int | None:
        if t is None:
            return None
        return _vec_ptr(t, name, self.stage_save_size(), self.device, at_least=True)

    def empty(self) -> torch.Tensor:
        """An uninitialised state tensor of the context's shape, allocated on its stream."""
        with torch.cuda.stream(self.stream):
            return torch.empty(self.shape, dtype=torch.float64, device=self.device)

    def node_coords(self) -> np.ndarray:
        """Physical node coordinates as a host array, shape (dim, n_elem, n_node)."""
        X = np.zeros((int(self.spec["dim"]), self.n_elem, self.n_node))
        check("dgsrhd_node_coords", self.lib.dgsrhd_node_coords(self.ctx, X.ctypes.data))
        return X

    # -- the C ABI ---------------------------------------------------------------------
    def prim2cons(self, W: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """Conserved state from the primitive (rho, v_x, v_y, v_z, P) at every node."""
        U = self.empty() if out is None else out
        check("dgsrhd_prim2cons", self.lib.dgsrhd_prim2cons(
            self.ctx, self._ptr(W, "W"), self._ptr(U, "U")))
        return U

    def con2prim(self, U: torch.Tensor, with_iters: bool = False):
        """Primitive (rho, v_x, v_y, v_z, P) at every node by the configured solver; with_iters
        also returns the iteration count of every node."""
        W = self.empty()
        with torch.cuda.stream(self.stream):
            it = torch.empty(self.shape[1:], dtype=torch.int32, device=self.device) if with_iters else None
        check("dgsrhd_con2prim", self.lib.dgsrhd_con2prim(
            self.ctx, self._ptr(U, "U"), self._ptr(W, "W"),
            it.data_ptr() if it is not None else None))
        return (W, it) if with_iters else W

    def rhs(self, U: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """The DG right-hand side R(U) (no physicality operator)."""
        R = self.empty() if out is None else out
        check("dgsrhd_rhs", self.lib.dgsrhd_rhs(self.ctx, self._ptr(U, "U"),
                                                self._ptr(R, "R")))
        return R

    def enforce(self, U: torch.Tensor, with_s: bool = False):
        """The physicality operator in place; with_s also returns each element's factor s."""
        with torch.cuda.stream(self.stream):
            s = torch.empty(self.n_elem, dtype=torch.float64, device=self.device) if with_s else None
        check("dgsrhd_enforce", self.lib.dgsrhd_enforce(
            self.ctx, self._ptr(U, "U"), s.data_ptr() if s is not None else None))
        return (U, s) if with_s else U

    def step(self, U: torch.Tensor, dt: float, nsteps: int = 1) -> torch.Tensor:
        """nsteps SSP-RK steps of size dt in place (limiter and operator after every stage)."""
        check("dgsrhd_step", self.lib.dgsrhd_step(self.ctx, self._ptr(U, "U"),
                                                  float(dt), int(nsteps)))
        return U

    def step_host(self, U_host: torch.Tensor, dt: float, nsteps: int = 1) -> torch.Tensor:
        """As step, with the state in host memory; synchronises the stream.  Pinned memory is
        read and written by the kernels over the host link, other memory is copied."""
        if U_host.is_cuda or U_host.dtype != torch.float64 or not U_host.is_contiguous() or \
                tuple(U_host.shape) != tuple(self.shape):
            raise ValueError("U_host must be a contiguous float64 CPU tensor of the state shape")
        check("dgsrhd_step_host", self.lib.dgsrhd_step_host(self.ctx, U_host.data_ptr(),
                                                            float(dt), int(nsteps)))
        return U_host

    def rhs_vjp(self, U: torch.Tensor, R_bar: torch.Tensor, out: torch.Tensor | None = None):
        """(dR/dU)^T R_bar at U."""
        Ub = self.empty() if out is None else out
        check("dgsrhd_rhs_vjp", self.lib.dgsrhd_rhs_vjp(
            self.ctx, self._ptr(U, "U"), self._ptr(R_bar, "R_bar"),
            self._ptr(Ub, "U_bar")))
        return Ub

    def enforce_vjp(self, s: torch.Tensor, Ut_bar: torch.Tensor, out: torch.Tensor | None = None):
        """Transpose of the operator with the element factors s frozen."""
        Ub = self.empty() if out is None else out
        check("dgsrhd_enforce_vjp", self.lib.dgsrhd_enforce_vjp(
            self.ctx, self._elem_ptr(s, "s"), self._ptr(Ut_bar, "Ut_bar"),
            self._ptr(Ub, "U_bar")))
        return Ub

    def stage_save_size(self) -> int:
        """Doubles of the save buffer step_stage fills for stage_vjp."""
        n = ctypes.c_int64()
        check("dgsrhd_stage_save_size", self.lib.dgsrhd_stage_save_size(self.ctx, ctypes.byref(n)))
        return n.value

    def step_stage(self, Un: torch.Tensor, Uk: torch.Tensor, Uout: torch.Tensor, stage: int,
                   dt: float, s_out: torch.Tensor | None = None,
                   save: torch.Tensor | None = None) -> torch.Tensor:
        """One Shu-Osher stage into Uout; optionally also the operator's element factors (s_out)
        and the forward quantities stage_vjp needs (save)."""
        check("dgsrhd_step_stage", self.lib.dgsrhd_step_stage(
            self.ctx, self._ptr(Un, "Un"), self._ptr(Uk, "Uk"),
            self._ptr(Uout, "Uout"), int(stage), float(dt),
            self._elem_ptr(s_out, "s_out"), self._save_ptr(save, "save")))
        return Uout

    def stage_vjp(self, Uk: torch.Tensor, s: torch.Tensor | None, Z_bar: torch.Tensor,
                  Un_bar: torch.Tensor, Uk_bar: torch.Tensor, stage: int, dt: float,
                  saved: torch.Tensor | None = None):
        """Reverse of one stage at Uk; Un_bar and Uk_bar accumulate."""
        check("dgsrhd_stage_vjp", self.lib.dgsrhd_stage_vjp(
            self.ctx, self._ptr(Uk, "Uk"), self._elem_ptr(s, "s"),
            self._save_ptr(saved, "saved"),
            self._ptr(Z_bar, "Z_bar"), self._ptr(Un_bar, "Un_bar"),
            self._ptr(Uk_bar, "Uk_bar"), int(stage), float(dt)))

    def con2prim_vjp(self, U: torch.Tensor, W_bar: torch.Tensor, out: torch.Tensor | None = None):
        """(dU/dW)^{-T} W_bar at the recovered primitive of U."""
        Ub = self.empty() if out is None else out
        check("dgsrhd_con2prim_vjp", self.lib.dgsrhd_con2prim_vjp(
            self.ctx, self._ptr(U, "U"), self._ptr(W_bar, "W_bar"),
            self._ptr(Ub, "U_bar")))
        return Ub

    def mean_square_velocity(self, U: torch.Tensor, axis: int = 1) -> float:
        """<v_axis^2> = (1/|Omega|) int v_axis^2 dV (the Kelvin-Helmholtz diagnostic of Sec. 4.5),
        evaluated by the library; synchronises the solver's stream."""
        out = ctypes.c_double()
        check("dgsrhd_mean_square_velocity", self.lib.dgsrhd_mean_square_velocity(
            self.ctx, self._ptr(U, "U"), int(axis), ctypes.byref(out)))
        return out.value

    def cfl_dt(self, cfl: float | None = None) -> float:
        """The time step for a CFL number (default: the spec's 'cfl', else 0.2)."""
        dt = ctypes.c_double()
        check("dgsrhd_cfl_dt", self.lib.dgsrhd_cfl_dt(self.ctx, float(cfl or self.spec.get("cfl", 0.2)),
                                                      ctypes.byref(dt)))
        return dt.value

    def stats(self, reset: bool = False):
        """(status, counters); status is the dgsrhd code the counters map to."""
        st = _lib.dgsrhd_stats()
        status = self.lib.dgsrhd_get_stats(self.ctx, ctypes.byref(st), int(reset))
        if status in (_lib.DGSRHD_EINVAL, _lib.DGSRHD_ECUDA):
            raise _lib.DGSRHDError("dgsrhd_get_stats", status)
        return status, st.as_dict()

    def kernel_launches(self) -> int:
        """Kernel launches issued by this context so far."""
        return int(self.lib.dgsrhd_kernel_launches(self.ctx))

    def set_profiling(self, enable: bool):
        """Time every kernel launch with CUDA events (launches are not captured in graphs then)."""
        check("dgsrhd_set_profiling", self.lib.dgsrhd_set_profiling(self.ctx, int(bool(enable))))

    def kernel_times(self, reset: bool = True) -> dict:
        """{kind: (total ms, launches)} of the kernels timed while profiling was on."""
        n = len(_lib.KERNEL_KINDS)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        check("dgsrhd_kernel_times", self.lib.dgsrhd_kernel_times(self.ctx, ms, cnt, int(reset)))
        return {k: (ms[i], int(cnt[i])) for i, k in enumerate(_lib.KERNEL_KINDS)}

    # -- convenience -------------------------------------------------------------------
    def node_coords_device(self) -> torch.Tensor:
        """Node coordinates as a float64 tensor on the solver's device, shape (dim, E, Nn)."""
        with torch.cuda.stream(self.stream):
            return torch.from_numpy(self.node_coords()).to(self.device)

    def initial_state(self, W) -> torch.Tensor:
        """Conserved state from a primitive field (5, n_elem, n_node): a host array is uploaded,
        a device tensor used in place; prim -> cons runs on the device."""
        with torch.cuda.stream(self.stream):
            if isinstance(W, torch.Tensor):
                W = W.to(self.device, torch.float64).contiguous()
            else:
                W = torch.from_numpy(np.ascontiguousarray(W, dtype=np.float64)).to(self.device)
        return self.prim2cons(W)

    def synchronize(self):
        """Wait for the context's stream."""
        self.stream.synchronize()


def arith_probe(kind: str, iters: int, sink: torch.Tensor, stream=None) -> int:
    """Queue the library's arithmetic throughput probe (dgsrhd_arith_probe) on `stream`: one
    kernel of sink.numel() threads (a multiple of 256), each running four independent chains of
    `iters` applications of the operation `kind` (a key of _lib.PROBE).  Returns the number of
    operations; the caller times the kernel with CUDA events on the same stream."""
    lib = _lib.load()
    ops = ctypes.c_int64()
    ptr = _vec_ptr(sink, "sink", sink.numel())
    check("dgsrhd_arith_probe", lib.dgsrhd_arith_probe(_lib.PROBE[kind], int(iters), ptr,
                                                       sink.numel(), _stream_handle(stream),
                                                       ctypes.byref(ops)))
    return ops.value
