"""Differentiation through the solver: torch.autograd functions over the library's hand-written
vector-Jacobian products.

* ``rhs(solver, U)``: R = dU/dt with ``dgsrhd_rhs_vjp`` as its backward.
* ``rollout(solver, U0, dt, nsteps, every)``: nsteps SSP-RK steps; the backward keeps only a
  checkpoint every ``every`` steps from the forward pass (whose last segment is run stage by
  stage and kept whole), recomputes each earlier segment stage by stage
  (``dgsrhd_step_stage``, which also returns the physicality operator's factors and keeps the
  quantities each stage's reverse sweep needs) and runs the stages' reverse sweeps
  (``dgsrhd_stage_vjp``, factors frozen at their forward values).  The recompute of the next
  segment runs on a second library context and stream while the current segment's reverse
  sweep runs on the solver's: both are FP64-bound, and blocks of the two share the SMs.
* ``transverse_kinetic_energy(solver, U)``: J = sum over elements and nodes of
  (prod_d dx_d/2) w_node rho gamma^2 v_y^2, with ``dgsrhd_con2prim_vjp`` in its backward.

Every step of the forward and reverse sweeps runs in the library's kernels; torch holds the
buffers and evaluates the objective's pointwise derivative.
"""
from __future__ import annotations

import numpy as np
import torch

from .solver import Solver


class _OnSolverStream:
    """Run a block on the solver's stream, ordered after the caller's stream and before it."""

    def __init__(self, solver: Solver):
        self.solver = solver

    def __enter__(self):
        self.caller = torch.cuda.current_stream(self.solver.device)
        self.solver.stream.wait_stream(self.caller)
        self.ctx = torch.cuda.stream(self.solver.stream)
        self.ctx.__enter__()

    def __exit__(self, *exc):
        self.ctx.__exit__(*exc)
        self.caller.wait_stream(self.solver.stream)


class _RHS(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, solver):
        U = U.detach().contiguous()
        ctx.solver = solver
        ctx.save_for_backward(U)
        with _OnSolverStream(solver):
            return solver.rhs(U)

    @staticmethod
    def backward(ctx, R_bar):
        (U,) = ctx.saved_tensors
        with _OnSolverStream(ctx.solver):
            return ctx.solver.rhs_vjp(U, R_bar.contiguous()), None


def rhs(solver: Solver, U: torch.Tensor) -> torch.Tensor:
    """R(U) = dU/dt, differentiable in U (its backward is dgsrhd_rhs_vjp)."""
    return _RHS.apply(U, solver)


def _recompute_solver(solver: Solver) -> Solver:
    """A second context for the same problem on its own stream (created once per solver)."""
    aux = getattr(solver, "_recompute_aux", None)
    if aux is None:
        aux = Solver(solver.spec, stream=torch.cuda.Stream(device=solver.device),
                     device=solver.device)
        solver._recompute_aux = aux
    return aux


def _run_segment(solver: Solver, U: torch.Tensor, dt: float, nseg: int, stages: int, nsave: int):
    """nseg steps stage by stage from U, keeping every stage input, operator factor and the
    forward quantities (nodal primitives, face traces) of each stage's RHS; returns the end
    state and the kept data."""
    X, S, SV = [], [], []
    cur = U
    for _ in range(nseg):
        xs, ss, sv = [cur], [], []
        for k in range(stages):
            out = torch.empty_like(cur)
            sk = torch.empty(solver.n_elem, dtype=torch.float64, device=cur.device)
            save = torch.empty(nsave, dtype=torch.float64, device=cur.device)
            solver.step_stage(xs[0], xs[k], out, k, dt, sk, save)
            ss.append(sk)
            sv.append(save)
            if k < stages - 1:
                xs.append(out)
        X.append(xs)
        S.append(ss)
        SV.append(sv)
        cur = out
    return cur, (X, S, SV)


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, solver, dt, nsteps, every):
        stages = int(solver.spec.get("rk_stages", 3))
        nsave = solver.stage_save_size()
        checkpoints = []
        with _OnSolverStream(solver):
            U = U0.detach().clone()
            done = 0
            last = None
            while done < nsteps:
                n = min(every, nsteps - done)
                checkpoints.append((done, U.clone()))
                if done + n < nsteps:
                    solver.step(U, dt, n)
                else:  # the last segment keeps its stage data: no recompute needed for it
                    U, last = _run_segment(solver, U, dt, n, stages, nsave)
                done += n
        ctx.solver, ctx.dt, ctx.nsteps = solver, dt, nsteps
        ctx.checkpoints = checkpoints
        ctx.last = last
        return U

    @staticmethod
    def backward(ctx, U_bar):
        s: Solver = ctx.solver
        dt, nsteps = ctx.dt, ctx.nsteps
        stages = int(s.spec.get("rk_stages", 3))
        nsave = s.stage_save_size()
        aux = _recompute_solver(s)
        main = s.stream
        with _OnSolverStream(s):
            Zb = U_bar.detach().clone().contiguous()
            bounds = [c[0] for c in ctx.checkpoints] + [nsteps]
            nsegs = len(ctx.checkpoints)

            def recompute(seg):
                """Queue segment seg's forward stages on the second context's stream; returns
                its kept data and an event the main stream waits on before using it."""
                start, U = ctx.checkpoints[seg]
                with torch.cuda.stream(aux.stream):
                    _, data = _run_segment(aux, U.clone(), dt, bounds[seg + 1] - start, stages,
                                           nsave)
                    done = torch.cuda.Event()
                    done.record(aux.stream)
                for lst in data:  # the main stream reads these: keep them from early reuse
                    for row in lst:
                        for t in row:
                            t.record_stream(main)
                return data, done

            aux.stream.wait_stream(main)  # the checkpoints were written on the main stream
            pending = None
            for seg in reversed(range(nsegs)):
                if seg == nsegs - 1 and ctx.last is not None:
                    X, S, SV = ctx.last
                    ctx.last = None
                else:
                    if pending is None:
                        pending = recompute(seg)
                    (X, S, SV), done = pending
                    main.wait_event(done)
                # the next segment's recompute overlaps this segment's reverse sweep
                pending = recompute(seg - 1) if seg > 0 else None
                nseg = bounds[seg + 1] - ctx.checkpoints[seg][0]
                # reverse sweep of the segment
                for j in reversed(range(nseg)):
                    Unb = torch.zeros_like(Zb)
                    z = Zb
                    for k in reversed(range(stages)):
                        if k > 0:
                            xb = torch.zeros_like(Zb)
                            s.stage_vjp(X[j][k], S[j][k], z, Unb, xb, k, dt, SV[j][k])
                            z = xb
                        else:
                            s.stage_vjp(X[j][0], S[j][0], z, Unb, Unb, 0, dt, SV[j][0])
                    Zb = Unb
        return Zb, None, None, None, None


def rollout(solver: Solver, U0: torch.Tensor, dt: float, nsteps: int, every: int = 20) -> torch.Tensor:
    """The state after nsteps SSP-RK steps of size dt from U0 (U0 is not modified),
    differentiable in U0; the backward keeps a checkpoint every `every` steps."""
    return _Rollout.apply(U0, solver, float(dt), int(nsteps), int(every))


def node_weights(solver: Solver) -> torch.Tensor:
    """Quadrature weight of every node, (prod_d dx_d / 2) w_a w_b ..., shape (n_elem, n_node)."""
    from .solver import node_weights_nd
    spec = solver.spec
    dim = int(spec["dim"])
    x = solver.node_coords()
    w = node_weights_nd(spec)
    jac = 1.0
    for d in range(dim):
        jac *= (spec["hi"][d] - spec["lo"][d]) / spec["n_elem"][d] / 2.0
    return torch.from_numpy(np.broadcast_to(w * jac, x.shape[1:]).copy()).to(solver.device)


class _KineticY(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, solver, weights):
        U = U.detach().contiguous()
        with _OnSolverStream(solver):
            W = solver.con2prim(U)
            rho, v = W[0], W[1:4]
            g2 = 1.0 / (1.0 - (v * v).sum(0))
            J = (weights * rho * g2 * v[1] * v[1]).sum()
        ctx.solver = solver
        ctx.save_for_backward(U, W, weights)
        return J

    @staticmethod
    def backward(ctx, Jb):
        U, W, wts = ctx.saved_tensors
        with _OnSolverStream(ctx.solver):
            rho, v = W[0], W[1:4]
            g2 = 1.0 / (1.0 - (v * v).sum(0))
            Wb = torch.zeros_like(W)
            Wb[0] = wts * g2 * v[1] * v[1]
            # d(gamma^2)/dv_k = 2 gamma^4 v_k
            for k in range(3):
                Wb[1 + k] = wts * rho * 2.0 * g2 * g2 * v[k] * v[1] * v[1]
            Wb[2] += wts * rho * g2 * 2.0 * v[1]
            Wb *= Jb
            Ub = ctx.solver.con2prim_vjp(U, Wb.contiguous())
        return Ub, None, None


def transverse_kinetic_energy(solver: Solver, U: torch.Tensor) -> torch.Tensor:
    """J = sum of (prod_d dx_d/2) w_node rho gamma^2 v_y^2 over all nodes, differentiable in U."""
    return _KineticY.apply(U, solver, node_weights(solver))
