"""Exact solution of the 1D special-relativistic Riemann problem with transverse velocity, for the
ideal and the Taub-Matthews equations of state.  TEST INFRASTRUCTURE ONLY (part of the oracle):
it is the reference for the paper's Riemann problem 3 (Sec. 4.2, a blast into a state moving
transversally at 0.99) and for the Taub-Matthews blast wave (Sec. 4.3, the test after the 1D
Riemann problems: transverse velocity on both sides, the three equations of state compared).

States are primitive (rho, v_x, v_t, P), c = 1; v_t is the velocity along y.

Method (the exact Riemann solution of Pons, Marti & Mueller 2000, restated from the equations
of the 1D system rather than from their closed forms):
  * a rarefaction is a simple wave U(xi), xi = x/t, so dF = xi dU along it with xi the
    acoustic speed lambda- (left wave) or lambda+ (right wave) of the state.  The energy and
    x-momentum components of dF = xi dU, with Q = rho h W^2, combine to
    Q (v_x - xi) dv_x + (1 - v_x xi) dP = 0, which with the closed form of lambda-+ reduces to
    dv_x/dP = -+ sqrt(1 - v_x^2 - c_s^2 v_t^2) / (rho h W c_s).  The wave is isentropic
    (dh = dP/rho, so drho/dP = 1/(h c_s^2), c_s^2 = h_rho / (h (1/rho - h_P))), and the
    transverse-momentum component gives u_t h = const (u = W v).  The curve is integrated in
    ln P from the outer state;
  * independently of that reduction, ``jacobian`` forms the quasi-linear matrix
    A = (dU/dY)^-1 dF/dY in Y = (rho, u_x, u_t, P) by complex-step differentiation of the
    definitions of U and F (Eq. primitive_to_conserved, Eq. srhd_flux); its acoustic
    eigenpairs check the closed forms (the tests use it, the solution does not);
  * a shock satisfies the Rankine-Hugoniot conditions [F] = V_s [U].  The Taub adiabat
    [h^2] = (h_b/rho_b + h_a/rho_a)[P] gives rho_b (one root in (rho_a, inf) for both
    equations of state); the invariant mass flux j = W_s rho W (V_s - v_x) has
    j^2 = -[P]/[h/rho]; the normal-momentum and energy conditions give
    [h W v_x] = W_s [P]/j and [h W] = W_s V_s [P]/j; the transverse-momentum condition gives
    [h W v_t] = 0;
  * the middle pressure is the root of v_x,left(P) - v_x,right(P); across the contact P and
    v_x are continuous, rho and v_t jump.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import solve_ivp
from scipy.optimize import brentq

_CSTEP = 1e-30


class GeneralExactRiemann:
    def __init__(self, left, right, eos: str = "ideal", gamma_ad: float = 5.0 / 3.0,
                 x0: float = 0.5):
        self.eos = {"ideal": "ideal", "tm": "tm", "taub_matthews": "tm"}[eos]
        self.G = float(gamma_ad)
        self.x0 = float(x0)
        self.L = tuple(float(v) for v in left)
        self.R = tuple(float(v) for v in right)
        self._curves = {}
        self._solve()

    # -- equation of state (Sec. 2.2) ------------------------------------------
    def h(self, rho, p):
        """Specific enthalpy; complex arguments are allowed (complex-step derivatives)."""
        th = p / rho
        if self.eos == "ideal":
            return 1.0 + self.G / (self.G - 1.0) * th
        return 2.5 * th + 1.5 * np.sqrt(th * th + 4.0 / 9.0)

    # -- conserved variables and x-flux from the primitive ---------------------
    # The rarefaction curves use Y = (rho, u_x, u_t, P) with the four-velocity u = W v in place of
    # v: near |v| = 1 the Jacobians in v lose digits to 1 - v^2, those in u do not.
    def cons(self, Y):
        rho, ux, ut, p = Y
        lor = np.sqrt(1.0 + ux * ux + ut * ut)
        rhw = rho * self.h(rho, p) * lor
        return np.array([rho * lor, rhw * ux, rhw * ut, rhw * lor - p])

    def flux(self, Y):
        rho, ux, ut, p = Y
        U = self.cons(Y)
        vx = ux / np.sqrt(1.0 + ux * ux + ut * ut)
        return np.array([U[0] * vx, U[1] * vx + p, U[2] * vx, U[1]])

    def jacobian(self, Y):
        """A = (dU/dY)^-1 dF/dY at Y, by complex-step differentiation of cons and flux."""
        Y = np.asarray(Y, dtype=np.float64)
        Yc = np.repeat(Y[:, None], 4, axis=1).astype(np.complex128)
        Yc[np.arange(4), np.arange(4)] += 1j * _CSTEP
        dU = self.cons(Yc).imag / _CSTEP
        dF = self.flux(Yc).imag / _CSTEP
        return np.linalg.solve(dU, dF)

    def acoustic(self, Y, sign):
        """(lambda, r): the acoustic eigenvalue lambda- (sign -1) or lambda+ (sign +1) of A at
        Y = (rho, u_x, u_t, P) and its right eigenvector scaled to unit pressure component."""
        lam, R = np.linalg.eig(self.jacobian(Y))
        k = int(np.argmin(lam.real)) if sign < 0 else int(np.argmax(lam.real))
        r = R[:, k].real
        return float(lam[k].real), r / r[3]

    @staticmethod
    def to_u(W):
        rho, vx, vt, p = W
        lor = 1.0 / math.sqrt(1.0 - vx * vx - vt * vt)
        return (rho, lor * vx, lor * vt, p)

    @staticmethod
    def to_v(Y):
        rho, ux, ut, p = Y
        lor = math.sqrt(1.0 + ux * ux + ut * ut)
        return (rho, ux / lor, ut / lor, p)

    def lam(self, W, sign):
        """Acoustic eigenvalue at the primitive W = (rho, v_x, v_t, P), from the Jacobian."""
        return self.acoustic(self.to_u(W), sign)[0]

    # -- rarefaction curves --------------------------------------------------
    def cs2(self, rho, p):
        """Sound speed squared from the EOS alone: (dP/drho at constant entropy) / h, with the
        isentrope dh = dP/rho; the partial derivatives of h by complex step."""
        h = self.h(rho, p)
        h_rho = self.h(rho + 1j * _CSTEP, p).imag / _CSTEP
        h_p = self.h(rho, p + 1j * _CSTEP).imag / _CSTEP
        return h_rho / (h * (1.0 / rho - h_p))

    def lam_closed(self, W, sign):
        """lambda-+ = [v_x (1 - c^2) -+ c sqrt((1 - v^2)(1 - v_x^2 - v_t^2 c^2))] / (1 - v^2 c^2)."""
        rho, vx, vt, p = W
        c2 = self.cs2(rho, p)
        v2 = vx * vx + vt * vt
        root = math.sqrt(c2 * (1.0 - v2) * (1.0 - vx * vx - vt * vt * c2))
        return (vx * (1.0 - c2) + sign * root) / (1.0 - v2 * c2)

    def _curve(self, state, sign, p_min):
        """The simple-wave curve through `state` of the family `sign`, integrated in s = ln P from
        P_a down to p_min with (ln rho, v_x) as unknowns (u_t = u_t,a h_a / h); dense output."""
        key = (state, sign)
        if key in self._curves and self._curves[key][0] <= p_min:
            return self._curves[key][1]
        rho_a, vx_a, vt_a, p_a = state
        A = self.h(rho_a, p_a) * vt_a / math.sqrt(1.0 - vx_a * vx_a - vt_a * vt_a)

        def rhs(s, y):
            p = math.exp(s)
            rho, vx = math.exp(y[0]), y[1]
            h = self.h(rho, p)
            c2 = self.cs2(rho, p)
            ut = A / h
            lor = math.sqrt((1.0 + ut * ut) / (1.0 - vx * vx))
            vt = ut / lor
            return [p / (rho * h * c2),
                    sign * p * math.sqrt(1.0 - vx * vx - c2 * vt * vt) / (rho * h * lor * math.sqrt(c2))]

        sol = solve_ivp(rhs, (math.log(p_a), math.log(p_min)), [math.log(rho_a), vx_a],
                        method="DOP853", rtol=1e-13, atol=1e-14, dense_output=True)
        if not sol.success:
            raise RuntimeError(f"rarefaction curve: {sol.message}")
        self._curves[key] = (p_min, sol.sol, A)
        return sol.sol

    def _rarefaction(self, state, p, sign):
        if p == state[3]:
            return tuple(state)
        y = self._curve(state, sign, p)(math.log(p))
        rho, vx = math.exp(y[0]), float(y[1])
        ut = self._curves[(state, sign)][2] / self.h(rho, p)
        lor = math.sqrt((1.0 + ut * ut) / (1.0 - vx * vx))
        return (rho, vx, ut / lor, p)

    # -- shocks --------------------------------------------------------------
    def _shock(self, state, p_b, sign):
        """(W_b, V_s) behind a shock of the family `sign` from `state` to p_b > P_a."""
        rho_a, vx_a, vt_a, p_a = state
        h_a = self.h(rho_a, p_a)
        dp = p_b - p_a

        def taub(rho_b):
            hb = self.h(rho_b, p_b)
            return hb * hb - h_a * h_a - (hb / rho_b + h_a / rho_a) * dp

        hi = 2.0 * rho_a
        while taub(hi) > 0.0:
            hi *= 2.0
        rho_b = brentq(taub, rho_a, hi, xtol=1e-300, rtol=1e-15, maxiter=500)
        h_b = self.h(rho_b, p_b)
        j2 = -dp / (h_b / rho_b - h_a / rho_a)
        lor_a = 1.0 / math.sqrt(1.0 - vx_a * vx_a - vt_a * vt_a)
        m2 = rho_a * rho_a * lor_a * lor_a
        Vs = (m2 * vx_a + sign * math.sqrt(j2) * math.sqrt(j2 + m2 * (1.0 - vx_a * vx_a))) / (m2 + j2)
        Ws = 1.0 / math.sqrt(1.0 - Vs * Vs)
        j = sign * math.sqrt(j2)
        hW = h_a * lor_a + Ws * Vs * dp / j
        vx_b = (h_a * lor_a * vx_a + Ws * dp / j) / hW
        A = h_a * lor_a * vt_a
        vt_b = math.copysign(math.sqrt(A * A * (1.0 - vx_b * vx_b) / (h_b * h_b + A * A)), vt_a) \
            if A != 0.0 else 0.0
        return (rho_b, vx_b, vt_b, p_b), Vs

    def _behind(self, state, p, sign):
        if p <= state[3]:
            return self._rarefaction(state, p, sign), None
        return self._shock(state, p, sign)

    # -- the middle state -----------------------------------------------------
    def _solve(self):
        def f(p):
            return self._behind(self.L, p, -1)[0][1] - self._behind(self.R, p, +1)[0][1]

        lo = 0.5 * min(self.L[3], self.R[3])
        while f(lo) <= 0.0:
            lo *= 0.1
            if lo < 1e-12 * min(self.L[3], self.R[3]):
                raise ValueError("the two rarefactions open a vacuum")
        hi = 10.0 * max(self.L[3], self.R[3])
        while f(hi) > 0.0:
            hi *= 10.0
        self.p_star = brentq(f, lo, hi, xtol=1e-300, rtol=1e-15, maxiter=500)
        self.WLs, self.Vs_L = self._behind(self.L, self.p_star, -1)
        self.WRs, self.Vs_R = self._behind(self.R, self.p_star, +1)
        self.v_star = 0.5 * (self.WLs[1] + self.WRs[1])

    # -- sampling -------------------------------------------------------------
    def fan_edges(self, sign):
        """(head, tail) speeds of the rarefaction of the family `sign`, or None for a shock."""
        if sign < 0:
            return None if self.Vs_L is not None else (self.lam_closed(self.L, -1),
                                                        self.lam_closed(self.WLs, -1))
        return None if self.Vs_R is not None else (self.lam_closed(self.R, +1),
                                                    self.lam_closed(self.WRs, +1))

    def _fan(self, state, xi, sign):
        def g(s):
            return self.lam_closed(self._rarefaction(state, math.exp(s), sign), sign) - xi

        s = brentq(g, math.log(self.p_star), math.log(state[3]), xtol=1e-15, rtol=1e-15,
                   maxiter=500)
        return self._rarefaction(state, math.exp(s), sign)

    def sample_xi(self, xi: float):
        """Primitive (rho, v_x, v_t, P) at x/t = xi (the interface at xi = 0)."""
        if xi <= self.v_star:
            if self.Vs_L is not None:
                return self.L if xi < self.Vs_L else self.WLs
            head, tail = self.fan_edges(-1)
            if xi <= head:
                return self.L
            if xi >= tail:
                return self.WLs
            return self._fan(self.L, xi, -1)
        if self.Vs_R is not None:
            return self.R if xi > self.Vs_R else self.WRs
        head, tail = self.fan_edges(+1)
        if xi >= head:
            return self.R
        if xi <= tail:
            return self.WRs
        return self._fan(self.R, xi, +1)

    def sample(self, x, t: float) -> np.ndarray:
        """Primitive W = (rho, vx, vy, vz, P) at positions x (array) and time t > 0, with the
        transverse velocity along y."""
        x = np.asarray(x, dtype=np.float64)
        out = np.zeros((5,) + x.shape)
        for k, xv in enumerate(x.ravel()):
            rho, vx, vt, p = self.sample_xi((xv - self.x0) / t)
            idx = np.unravel_index(k, x.shape)
            out[(0,) + idx] = rho
            out[(1,) + idx] = vx
            out[(2,) + idx] = vt
            out[(4,) + idx] = p
        return out
