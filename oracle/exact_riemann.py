"""Exact solution of the 1D special-relativistic Riemann problem (ideal EOS, no transverse
velocity).  TEST INFRASTRUCTURE ONLY (part of the oracle): it is the reference the blast-wave
problem of Sec. 4.2 (problem 1) is measured against.

Method (Marti & Mueller 1994, restated from the published method):
  * each outer state a is connected to the middle pressure p by a rarefaction (p < p_a) or a
    shock (p > p_a);
  * rarefaction: isentropic (P / rho^Gamma fixed); the rapidity phi = atanh(v) changes by
    -+ int c_s d rho / rho along it (a Riemann invariant of the simple wave);
  * shock: the Taub adiabat [h^2] = (h_b/rho_b + h_a/rho_a)(p_b - p_a) gives the post-shock
    enthalpy, the mass flux is j^2 = -[p] / [h/rho], the shock speed and post-shock velocity
    follow from the jump conditions;
  * the middle pressure is the root of v_left(p) - v_right(p); the solution is sampled on
    x/t.
Units c = 1.  States are (rho, v, P)."""
from __future__ import annotations

import math
import warnings

import numpy as np
from scipy.integrate import quad
from scipy.optimize import brentq


class ExactRiemann:
    def __init__(self, left, right, gamma_ad: float, x0: float = 0.5):
        self.G = float(gamma_ad)
        self.x0 = float(x0)
        self.L = tuple(float(v) for v in left)
        self.R = tuple(float(v) for v in right)
        self._solve()

    # -- equation of state -------------------------------------------------
    def h(self, rho, p):
        return 1.0 + self.G / (self.G - 1.0) * p / rho

    def cs(self, rho, p):
        return math.sqrt(self.G * p / (rho * self.h(rho, p)))

    # -- rarefaction ---------------------------------------------------------
    def _rarefaction(self, state, p, sign):
        """State behind a rarefaction from `state` to pressure p; sign -1 for the left wave
        (phi rises as the pressure falls), +1 for the right wave."""
        rho_a, v_a, p_a = state
        K = p_a / rho_a ** self.G
        rho = (p / K) ** (1.0 / self.G)
        with warnings.catch_warnings():
            # near p_a the interval is tiny and quad reports round-off; its value is exact enough
            warnings.simplefilter("ignore")
            integral, _ = quad(lambda r: self.cs(r, K * r ** self.G) / r, rho_a, rho,
                               epsabs=1e-15, epsrel=1e-13, limit=200)
        phi = math.atanh(v_a) + sign * integral
        return rho, math.tanh(phi)

    # -- shock -----------------------------------------------------------
    def _shock(self, state, p_b, sign):
        """(rho_b, v_b, V_s) behind a shock from `state` to p_b > p_a; sign -1 left, +1 right."""
        rho_a, v_a, p_a = state
        h_a = self.h(rho_a, p_a)
        k = (self.G - 1.0) / self.G
        dp = p_b - p_a
        A = 1.0 - k * dp / p_b
        B = k * dp / p_b
        C = -h_a * h_a - dp * h_a / rho_a
        h_b = (-B + math.sqrt(B * B - 4.0 * A * C)) / (2.0 * A)
        rho_b = self.G * p_b / ((self.G - 1.0) * (h_b - 1.0))
        j2 = -dp / (h_b / rho_b - h_a / rho_a)
        j = sign * math.sqrt(j2)
        W_a = 1.0 / math.sqrt(1.0 - v_a * v_a)
        Vs = (rho_a ** 2 * W_a ** 2 * v_a + sign * math.sqrt(j2) * math.sqrt(j2 + rho_a ** 2)) / (
            rho_a ** 2 * W_a ** 2 + j2)
        W_s = 1.0 / math.sqrt(1.0 - Vs * Vs)
        v_b = (h_a * W_a * v_a + W_s * dp / j) / (h_a * W_a + dp * (W_s * v_a / j + 1.0 / (rho_a * W_a)))
        return rho_b, v_b, Vs

    def _behind(self, state, p, sign):
        if p <= state[2]:
            rho, v = self._rarefaction(state, p, sign)
            return rho, v, None
        return self._shock(state, p, sign)

    def _solve(self):
        def f(p):
            return self._behind(self.L, p, -1)[1] - self._behind(self.R, p, +1)[1]

        lo = 1e-14 * min(self.L[2], self.R[2])
        hi = 10.0 * max(self.L[2], self.R[2])
        while f(hi) > 0.0:
            hi *= 10.0
        self.p_star = brentq(f, lo, hi, xtol=1e-300, rtol=1e-15, maxiter=500)
        self.rho_Ls, self.v_star, self.Vs_L = self._behind(self.L, self.p_star, -1)
        self.rho_Rs, v_r, self.Vs_R = self._behind(self.R, self.p_star, +1)

    # -- wavespeeds inside a fan ---------------------------------------------
    def _lambda(self, rho, v, p, sign):
        c = self.cs(rho, p)
        return (v + sign * c) / (1.0 + sign * v * c)

    def _fan(self, state, xi, sign):
        """Inside a rarefaction fan: the state whose characteristic speed equals xi."""
        rho_a, v_a, p_a = state

        def g(p):
            rho, v = self._rarefaction(state, p, sign)
            return self._lambda(rho, v, p, sign) - xi

        p = brentq(g, self.p_star, p_a, xtol=1e-300, rtol=1e-15, maxiter=500)
        rho, v = self._rarefaction(state, p, sign)
        return rho, v, p

    def sample_xi(self, xi: float):
        """Primitive (rho, v, P) at x/t = xi (the interface at xi = 0)."""
        if xi <= self.v_star:
            st = self.L
            if self.Vs_L is not None:
                return st if xi < self.Vs_L else (self.rho_Ls, self.v_star, self.p_star)
            head = self._lambda(*st, -1)
            tail = self._lambda(self.rho_Ls, self.v_star, self.p_star, -1)
            if xi <= head:
                return st
            if xi >= tail:
                return (self.rho_Ls, self.v_star, self.p_star)
            return self._fan(st, xi, -1)
        st = self.R
        if self.Vs_R is not None:
            return st if xi > self.Vs_R else (self.rho_Rs, self.v_star, self.p_star)
        head = self._lambda(*st, +1)
        tail = self._lambda(self.rho_Rs, self.v_star, self.p_star, +1)
        if xi >= head:
            return st
        if xi <= tail:
            return (self.rho_Rs, self.v_star, self.p_star)
        return self._fan(st, xi, +1)

    def sample(self, x, t: float) -> np.ndarray:
        """Primitive W = (rho, vx, vy, vz, P) at positions x (array) and time t > 0."""
        x = np.asarray(x, dtype=np.float64)
        out = np.zeros((5,) + x.shape)
        flat = x.ravel()
        for k, xv in enumerate(flat):
            rho, v, p = self.sample_xi((xv - self.x0) / t)
            idx = np.unravel_index(k, x.shape)
            out[(0,) + idx] = rho
            out[(1,) + idx] = v
            out[(4,) + idx] = p
        return out
