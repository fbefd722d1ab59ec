// Pointwise physics of the SRHD DG hot path, device side (FP64).
//
// Equations of state (Sec. 2.2), prim -> cons (Eq. primitive_to_conserved), the four
// conserved-to-primitive solvers (Sec. 3), the flux (Eq. srhd_flux), the wavespeeds of
// Sec. 2.4 and the LLF/HLL numerical fluxes, and the admissibility test of Eq. physicality.
// Units c = 1; conserved variables (D, S, tau) with tau = E - D.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "params.h"

namespace dgsrhd {

// ---------------------------------------------------------------------------------------
// Equations of state.  h - 1 is kept apart from the rest mass so that cold states keep
// their internal energy: ideal  h - 1 = Gamma/(Gamma-1) Theta;  Taub-Matthews
// h = 5/2 Theta + 3/2 sqrt(Theta^2 + 4/9)  =>  h - 1 = 5/2 Theta + 3/2 Theta^2/(r + 2/3),
// r = sqrt(Theta^2 + 4/9).
// ---------------------------------------------------------------------------------------
struct EosEval {
  double hm1;  // h - 1
  double cs2;  // sound speed squared
};

__device__ __forceinline__ EosEval eos_eval(const Params& p, double rho, double P) {
  EosEval r;
  const double th = P / rho;
  if (p.eos == 0) {
    r.hm1 = p.alpha * th;
    r.cs2 = p.gamma_ad * th / (1.0 + r.hm1);
  } else {
    const double s = sqrt(fma(th, th, 4.0 / 9.0));
    r.hm1 = 2.5 * th + 1.5 * th * th / (s + 2.0 / 3.0);
    // (3 Th^2 + 5 Th s) / (12 Th^2 + 2 + 12 Th s)
    r.cs2 = th * fma(3.0, th, 5.0 * s) / fma(12.0 * th, th + s, 2.0);
  }
  return r;
}

// Face / node state in the interpolated primitive (rho, u, P), u = gamma v.
struct ConsFlux {
  double U[5];
  double v[3];
  double P;
  double lor;  // Lorentz factor
  double cs2;
};

// prim (rho, u, P) -> conserved state, 3-velocity and sound speed.
// tau = gamma^2 rho h - P - D  written as  D u^2/(gamma + 1) + gamma^2 rho (h - 1) - P.
__device__ __forceinline__ void prim_u_to_cons(const Params& p, const double Wu[5], ConsFlux& c) {
  const double rho = Wu[0], P = Wu[4];
  const double u2 = Wu[1] * Wu[1] + Wu[2] * Wu[2] + Wu[3] * Wu[3];
  const double lor = sqrt(1.0 + u2);
  const double ilor = 1.0 / lor;
  const EosEval e = eos_eval(p, rho, P);
  const double D = lor * rho;
  const double rhoh_lor = rho * (1.0 + e.hm1) * lor;  // S = rho h gamma u
  c.U[0] = D;
  c.U[1] = rhoh_lor * Wu[1];
  c.U[2] = rhoh_lor * Wu[2];
  c.U[3] = rhoh_lor * Wu[3];
  c.U[4] = D * u2 / (lor + 1.0) + lor * lor * rho * e.hm1 - P;
  c.v[0] = Wu[1] * ilor;
  c.v[1] = Wu[2] * ilor;
  c.v[2] = Wu[3] * ilor;
  c.P = P;
  c.lor = lor;
  c.cs2 = e.cs2;
}

// prim (rho, v, P) -> cons; same arithmetic with gamma from v.
__device__ __forceinline__ void prim_v_to_cons(const Params& p, const double W[5], double U[5]) {
  const double v2 = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
  const double lor = 1.0 / sqrt(1.0 - v2);
  const EosEval e = eos_eval(p, W[0], W[4]);
  const double D = lor * W[0];
  const double rhoh_lor2 = W[0] * (1.0 + e.hm1) * lor * lor;
  U[0] = D;
  U[1] = rhoh_lor2 * W[1];
  U[2] = rhoh_lor2 * W[2];
  U[3] = rhoh_lor2 * W[3];
  U[4] = D * lor * lor * v2 / (lor + 1.0) + lor * lor * W[0] * e.hm1 - W[4];
}

// ---------------------------------------------------------------------------------------
// Admissible set (Eq. physicality): D > 0 and q = E - sqrt(D^2 + |S|^2) > 0, evaluated as
// q = tau - |S|^2 / (D + sqrt(D^2 + |S|^2)) (no cancellation of D against the root).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double q_func(double D, double S2, double tau) {
  return tau - S2 / (D + sqrt(fma(D, D, S2)));
}

__device__ __forceinline__ bool admissible(const double U[5]) {
  const double S2 = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
  return U[0] > 0.0 && q_func(U[0], S2, U[4]) > 0.0;
}

// ---------------------------------------------------------------------------------------
// Conserved -> primitive (Sec. 3).  xi = |S|/D, eta = E/D.
// ---------------------------------------------------------------------------------------

// Ideal EOS, closed form: monic quartic beta^4 + a3 beta^3 + a2 beta^2 + a1 beta + a0 with
// the coefficients of Sec. 3.1, its resolvent cubic (i1, i2, i3), Cardano's root x of the
// resolvent (trigonometric form when T < 0), the quadratic factor beta^2 + B beta + C.
__device__ __forceinline__ double beta_ideal_closed_form(double G, double xi, double eta) {
  const double gm1 = G - 1.0;
  const double inv = 1.0 / (gm1 * gm1 * fma(xi, xi, 1.0));
  const double a3 = -2.0 * G * gm1 * xi * eta * inv;
  const double a2 = (G * G * eta * eta + 2.0 * gm1 * xi * xi - gm1 * gm1) * inv;
  const double a1 = -2.0 * G * xi * eta * inv;
  const double a0 = xi * xi * inv;
  const double i1 = -a2;
  const double i2 = a3 * a1 - 4.0 * a0;
  const double i3 = 4.0 * a2 * a0 - a1 * a1 - a3 * a3 * a0;
  const double R = (9.0 * i1 * i2 - 27.0 * i3 - 2.0 * i1 * i1 * i1) * (1.0 / 54.0);
  const double S = (3.0 * i2 - i1 * i1) * (1.0 / 9.0);
  const double T = R * R + S * S * S;
  double x;
  if (T < 0.0) {
    x = 2.0 * pow(R * R - T, 1.0 / 6.0) * cos(atan2(sqrt(-T), R) * (1.0 / 3.0)) - i1 * (1.0 / 3.0);
  } else {
    const double sT = sqrt(T);
    x = cbrt(R + sT) + cbrt(R - sT) - i1 * (1.0 / 3.0);
  }
  const double B = 0.5 * (a3 + sqrt(a3 * a3 - 4.0 * a2 + 4.0 * x));
  const double C = 0.5 * (x - sqrt(x * x - 4.0 * a0));
  return 0.5 * (-B + sqrt(B * B - 4.0 * C));
}

// Ideal EOS, Newton-Raphson on the Riccardi quartic in w, beta = 2w/(1 + w^2)
// (Eqs. iterative_quartic_unknown, iterative_quartic), started from the small-xi series of
// Eq. iterative_cubic_approximation; stop at |dw| <= 1e-14 w; for xi < 1e-4 the series.
__device__ __forceinline__ double w_ideal_newton(double al, double xi, double eta, int max_iter,
                                                 int& iters, bool& conv) {
  const double k1 = al * eta - 1.0;
  const double ik1 = 1.0 / k1;
  const double ik1sq = ik1 * ik1;
  const double series = (al - 1.0) * 0.5 * ik1 * xi +
                        (al - 1.0) * (al - 1.0) * 0.125 * ik1sq * ik1sq *
                            ((al + 3.0) * (al * eta + 1.0) - 4.0 * (al + 1.0)) * xi * xi * xi;
  iters = 0;
  conv = true;
  if (xi < 1e-4) return series;
  double w = fmin(fmax(series, 1e-300), 1.0 - 1e-15);
  const double c4 = (al - 1.0) * xi, c3 = -2.0 * (al * eta + 1.0), c2 = 2.0 * (al + 1.0) * xi,
               c1 = -2.0 * k1, c0 = c4;
  conv = false;
  for (int it = 1; it <= max_iter; ++it) {
    const double Pw = fma(fma(fma(fma(c4, w, c3), w, c2), w, c1), w, c0);
    const double dP = fma(fma(fma(4.0 * c4, w, 3.0 * c3), w, 2.0 * c2), w, c1);
    const double dw = Pw / dP;
    w -= dw;
    iters = it;
    if (fabs(dw) <= 1e-14 * w) {
      conv = true;
      break;
    }
  }
  return w;
}

// Taub-Matthews cubic W^3 + c1 W^2 + c2 W + c3 in W = gamma^2 - 1 (Eq. synge_cubic).
struct Cubic {
  double c1, c2, c3;
};

__device__ __forceinline__ Cubic tm_cubic(double xi, double eta) {
  const double e2 = eta * eta, x2 = xi * xi;
  const double s = e2 + x2;
  const double dm = e2 - x2;
  const double idm2 = 1.0 / (dm * dm);
  const double k = 4.0 * s - (x2 + 1.0);
  Cubic c;
  c.c1 = (s * k - 14.0 * x2 * e2) * 0.5 * idm2;
  c.c2 = (k * k - 57.0 * x2 * e2) * 0.0625 * idm2;
  c.c3 = -9.0 * x2 * e2 * 0.0625 * idm2;
  return c;
}

__device__ __forceinline__ double cubic_at(const Cubic& c, double W) {
  return fma(fma(W + c.c1, W, c.c2), W, c.c3);
}

// Taub-Matthews closed form: discriminant d = Q^3 + R^2, trigonometric root for d < 0,
// Cardano otherwise (Sec. 3.2); clamped to W >= 0.
__device__ __forceinline__ double W_tm_closed_form(double xi, double eta) {
  const Cubic c = tm_cubic(xi, eta);
  const double Q = (3.0 * c.c2 - c.c1 * c.c1) * (1.0 / 9.0);
  const double R = (9.0 * c.c1 * c.c2 - 27.0 * c.c3 - 2.0 * c.c1 * c.c1 * c.c1) * (1.0 / 54.0);
  const double d = Q * Q * Q + R * R;
  double W;
  if (d < 0.0) {
    const double iota = acos(R / sqrt(-Q * Q * Q));
    W = 2.0 * sqrt(-Q) * cos(iota * (1.0 / 3.0)) - c.c1 * (1.0 / 3.0);
  } else {
    const double sd = sqrt(d);
    W = -c.c1 * (1.0 / 3.0) + cbrt(R + sd) + cbrt(R - sd);
  }
  return fmax(W, 0.0);
}

// Taub-Matthews iterative: Brent's zero finder (Brent 1973) on the cubic, bracketed by
// gamma in [1, 200] with the upper end multiplied by 4 (at most 10 times) until the sign
// changes; tolerance 2 eps |b| + 1e-300.
static __device__ __noinline__ double W_tm_brent(double xi, double eta, int max_iter, int& iters,
                                          bool& conv) {
  const Cubic cc = tm_cubic(xi, eta);
  double a = 0.0, b = 200.0 * 200.0 - 1.0;
  double fa = cubic_at(cc, a), fb = cubic_at(cc, b);
  iters = 0;
  conv = false;
  if (fa == 0.0) {
    conv = true;
    return 0.0;
  }
  for (int k = 0; k < 10 && fa * fb > 0.0; ++k) {
    b *= 4.0;
    fb = cubic_at(cc, b);
  }
  if (fa * fb > 0.0) return __longlong_as_double(0x7ff8000000000000LL);
  double c = a, fc = fa, d = b - a, e = d;
  for (int it = 1; it <= max_iter; ++it) {
    iters = it;
    if (fb * fc > 0.0) {
      c = a;
      fc = fa;
      d = b - a;
      e = d;
    }
    if (fabs(fc) < fabs(fb)) {
      a = b;
      b = c;
      c = a;
      fa = fb;
      fb = fc;
      fc = fa;
    }
    const double tol = 2.0 * 2.220446049250313e-16 * fabs(b) + 1e-300;
    const double m = 0.5 * (c - b);
    if (fabs(m) <= tol || fb == 0.0) {
      conv = true;
      return b;
    }
    if (fabs(e) >= tol && fabs(fa) > fabs(fb)) {
      const double s = fb / fa;
      double pp, qq;
      if (a == c) {
        pp = 2.0 * m * s;
        qq = 1.0 - s;
      } else {
        const double q1 = fa / fc, r1 = fb / fc;
        pp = s * (2.0 * m * q1 * (q1 - r1) - (b - a) * (r1 - 1.0));
        qq = (q1 - 1.0) * (r1 - 1.0) * (s - 1.0);
      }
      if (pp > 0.0)
        qq = -qq;
      else
        pp = -pp;
      if (2.0 * pp < fmin(3.0 * m * qq - fabs(tol * qq), fabs(e * qq))) {
        e = d;
        d = pp / qq;
      } else {
        d = m;
        e = m;
      }
    } else {
      d = m;
      e = m;
    }
    a = b;
    fa = fb;
    b += (fabs(d) > tol) ? d : (m > 0.0 ? tol : -tol);
    fb = cubic_at(cc, b);
  }
  return b;
}

// Result of one recovery.
struct Prim {
  double rho, v[3], P;
  double lor;  // Lorentz factor
};

// status: 0 ok, 1 invalid input, 2 not converged / closed form failed.
__device__ __forceinline__ int con2prim(const Params& p, const double U[5], Prim& W, int& iters) {
  const double D = U[0], tau = U[4];
  const double S2 = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
  iters = 0;
  const double nanv = __longlong_as_double(0x7ff8000000000000LL);
  if (!(D > 0.0) || !(q_func(D, S2, tau) > 0.0) || !isfinite(S2) || !isfinite(tau)) {
    W.rho = W.v[0] = W.v[1] = W.v[2] = W.P = W.lor = nanv;
    return 1;
  }
  const double iD = 1.0 / D;
  const double S = sqrt(S2);
  const double xi = S * iD;
  const double eta = fma(tau, iD, 1.0);
  // beta = |v|, ginv = 1/gamma, omg = 1 - 1/gamma (cancellation-free per method)
  double beta, ginv, omg;
  bool conv = true;
  if (S2 == 0.0) {
    beta = 0.0;
    ginv = 1.0;
    omg = 0.0;
  } else if (p.eos == 0 && p.c2p == 0) {
    beta = beta_ideal_closed_form(p.gamma_ad, xi, eta);
    conv = (beta >= 0.0 && beta < 1.0);
    ginv = sqrt(1.0 - beta * beta);
    omg = beta * beta / (1.0 + ginv);
  } else if (p.eos == 0) {
    const double w = w_ideal_newton(p.alpha, xi, eta, p.max_iter, iters, conv);
    const double w2 = w * w;
    const double i1w2 = 1.0 / (1.0 + w2);
    beta = 2.0 * w * i1w2;
    ginv = (1.0 - w2) * i1w2;
    omg = 2.0 * w2 * i1w2;
    conv = conv && (w > 0.0 && w < 1.0);
  } else {
    const double Wl = (p.c2p == 0) ? W_tm_closed_form(xi, eta)
                                   : W_tm_brent(xi, eta, p.max_iter, iters, conv);
    conv = conv && (Wl >= 0.0) && isfinite(Wl);
    const double lor = sqrt(Wl + 1.0);
    ginv = 1.0 / lor;
    beta = sqrt(Wl) * ginv;
    omg = Wl * ginv / (lor + 1.0);
  }
  const double rho = D * ginv;
  const double vs = (S2 == 0.0) ? 0.0 : beta / S;  // v = beta S / |S|
  W.v[0] = vs * U[1];
  W.v[1] = vs * U[2];
  W.v[2] = vs * U[3];
  const double Sv = beta * S;  // S.v
  const double e_m_rho = tau - Sv + D * omg;  // E - S.v - rho
  double P;
  if (p.eos == 0) {
    P = (p.gamma_ad - 1.0) * e_m_rho;
  } else {
    const double Ev = tau + D - Sv;  // E - S.v
    P = e_m_rho * (Ev + rho) / (3.0 * Ev);
  }
  W.rho = rho;
  W.P = P;
  W.lor = 1.0 / ginv;
  return conv ? 0 : 2;
}

// ---------------------------------------------------------------------------------------
// Fluxes (Eq. srhd_flux) and numerical fluxes (Sec. 2.4)
// ---------------------------------------------------------------------------------------

// Physical flux along d from the conserved state, 3-velocity and pressure:
// (D v_d, S v_d + P e_d, (tau + P) v_d).
__device__ __forceinline__ void phys_flux(const double U[5], const double v[3], double P, int d,
                                          double F[5]) {
  const double vd = v[d];
  F[0] = U[0] * vd;
  F[1] = U[1] * vd;
  F[2] = U[2] * vd;
  F[3] = U[3] * vd;
  F[1 + d] += P;
  F[4] = (U[4] + P) * vd;
}

// lambda_pm = (v_d +- sqrt(sig (1 - v_d^2 + sig))) / (1 + sig), sig = cs2/(gamma^2 (1 - cs2)).
__device__ __forceinline__ void wavespeeds(const ConsFlux& c, int d, double& lm, double& lp) {
  const double sig = c.cs2 / (c.lor * c.lor * (1.0 - c.cs2));
  const double vd = c.v[d];
  const double r = sqrt(sig * (1.0 - vd * vd + sig));
  const double i = 1.0 / (1.0 + sig);
  lm = (vd - r) * i;
  lp = (vd + r) * i;
}

// Numerical flux between face states given as (rho, u, P).  HLL: S_L = min(lambda_L, 0),
// S_R = max(lambda_R, 0), (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L) (the
// average when both vanish); LLF: (F_L + F_R)/2 - a (U_R - U_L)/2, a = max |lambda|.
__device__ __forceinline__ void numerical_flux(const Params& p, const double WL[5],
                                               const double WR[5], int d, double Fs[5]) {
  ConsFlux L, R;
  prim_u_to_cons(p, WL, L);
  prim_u_to_cons(p, WR, R);
  double FL[5], FR[5];
  phys_flux(L.U, L.v, L.P, d, FL);
  phys_flux(R.U, R.v, R.P, d, FR);
  double lmL, lpL, lmR, lpR;
  wavespeeds(L, d, lmL, lpL);
  wavespeeds(R, d, lmR, lpR);
  const double lamL = fmin(lmL, lmR), lamR = fmax(lpL, lpR);
  if (p.flux == 1) {
    const double sL = fmin(lamL, 0.0), sR = fmax(lamR, 0.0);
    const double den = sR - sL;
    if (den == 0.0) {
#pragma unroll
      for (int v = 0; v < 5; ++v) Fs[v] = 0.5 * (FL[v] + FR[v]);
    } else {
      const double id = 1.0 / den;
#pragma unroll
      for (int v = 0; v < 5; ++v) Fs[v] = (sR * FL[v] - sL * FR[v] + sL * sR * (R.U[v] - L.U[v])) * id;
    }
  } else {
    const double a = fmax(fabs(lamL), fabs(lamR));
#pragma unroll
    for (int v = 0; v < 5; ++v) Fs[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * a * (R.U[v] - L.U[v]);
  }
}

}  // namespace dgsrhd
