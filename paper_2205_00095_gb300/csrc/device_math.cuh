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

#include "bits.cuh"
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
// Admissible set (Eq. physicality): D > 0 and q = E - sqrt(D^2 + |S|^2) > 0.  With E = tau + D
// and D > 0 this holds exactly when tau > 0 and tau (tau + 2 D) > |S|^2: no root, no division,
// no cancellation of D for cold states.
// ---------------------------------------------------------------------------------------
// Sign and order tests read from the bit pattern (integer pipe instead of FP64 compares).  A
// double that is not NaN is > 0 exactly when its pattern, as a signed 64-bit integer, lies in
// (0, +inf], and two non-negative doubles order as their patterns do.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
constexpr long long kInfBits = 0x7ff0000000000000LL;
__device__ __forceinline__ bool pos_bits(double x) {  // x > 0 (false for NaN)
  const long long b = dbits(x);
  return b > 0 && b <= kInfBits;
}
__device__ __forceinline__ bool finite_bits(double x) { return (dbits(x) & kInfBits) != kInfBits; }
// Order key of a non-NaN double as a signed 64-bit integer (negative patterns mirrored), and the
// min/max chosen by comparing keys on the integer pipe.  -0 orders below +0; with a NaN operand
// either operand may be returned.
__device__ __forceinline__ long long order_key(double x) {
  const long long b = dbits(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double min_bits(double a, double b) {
  return order_key(a) <= order_key(b) ? a : b;
}
__device__ __forceinline__ double max_bits(double a, double b) {
  return order_key(a) >= order_key(b) ? a : b;
}
// |x| by clearing the sign bit
__device__ __forceinline__ double abs_bits(double x) {
  return __longlong_as_double(dbits(x) & 0x7fffffffffffffffLL);
}

// D > 0, tau > 0 and tau (tau + 2D) > S^2 (S2 >= 0 or NaN; a NaN makes it false)
__device__ __forceinline__ bool admissible_parts(double D, double S2, double tau) {
  const long long s2 = dbits(S2);
  return pos_bits(D) && pos_bits(tau) && s2 >= 0 && s2 <= kInfBits &&
         dbits(tau * (tau + 2.0 * D)) > s2;
}

// The same decision as admissible_parts, screened in FP32 first.  With D, tau and S2 truncated
// to FP32 (relative error below 2^-23) and three FP32 operations, tau (tau + 2D) comes out within
// a relative 2^-21 of its exact value and S2 within 2^-23 of the FP64 one, so
// tau (tau + 2D) > S2 (1 + 2^-14) in FP32, with D, tau > 0 and tau (tau + 2D) inside
// [2^-100, 1e38] (clear of FP32 underflow and overflow), implies the FP64 test by a wide margin.
// Every other state, including NaN and infinite ones, takes the FP64 test.
__device__ __forceinline__ bool admissible_parts_screen(double D, double S2, double tau) {
  const float Df = f64_to_f32_bits(D), tf = f64_to_f32_bits(tau), sf = f64_to_f32_bits(S2);
  const float lhs = tf * (tf + 2.0f * Df);
  if (Df > 0.0f && tf > 0.0f && lhs >= 0x1p-100f && lhs <= 1e38f && lhs > sf * (1.0f + 0x1p-14f))
    return true;
  return admissible_parts(D, S2, tau);
}

__device__ __forceinline__ bool admissible(const double U[5]) {
  return admissible_parts(U[0], U[1] * U[1] + U[2] * U[2] + U[3] * U[3], U[4]);
}

// The same decision as admissible(U), screened in FP32 first: with every input truncated to FP32
// (relative error below 2^-23) and five FP32 operations, tau (tau + 2D) and |S|^2 come out within
// a relative 2^-20 of their exact values, so tau (tau + 2D) > |S|^2 (1 + 2^-14) in FP32, with
// D, tau > 0 and tau (tau + 2D) inside [2^-100, 1e38] (clear of FP32 underflow and overflow),
// implies the exact inequality by a wide margin and hence the FP64 test.  Every other state,
// including NaN and infinite ones, takes the FP64 test, so the result never differs from it.
__device__ __forceinline__ bool admissible_screen(const double U[5]) {
  const float D = f64_to_f32_bits(U[0]), tau = f64_to_f32_bits(U[4]);
  const float s1 = f64_to_f32_bits(U[1]), s2 = f64_to_f32_bits(U[2]), s3 = f64_to_f32_bits(U[3]);
  const float lhs = tau * (tau + 2.0f * D);
  const float S2 = fmaf(s1, s1, fmaf(s2, s2, s3 * s3));
  if (D > 0.0f && tau > 0.0f && lhs >= 0x1p-100f && lhs <= 1e38f && lhs > S2 * (1.0f + 0x1p-14f))
    return true;
  return admissible(U);
}

// ---------------------------------------------------------------------------------------
// Conserved -> primitive (Sec. 3).  xi = |S|/D, eta = E/D.
// ---------------------------------------------------------------------------------------

// Ideal EOS, closed form (Sec. 3.1): the monic quartic beta^4 + a3 beta^3 + a2 beta^2 + a1 beta
// + a0 in beta = |v|, its resolvent cubic (i1, i2, i3), Cardano's root x of the resolvent
// (trigonometric form when T < 0), and the quadratic factors beta^2 + B beta + C.  The section's
// coefficients, in xi = |S|/D and eta = E/D over (G - 1)^2 (1 + xi^2), are multiplied through by
// D^2 so that they come from (D^2, |S|, E) and the one reciprocal w = 1/((G - 1)^2 (D^2 + |S|^2)):
//   a0 = |S|^2 w,  a1 = -2 G |S| E w,  a3 = (G - 1) a1,
//   a2 = (G^2 E^2 + 2 (G - 1) |S|^2 - (G - 1)^2 D^2) w.
// g1 = (G - 1)^2 D^2 is passed in (the caller forms w's denominator from it), and a3^2 is taken
// as (G - 1)^2 a1^2.
// B and C are carried doubled (B' = 2B, C' = 2C), which moves the factors 1/2 into the final
// 1/4: beta = (sqrt(B'^2 - 8 C') - B') / 4 (scalings by powers of two are exact).
__device__ __forceinline__ double beta_ideal_closed_form(const Params& p, double g1, double S2,
                                                         double S, double E, double w) {
  const double a0 = S2 * w;
  const double SEw = (S * E) * w;
  const double a1 = p.m2G * SEw;
  const double a3 = p.m2Ggm1 * SEw;
  const double a2 = fma(p.G2, E * E, fma(p.tgm1, S2, -g1)) * w;
  // resolvent cubic x^3 + i1 x^2 + i2 x + i3 with i1 = -a2, i2 = a1 a3 - 4 a0,
  // i3 = 4 a2 a0 - a1^2 - a3^2 a0; with t = i1/3 its depressed form has
  // R = (9 i1 i2 - 27 i3 - 2 i1^3)/54 = (t i2 - i3)/2 - t^3 and S = (3 i2 - i1^2)/9 = i2/3 - t^2
  // multiplications by powers of two are exponent additions on the integer pipe (ldexp_bits)
  const double m4a0 = -ldexp_bits<2>(a0);
  const double i2 = fma(a3, a1, m4a0);
  const double A1 = a1 * a1;
  const double i3 = fma(a0, fma(-p.gm1sq, A1, ldexp_bits<2>(a2)), -A1);
  const double t = a2 * (-1.0 / 3.0);  // i1 / 3
  const double t2 = t * t;
  const double R = fma(0.5, fma(t, i2, -i3), -t2 * t);
  const double Sq = fma(i2, 1.0 / 3.0, -t2);
  const double T = fma(R, R, Sq * Sq * Sq);
  double x;
  if (dbits(T) < 0 && dbits(T) != (long long)0x8000000000000000ULL) {  // T < 0
    x = 2.0 * pow(R * R - T, 1.0 / 6.0) * cos(atan2(sqrt(-T), R) * (1.0 / 3.0)) - t;
  } else {
    // Cardano's pair cbrt(R + sqrt(T)) + cbrt(R - sqrt(T)): their product is -Sq, so with
    // y = R + sign(R) sqrt(T) (no cancellation) the pair is y^(1/3) - Sq y^(-1/3), both from
    // one reciprocal cube root r = y^(-1/3): y^(1/3) = y r^2.
    const double y = R + copysign(sqrt_nr(T), R);
    if ((dbits(y) << 1) == 0) {  // y = +-0
      x = -t;
    } else {
      const double r = rcbrt_nr(y);
      x = fma(y * r, r, -Sq * r) - t;
    }
  }
  // The three radicands are non-negative for an admissible state; as xi -> 0 they shrink to
  // rounding level and can round below zero, so a negative one is taken as zero.
  auto root0 = [](double r) { return sqrt_nr(dbits(r) < 0 ? 0.0 : r); };
  const double Bp = a3 + root0(fma(a3, a3, ldexp_bits<2>(x - a2)));
  const double Cp = x - root0(fma(x, x, m4a0));
  return ldexp_bits<-2>(root0(fma(Bp, Bp, -ldexp_bits<3>(Cp))) - Bp);
}

// Ideal EOS, Newton-Raphson on the Riccardi quartic in w, beta = 2w/(1 + w^2)
// (Eqs. iterative_quartic_unknown, iterative_quartic), started from the small-xi series of
// Eq. iterative_cubic_approximation; stop at |dw| <= 1e-14 w; for xi < 1e-4 the series.
// The iterations run first in FP32 (FP32 issues 58x faster than FP64 on this GPU) until the
// step is below 1e-6 w or stops shrinking (at most 12), then continue in FP64 from that
// iterate to the FP64 stop rule; `iters` counts both phases and max_iter caps their sum.
__device__ __forceinline__ double w_ideal_newton(double al, double xi, double eta, int max_iter,
                                                 double rtol, int& iters, bool& conv) {
  const double k1 = al * eta - 1.0;
  const double ik1 = recip_nr(k1);
  const double ik1sq = ik1 * ik1;
  const double series = (al - 1.0) * 0.5 * ik1 * xi +
                        (al - 1.0) * (al - 1.0) * 0.125 * ik1sq * ik1sq *
                            ((al + 3.0) * (al * eta + 1.0) - 4.0 * (al + 1.0)) * xi * xi * xi;
  iters = 0;
  conv = true;
  if (xi < 1e-4) return series;
  const double c4 = (al - 1.0) * xi, c3 = -2.0 * (al * eta + 1.0), c2 = 2.0 * (al + 1.0) * xi,
               c1 = -2.0 * k1, c0 = c4;
  // FP32 phase
  // conversions on the bit patterns (a cast would issue on the FP64 pipe)
  const float f4 = f64_to_f32_bits(c4), f3 = f64_to_f32_bits(c3), f2 = f64_to_f32_bits(c2),
              f1 = f64_to_f32_bits(c1), f0 = f64_to_f32_bits(c0);
  float wf = fminf(fmaxf(f64_to_f32_bits(series), 1e-30f), 1.0f - 6e-8f);
  int it = 0;
  // At most 12 FP32 iterations (the FP64 phase keeps the rest, at least two).  Near |v| = 1
  // the quartic is close to palindromic (c0 = c4, c1 ~ c3) and its root w < 1 has a partner
  // 1/w close by; there FP32 rounding can keep the step above 1e-6 w for good, so the phase
  // also ends once a step fails to shrink.
  const int max32 = min(max_iter - 2, 12);
  float dprev = 3.0e38f;
  while (it < max32) {
    const float Pw = fmaf(fmaf(fmaf(fmaf(f4, wf, f3), wf, f2), wf, f1), wf, f0);
    const float dP = fmaf(fmaf(fmaf(4.0f * f4, wf, 3.0f * f3), wf, 2.0f * f2), wf, f1);
    const float dw = Pw / dP;
    const float adw = fabsf(dw);
    wf -= dw;
    ++it;
    if (!(adw > 1e-6f * wf)) break;  // also leaves on NaN
    if (it > 2 && !(adw < dprev)) break;
    dprev = adw;
  }
  double w = (wf > 0.0f && wf < 1.0f) ? f32_to_f64_bits(wf) : fmin(fmax(series, 1e-300), 1.0 - 1e-15);
  // FP64 phase; besides |dw| <= 1e-14 w it stops once the residual before the step is at the
  // rounding level of the quartic on (0, 1), |P(w)| <= 8 eps sum |c_k| (for xi ~ 1e3 that level
  // keeps the step near 1e-14 w)
  const double pres = 8.0 * 2.220446049250313e-16 *
                      (fabs(c4) + fabs(c3) + fabs(c2) + fabs(c1) + fabs(c0));
  conv = false;
  while (it < max_iter) {
    const double Pw = fma(fma(fma(fma(c4, w, c3), w, c2), w, c1), w, c0);
    const double dP = fma(fma(fma(4.0 * c4, w, 3.0 * c3), w, 2.0 * c2), w, c1);
    const double dw = Pw * recip_nr(dP);
    w -= dw;
    ++it;
    if (fabs(dw) <= fmax(1e-14, rtol) * w || fabs(Pw) <= pres) {
      conv = true;
      break;
    }
  }
  iters = it;
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
  const double idm2 = recip_nr(dm * dm);
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
    // (d < 0 implies Q < 0) sqrt(-Q^3) and sqrt(-Q) from one reciprocal square root of -Q
    const double rq = rsqrt_nr(-Q);
    const double iota = acos(R * rq * rq * rq);
    W = 2.0 * (-Q) * rq * cos(iota * (1.0 / 3.0)) - c.c1 * (1.0 / 3.0);
  } else {
    // Cardano's pair cbrt(R + sqrt(d)) + cbrt(R - sqrt(d)): the product of the two is -Q, so
    // with y = R + sign(R) sqrt(d) (no cancellation) the pair is y^(1/3) - Q y^(-1/3), from one
    // reciprocal cube root
    const double y = R + copysign(sqrt_nr(d), R);
    if (y == 0.0) {
      W = -c.c1 * (1.0 / 3.0);
    } else {
      const double r = rcbrt_nr(y);
      W = fma(y * r, r, -Q * r) - c.c1 * (1.0 / 3.0);
    }
  }
  return fmax(W, 0.0);
}

// Brent's zero finder (Brent 1973) on the cubic over the bracket [a, b] with f(a) f(b) <= 0,
// tolerance 2 eps |b| + tiny, at most max_iter iterations; T is float or double.
template <typename T>
__device__ __forceinline__ T brent_cubic(T c1, T c2, T c3, T a, T b, T fa, T fb, int max_iter,
                                         T eps, T tiny, int& iters, bool& conv) {
  auto f = [&](T W) { return ((W + c1) * W + c2) * W + c3; };
  T c = a, fc = fa, d = b - a, e = d;
  conv = false;
  for (int it = 1; it <= max_iter; ++it) {
    iters = it;
    if (fb * fc > T(0)) {
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
    const T tol = T(2) * eps * fabs(b) + tiny;
    const T m = T(0.5) * (c - b);
    if (fabs(m) <= tol || fb == T(0)) {
      conv = true;
      return b;
    }
    if (fabs(e) >= tol && fabs(fa) > fabs(fb)) {
      const T s = fb / fa;
      T pp, qq;
      if (a == c) {
        pp = T(2) * m * s;
        qq = T(1) - s;
      } else {
        const T q1 = fa / fc, r1 = fb / fc;
        pp = s * (T(2) * m * q1 * (q1 - r1) - (b - a) * (r1 - T(1)));
        qq = (q1 - T(1)) * (r1 - T(1)) * (s - T(1));
      }
      if (pp > T(0))
        qq = -qq;
      else
        pp = -pp;
      if (T(2) * pp < fmin(T(3) * m * qq - fabs(tol * qq), fabs(e * qq))) {
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
    b += (fabs(d) > tol) ? d : (m > T(0) ? tol : -tol);
    fb = f(b);
  }
  return b;
}

// Taub-Matthews iterative (Sec. 3.2): Brent on the cubic, bracketed by gamma in [1, 200]
// with the upper end multiplied by 4 (at most 10 times) until the sign changes.  Brent runs in
// FP32 (FP32 issues 58x faster than FP64 on this GPU); the FP32 root W32 is then polished in
// FP64 by Newton's method on the cubic, safeguarded inside the bracket W32 (1 -+ 1e-5): a step
// that leaves the bracket is replaced by bisection, and the bracket shrinks with the sign of
// the cubic.  The bracket holds the unique non-negative root, so the polish cannot stray to
// another root (the reason Sec. 3.2 gives for a bracketed solver).  When the cubic does not
// change sign across that bracket, FP64 Brent runs on the paper's bracket instead.  The polish
// stops once the step, or the error left after it (Newton's quadratic error term), is within
// 2 eps |W| + 1e-300 (Brent's tolerance); `iters` counts all iterations and max_iter caps
// their sum.
static __device__ __noinline__ double W_tm_brent(double xi, double eta, int max_iter, double rtol,
                                                 int& iters, bool& conv) {
  const Cubic cc = tm_cubic(xi, eta);
  iters = 0;
  conv = false;
  const double f0 = cc.c3;  // the cubic at W = 0
  if (f0 == 0.0) {
    conv = true;
    return 0.0;
  }
  // FP32 phase.  Its bracket: |v| < |S|/E, so W = u^2 < xi^2 / ((eta - xi)(eta + xi)) for an
  // admissible state; eta - xi is formed in FP64 (it cancels at large Lorentz factors) and the
  // bound is widened by 1e-3 relative and capped at the paper's 200^2 - 1.  Any state whose
  // bound fails the sign check takes FP64 Brent on the paper's bracket below.
  // conversions on the bit patterns (a cast would issue on the FP64 pipe)
  const float g1 = f64_to_f32_bits(cc.c1), g2 = f64_to_f32_bits(cc.c2), g3 = f64_to_f32_bits(cc.c3);
  auto ff = [&](float W) { return ((W + g1) * W + g2) * W + g3; };
  int it32 = 0;
  bool conv32 = false;
  float W32 = 0.0f;
  const float x = f64_to_f32_bits(xi), exm = f64_to_f32_bits(eta - xi);
  if (exm > 0.0f && g3 < 0.0f) {
    const float hi32 = fminf(x * x / (exm * (f64_to_f32_bits(eta) + x)) * 1.001f + 1e-30f, 39999.0f);
    const float fh32 = ff(hi32);
    if (fh32 > 0.0f) {
      // the FP32 phase takes at most half the iterations: the FP64 polish or the FP64 Brent
      // fallback keeps the rest
      const int max32 = max_iter > 3 ? max_iter / 2 : 1;
      W32 = brent_cubic<float>(g1, g2, g3, 0.0f, hi32, g3, fh32, max32, 1.1920929e-07f, 1e-37f,
                               it32, conv32);
    }
  }
  // FP64 phase: safeguarded Newton inside a tight bracket around the FP32 root
  if (conv32 && W32 > 0.0f) {
    const double W32d = f32_to_f64_bits(W32);
    double a = W32d * (1.0 - 1e-5), b = W32d * (1.0 + 1e-5);
    const double fa = cubic_at(cc, a), fb = cubic_at(cc, b);
    if (fa * fb <= 0.0) {
      const bool rising = fa < 0.0;  // the cubic runs from fa to fb across [a, b]
      const double tol = fmax(2.0 * 2.220446049250313e-16, rtol);
      const double c1x2 = 2.0 * cc.c1;
      double W = W32d;
      int it = it32;
      // The first step from the FP32 root is of the FP32 rounding size, far above the FP64
      // tolerance, so the stop test starts with the second (with the first for a caller's
      // relative tolerance, which that step may already meet).
      bool test = rtol > 0.0;
      while (it < max_iter) {
        ++it;
        const double f = cubic_at(cc, W);
        if (f == 0.0) {
          conv = true;
          break;
        }
        if ((f < 0.0) == rising)
          a = W;
        else
          b = W;
        const double r = recip_nr(fma(fma(3.0, W, c1x2), W, cc.c2));  // 1 / f'(W)
        const double dW = f * r;
        const double Wn = W - dW;
        if (test) {
          // Stop once the step, or the error it leaves, is within the tolerance; the latter
          // spares the last iteration, whose own step would be at rounding level.  For the
          // monic cubic a Newton step from W* + e leaves (f''(W*) e^2 / 2 + 2 e^3) / f'(W),
          // bounded here with e ~ dW, |f''(W*)| <= |f''(W)| + 6|e| and a factor 4 to spare.
          // Both sides are non-negative, so the comparison runs on the bit patterns (integer
          // pipe); the step is taken before the bracket test: once W sits on the root,
          // rounding noise in f can move a bracket end onto W itself.
          const double adW = fabs(dW);
          const double est = fabs(r) * (adW * adW) * fma(2.0, fabs(fma(6.0, W, c1x2)), 20.0 * adW);
          const long long thr = dbits(fma(tol, fabs(W), 1e-300));
          if (min(dbits(adW), dbits(est)) <= thr) {
            W = Wn;
            conv = true;
            break;
          }
        }
        test = true;
        W = (Wn > a && Wn < b) ? Wn : 0.5 * (a + b);
      }
      iters = it;
      return W;
    }
  }
  // FP64 Brent on the paper's bracket [0, 200^2 - 1], upper end x4 until the sign changes
  double hi = 200.0 * 200.0 - 1.0, fhi = cubic_at(cc, hi);
  for (int k = 0; k < 10 && f0 * fhi > 0.0; ++k) {
    hi *= 4.0;
    fhi = cubic_at(cc, hi);
  }
  iters = it32;
  if (f0 * fhi > 0.0) return __longlong_as_double(0x7ff8000000000000LL);
  int it64 = 0;
  // tolerance 2 eps |b| + 1e-300, or rtol |b| for a caller's larger relative tolerance
  const double W = brent_cubic<double>(cc.c1, cc.c2, cc.c3, 0.0, hi, f0, fhi, max_iter - it32,
                                       fmax(2.220446049250313e-16, 0.5 * rtol), 1e-300, it64, conv);
  iters = it32 + it64;
  return W;
}

// Result of one recovery.
struct Prim {
  double rho, v[3], P;
  double lor;   // Lorentz factor
  double ginv;  // 1 / Lorentz factor
};

// status: 0 ok, 1 invalid input, 2 not converged / closed form failed.
__device__ __forceinline__ int con2prim(const Params& p, const double U[5], Prim& W, int& iters) {
  const double D = U[0], tau = U[4];
  const double S2 = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
  iters = 0;
  const double nanv = __longlong_as_double(0x7ff8000000000000LL);
  if (!admissible_parts_screen(D, S2, tau) || !finite_bits(S2) || !finite_bits(tau)) {
    W.rho = W.v[0] = W.v[1] = W.v[2] = W.P = W.lor = nanv;
    return 1;
  }
  const bool moving = dbits(S2) != 0;  // S2 > 0 (S2 is finite and >= 0 here)
  const double rS = moving ? rsqrt_nr(S2) : 0.0;  // 1/|S|
  const double S = S2 * rS;
  const bool closed_ideal = p.eos == 0 && p.c2p == 0;
  // beta = |v|, ginv = 1/gamma, omg = 1 - 1/gamma (cancellation-free per method)
  double beta, ginv, lor, omg = 0.0, Wl = 0.0;
  bool conv = true;
  if (!moving) {
    beta = 0.0;
    ginv = 1.0;
    lor = 1.0;
  } else if (closed_ideal) {
    const double g1 = p.gm1sq * (D * D);  // (G - 1)^2 D^2
    beta = beta_ideal_closed_form(p, g1, S2, S, tau + D, recip_nr(fma(p.gm1sq, S2, g1)));
    conv = dbits(beta) >= 0 && dbits(beta) < dbits(1.0);  // 0 <= beta < 1
    // gamma = (1 - beta^2)^(-1/2); 1 - 1/gamma = beta^2 gamma / (gamma + 1)
    const double b2 = beta * beta;
    const double om = 1.0 - b2;
    lor = rsqrt_nr(om);
    ginv = om * lor;
    omg = b2 * recip_nr(1.0 + ginv);  // = b2 gamma / (gamma + 1)
  } else {
    const double iD = recip_nr(D);
    const double xi = S * iD;
    const double eta = fma(tau, iD, 1.0);
    if (p.eos == 0) {
      const double w = w_ideal_newton(p.alpha, xi, eta, p.max_iter, p.c2p_rtol, iters, conv);
      const double w2 = w * w;
      // beta = 2w/(1 + w^2), 1/gamma = (1 - w^2)/(1 + w^2), gamma from the same division
      const double ap = 1.0 + w2, am = 1.0 - w2;
      const double t = recip_nr(ap * am);
      const double i1w2 = t * am;
      beta = 2.0 * w * i1w2;
      ginv = am * i1w2;
      omg = 2.0 * w2 * i1w2;
      lor = t * ap * ap;
      conv = conv && dbits(w) > 0 && dbits(w) < dbits(1.0);  // 0 < w < 1
    } else {
      Wl = (p.c2p == 0) ? W_tm_closed_form(xi, eta)
                        : W_tm_brent(xi, eta, p.max_iter, p.c2p_rtol, iters, conv);
      conv = conv && dbits(Wl) >= 0 && finite_bits(Wl);  // Wl >= 0 and finite
      const double q = Wl + 1.0;  // gamma^2
      ginv = rsqrt_nr(q);
      lor = q * ginv;
      beta = sqrt_nr(Wl) * ginv;
    }
  }
  const double rho = D * ginv;
  const double vs = beta * rS;  // v = beta S / |S|
  W.v[0] = vs * U[1];
  W.v[1] = vs * U[2];
  W.v[2] = vs * U[3];
  const double Sv = beta * S;  // S.v
  double P;
  if (p.eos == 0) {
    const double e_m_rho = tau - Sv + D * omg;  // E - S.v - rho
    P = p.gm1 * e_m_rho;
  } else {
    // 1 - 1/gamma = W/(gamma (gamma + 1)) and P = (E - S.v - rho)(E - S.v + rho)/(3(E - S.v)):
    // 1/(gamma + 1) and 1/(3(E - S.v)) from one division
    const double Ev = tau + D - Sv;  // E - S.v
    const double L1 = lor + 1.0, E3 = 3.0 * Ev;
    const double t = recip_nr(L1 * E3);
    omg = Wl * ginv * E3 * t;
    const double e_m_rho = tau - Sv + D * omg;
    P = e_m_rho * (Ev + rho) * L1 * t;
  }
  W.rho = rho;
  W.P = P;
  W.lor = lor;
  W.ginv = ginv;
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

// Face state from the interpolated primitive (rho, u, P): conserved state, 3-velocity, and the
// sound-speed ratio sig = cs^2 / (gamma^2 (1 - cs^2)) of Sec. 2.4 kept as the fraction A / B,
// with both scaled by rho so that the ideal EOS needs no division:
//   ideal: A = Gamma P,          B = gamma^2 (rho + alpha P - Gamma P)
//   TM:    A = P (3 P + 5 s),    B = gamma^2 (12 P^2 + 2 rho^2 + 12 P s - A),  s = sqrt(P^2 + 4 rho^2 / 9)
// (cs^2 = Gamma Theta / h, resp. the Taub-Matthews ratio, multiplied through by rho or rho^2).
struct FaceState {
  double U[5];
  double v[3];
  double P, A, B;
  // intermediates, kept for the reverse sweep
  double u2, q, ilor, lor, rho_hm1, sg, isg, Z, iZ, K, id1, i;
};

// Face state from (rho, u, P).  The three reciprocals 1/Z, 1/(gamma + 1) and 1/(A + B) come
// from one division of their product, and the roots from the reciprocal square root rsqrt_nr
// (the root itself is x rsqrt_nr(x)).
// With `rec` given, the roots and reciprocals are read from it instead (values saved by an
// earlier evaluation on the same state), and no root or division is evaluated.
__device__ __forceinline__ void face_state_core(const Params& p, const double Wu[5], FaceState& c,
                                                const double* rec) {
  // Sums that take a product are written with __dadd_rn / __dsub_rn, which the compiler never
  // fuses into an FMA: the roots and reciprocals must come out bit-identical in every kernel
  // that evaluates them, whether they are saved by one and read by another or recomputed.
  const double rho = Wu[0], P = Wu[4];
  c.u2 = fma(Wu[1], Wu[1], fma(Wu[2], Wu[2], Wu[3] * Wu[3]));
  c.q = __dadd_rn(1.0, c.u2);  // gamma^2
  c.ilor = rec ? rec[0] : rsqrt_nr(c.q);
  c.lor = c.q * c.ilor;
  c.P = P;
  if (p.eos == 0) {
    c.A = p.gamma_ad * P;
    c.K = fma(p.amG, P, rho);  // rho + (alpha - Gamma) P
    c.sg = c.isg = c.Z = c.iZ = 0.0;
  } else {
    const double rho2 = rho * rho;
    const double x2 = fma(P, P, (4.0 / 9.0) * rho2);
    c.isg = rec ? rec[1] : rsqrt_nr(x2);
    c.sg = x2 * c.isg;
    c.Z = fma(2.0 / 3.0, rho, c.sg);
    c.A = P * fma(3.0, P, 5.0 * c.sg);
    // 12 P (P + s) + 2 rho^2 - A = 9 P^2 + 7 P s + 2 rho^2: positive terms only
    c.K = fma(P, fma(9.0, P, 7.0 * c.sg), ldexp_bits<1>(rho2));
  }
  c.B = c.q * c.K;
  const double L1 = __dadd_rn(c.lor, 1.0), AB = __dadd_rn(c.A, c.B);
  if (rec) {
    c.iZ = rec[2];
    c.id1 = rec[3];
    c.i = rec[4];
  } else if (p.eos == 0) {
    const double t = recip_nr(L1 * AB);
    c.id1 = t * AB;
    c.i = t * L1;
  } else {
    const double ZL = c.Z * L1;
    const double t = recip_nr(ZL * AB);
    const double tAB = t * AB;
    c.iZ = tAB * L1;
    c.id1 = tAB * c.Z;
    c.i = t * ZL;
  }
  c.rho_hm1 = p.eos == 0 ? p.alpha * P : P * fma(1.5 * P, c.iZ, 2.5);
  const double D = c.lor * rho;
  const double rhoh_lor = __dadd_rn(rho, c.rho_hm1) * c.lor;  // S = rho h gamma u
  c.U[0] = D;
  c.U[1] = rhoh_lor * Wu[1];
  c.U[2] = rhoh_lor * Wu[2];
  c.U[3] = rhoh_lor * Wu[3];
  c.U[4] = fma(D * c.u2, c.id1, fma(c.q, c.rho_hm1, -P));
  c.v[0] = Wu[1] * c.ilor;
  c.v[1] = Wu[2] * c.ilor;
  c.v[2] = Wu[3] * c.ilor;
}

__device__ __forceinline__ void face_state(const Params& p, const double Wu[5], FaceState& c) {
  face_state_core(p, Wu, c, nullptr);
}

// lambda_pm = (v_d +- sqrt(sig (1 - v_d^2 + sig))) / (1 + sig) with sig = A / B, evaluated as
// (v_d B +- r) i with r = sqrt(X), X = A (B (1 - v_d^2) + A), and i = 1/(A + B) from the face
// state.  Also returns X, r and 1/r (0 where r = 0); 1/r is read from `ir_saved` when given.
template <int D>
__device__ __forceinline__ void wave_root(const FaceState& c, double& X, double& r, double& ir,
                                          const double* ir_saved) {
  const double vd = c.v[D];
  X = c.A * fma(c.B, fma(-vd, vd, 1.0), c.A);
  ir = ir_saved ? *ir_saved : (pos_bits(X) ? rsqrt_nr(X) : 0.0);
  r = X * ir;
}

template <int D>
__device__ __forceinline__ void wavespeeds_full(const FaceState& c, double& lm, double& lp,
                                                double& X, double& r, double& ir,
                                                const double* ir_saved) {
  wave_root<D>(c, X, r, ir, ir_saved);
  const double vd = c.v[D];
  lm = fma(vd, c.B, -r) * c.i;
  lp = fma(vd, c.B, r) * c.i;
}

template <int D>
__device__ __forceinline__ void phys_flux_dir(const double U[5], const double v[3], double P,
                                              double F[5]) {
  const double vd = v[D];
  F[0] = U[0] * vd;
  F[1] = U[1] * vd;
  F[2] = U[2] * vd;
  F[3] = U[3] * vd;
  F[1 + D] = fma(U[1 + D], vd, P);  // one rounding, the same in every kernel
  F[4] = (U[4] + P) * vd;
}

// The kFaceTape values of one face state, in the order documented with kFaceTape.
__device__ __forceinline__ void face_tape(const FaceState& c, const double F[5], double r,
                                          double ir, double lm, double lp, double t[kFaceTape]) {
  t[0] = c.ilor, t[1] = c.isg, t[2] = c.iZ, t[3] = c.id1, t[4] = c.i, t[5] = ir;
  t[6] = c.u2, t[7] = c.lor, t[8] = c.sg, t[9] = c.A, t[10] = c.B, t[11] = c.K;
  t[12] = c.rho_hm1;
#pragma unroll
  for (int k = 0; k < 5; ++k) t[13 + k] = c.U[k];
  t[18] = r, t[19] = lm, t[20] = lp;
#pragma unroll
  for (int k = 0; k < 5; ++k) t[21 + k] = F[k];
}

// HLLC along axis D (the paper names the solver but prints no formula; this is the relativistic
// HLLC construction of the literature it cites, in the variables (D, S, tau)).  With the outer
// speeds lamL < 0 < lamR and the HLL averages U_hll = (lamR U_R - lamL U_L - F_R + F_L)/(lamR -
// lamL), F_hll = (lamR F_L - lamL F_R + lamR lamL (U_R - U_L))/(lamR - lamL): with E = tau + D,
// F_E = F_tau + F_D and m = S_D, the contact speed is the root of F_E x^2 - (E + F_m) x + m = 0
// that equals v_D for equal states, x = 2m/(b + sqrt(b^2 - 4 F_E m)), b = E + F_m, and the
// contact pressure p* = F_m - x F_E.  On the side K the contact faces (left when x >= 0), with
// v = v_D, P and lam of that side: D* = D (lam - v)/(lam - x), S*_D = (S_D (lam - v) + p* - P)/
// (lam - x), S*_t = S_t (lam - v)/(lam - x), tau* = (tau (lam - v) + p* x - P v)/(lam - x), and
// F* = F_K + lam (U* - U_K).  lamL >= 0 gives F_L, lamR <= 0 gives F_R.
template <int D>
__device__ __forceinline__ void hllc_flux(const FaceState& L, const FaceState& R,
                                          const double FL[5], const double FR[5], double lamL,
                                          double lamR, double Fs[5]) {
  if (lamL >= 0.0 || lamR <= 0.0) {
    const bool useL = lamL >= 0.0;
#pragma unroll
    for (int v = 0; v < 5; ++v) Fs[v] = useL ? FL[v] : FR[v];
    return;
  }
  const double idl = recip_nr(lamR - lamL), lrl = lamR * lamL;
  auto Uh = [&](int v) { return (lamR * R.U[v] - lamL * L.U[v] - FR[v] + FL[v]) * idl; };
  auto Fh = [&](int v) { return (lamR * FL[v] - lamL * FR[v] + lrl * (R.U[v] - L.U[v])) * idl; };
  const double Eh = Uh(4) + Uh(0), FEh = Fh(4) + Fh(0), mh = Uh(1 + D), Fmh = Fh(1 + D);
  const double b = Eh + Fmh;
  const double xs = 2.0 * mh * recip_nr(b + sqrt(fma(b, b, -4.0 * FEh * mh)));
  const double ps = fma(-xs, FEh, Fmh);
  const bool left = xs >= 0.0;
  const double lam = left ? lamL : lamR, v = left ? L.v[D] : R.v[D], P = left ? L.P : R.P;
  const double lv = lam - v, di = recip_nr(lam - xs);
  double UK[5], FK[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    UK[k] = left ? L.U[k] : R.U[k];
    FK[k] = left ? FL[k] : FR[k];
  }
  double Us[5];
  Us[0] = UK[0] * lv * di;
#pragma unroll
  for (int k = 0; k < 3; ++k) Us[1 + k] = (k == D) ? (UK[1 + D] * lv + ps - P) * di : UK[1 + k] * lv * di;
  Us[4] = (UK[4] * lv + ps * xs - P * v) * di;
#pragma unroll
  for (int k = 0; k < 5; ++k) Fs[k] = fma(lam, Us[k] - UK[k], FK[k]);
}

// wL F_L + wR F_R + c (U_R - U_L) along D from the two face states.  With the normal fluxes
// F = (U v_d; S_D v_d + P; (tau + P) v_d) every conserved component regroups per side as
// U_L (wL v_L - c) + U_R (wR v_R + c), plus the pressure terms wL P_L + wR P_R (momentum along
// D) and wL P_L v_L + wR P_R v_R (energy): two fused multiply-adds per component, with the
// side weights bL = wL v_L - c and bR = wR v_R + c formed once.
template <int D>
__device__ __forceinline__ void flux_mix(const FaceState& L, const FaceState& R, double wL,
                                         double wR, double c, double out[5]) {
  const double aL = wL * L.v[D], aR = wR * R.v[D];
  const double bL = aL - c, bR = aR + c;
  const double pp = fma(wL, L.P, wR * R.P);
  const double pv = fma(aL, L.P, aR * R.P);
#pragma unroll
  for (int k = 0; k < 4; ++k)
    out[k] = fma(L.U[k], bL, (k == 1 + D) ? fma(R.U[k], bR, pp) : R.U[k] * bR);
  out[4] = fma(L.U[4], bL, fma(R.U[4], bR, pv));
}

// The same combination as FP32 head-and-tail pairs (the split-precision update consumes the face
// flux in that form): the side weights and the pressure terms in FP64 (five FP64 operations for
// LLF), the products and sums in pair arithmetic, within about 2^-46 of the FP64 combination
// relative to the magnitudes of its terms.
template <int D>
__device__ __forceinline__ void flux_mix(const FaceState& L, const FaceState& R, double wL,
                                         double wR, double c, F32Pair out[5]) {
  const double aL = wL * L.v[D], aR = wR * R.v[D];
  const F32Pair bL = f32_pair(aL - c), bR = f32_pair(aR + c);
  const F32Pair pp = f32_pair(fma(wL, L.P, wR * R.P));
  const F32Pair pv = f32_pair(fma(aL, L.P, aR * R.P));
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const F32Pair x = add_pair(mul_pair(f32_pair(L.U[k]), bL), mul_pair(f32_pair(R.U[k]), bR));
    out[k] = (k == 1 + D) ? add_pair(x, pp) : (k == 4 ? add_pair(x, pv) : x);
  }
}

// 2 F* stored into a flux output of either form
__device__ __forceinline__ void put_flux(double& o, double x) { o = x; }
__device__ __forceinline__ void put_flux(F32Pair& o, double x) { o = f32_pair(x); }

// Numerical flux along axis D between face states given as (rho, u, P), returned DOUBLED (2 F*:
// the factor 1/2 of LLF and of the HLL denominator moves into the lift coefficients, which
// are exact powers-of-two scalings of the tables).  HLL: S_L = min(lambda_L, 0), S_R =
// max(lambda_R, 0), F* = (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L) (the average when
// both vanish); LLF: F* = (F_L + F_R)/2 - a (U_R - U_L)/2 with a = max |lambda|; HLLC as above.
// TAPE: also fill recL / recR with the face-state tape (the forward pass of the reverse sweep).
// Both variants give the same bits.
// O: double, or F32Pair for the split-precision update (LLF and HLL then combine in pair
// arithmetic; HLLC forms its flux in FP64 and splits it).
template <int D, bool TAPE, class O = double>
__device__ __forceinline__ void numerical_flux(const Params& p, const double WL[5],
                                               const double WR[5], O Fs2[5],
                                               double recL[kFaceTape], double recR[kFaceTape]) {
  FaceState L, R;
  face_state(p, WL, L);
  face_state(p, WR, R);
  if (!TAPE && p.flux == 0) {
    // LLF needs a = max |lambda| only.  Per side, with r >= 0 and (A + B) > 0, the larger of
    // |v_d B - r| and |v_d B + r| is |v_d| B + r, and rounding is monotone and symmetric, so
    // (|v_d| B + r) i is bit for bit the larger of |lambda_-| and |lambda_+|; the largest
    // |lambda| over both sides is that of max(lambda_+) or min(lambda_-), as below.
    double XL, rL, irL, XR, rR, irR;
    wave_root<D>(L, XL, rL, irL, nullptr);
    wave_root<D>(R, XR, rR, irR, nullptr);
    const double a = max_bits(fma(abs_bits(L.v[D]), L.B, rL) * L.i, fma(abs_bits(R.v[D]), R.B, rR) * R.i);
    flux_mix<D>(L, R, 1.0, 1.0, -a, Fs2);
    return;
  }
  double lmL, lpL, lmR, lpR, XL, rL, irL, XR, rR, irR;
  wavespeeds_full<D>(L, lmL, lpL, XL, rL, irL, nullptr);
  wavespeeds_full<D>(R, lmR, lpR, XR, rR, irR, nullptr);
  double FL[5], FR[5];  // the normal fluxes, for HLLC and the tape
  if (TAPE || p.flux == 2) {
    phys_flux_dir<D>(L.U, L.v, L.P, FL);
    phys_flux_dir<D>(R.U, R.v, R.P, FR);
  }
  if (TAPE) {
    face_tape(L, FL, rL, irL, lmL, lpL, recL);
    face_tape(R, FR, rR, irR, lmR, lpR, recR);
  }
  // the selections compare bit patterns on the integer pipe (the FP64 pipe is the bottleneck)
  const double lamL = min_bits(lmL, lmR), lamR = max_bits(lpL, lpR);
  if (p.flux == 1) {
    const double sL = dbits(lamL) < 0 ? lamL : 0.0, sR = pos_bits(lamR) ? lamR : 0.0;
    const double den = sR - sL;
    if (den == 0.0) {
      flux_mix<D>(L, R, 1.0, 1.0, 0.0, Fs2);
    } else {
      const double id2 = recip_nr(0.5 * den);  // 2 / (S_R - S_L)
      const double cR = sR * id2, cL = sL * id2;
      flux_mix<D>(L, R, cR, -cL, sL * cR, Fs2);
    }
  } else if (p.flux == 2) {
    double Fs[5];
    hllc_flux<D>(L, R, FL, FR, lamL, lamR, Fs);
#pragma unroll
    for (int v = 0; v < 5; ++v) put_flux(Fs2[v], 2.0 * Fs[v]);
  } else {
    const double a = max_bits(abs_bits(lamL), abs_bits(lamR));
    flux_mix<D>(L, R, 1.0, 1.0, -a, Fs2);
  }
}

// con2prim adjoint by the implicit-function theorem: W = (rho, v, P) inverts
// U = prim2cons(W) (Eq. primitive_to_conserved), so U_bar = (dU/dW)^{-T} W_bar.
// With E = tau + D the map is D = gamma rho, S = w gamma^2 v, E = w gamma^2 - P (w = rho h), and
// (dU/dW)^T x = W_bar becomes, for y = (x_D - x_tau, x_S, x_tau) and a = v . y_S,
//   gamma y_D + w_rho gamma^2 (a + y_E)                       = W_bar_rho
//   rho gamma^3 v y_D + w gamma^2 y_S + 2 w gamma^4 v (a + y_E) = W_bar_v
//   w_P gamma^2 a + (w_P gamma^2 - 1) y_E                     = W_bar_P
// The v equation gives y_S = (W_bar_v - c v) / (w gamma^2), c = rho gamma^3 y_D + 2 w gamma^4 s
// with s = a + y_E; projected on v it closes a 3 x 3 system in (y_D, a, y_E).  Its first and
// third rows give y_D = W_bar_rho / gamma - w_rho gamma s and y_E = w_P gamma^2 s - W_bar_P, and
// the projected second row then leaves one equation for s:
//   gamma^2 [w (1 - w_P gamma^2) + u^2 (2w - rho w_rho)] s
//       = v . W_bar_v - w gamma^2 W_bar_P - rho u^2 W_bar_rho        (u^2 = gamma^2 v^2).
// lor = gamma, ilor = 1/gamma, g2 = gamma^2, u2 = gamma^2 v^2 are passed in.
__device__ __forceinline__ void c2p_adjoint(const Params& p, double rho, const double v[3], double P,
                                            double lor, double ilor, double g2, double u2,
                                            const double Wb[5], double Ub[5]) {
  double w, w_r, w_P;
  if (p.eos == 0) {
    w = fma(p.alpha, P, rho);
    w_r = 1.0;
    w_P = p.alpha;
  } else {
    const double x2 = fma(P, P, (4.0 / 9.0) * rho * rho);
    const double isg = rsqrt_nr(x2);
    const double sg = x2 * isg;
    w = fma(2.5, P, 1.5 * sg);
    w_r = (2.0 / 3.0) * rho * isg;
    w_P = fma(1.5 * P, isg, 2.5);
  }
  const double vW = fma(v[0], Wb[1], fma(v[1], Wb[2], v[2] * Wb[3]));
  const double wg2 = w * g2, wPg2 = w_P * g2;
  const double Kp = fma(u2, fma(-rho, w_r, 2.0 * w), w * (1.0 - wPg2));
  const double num = fma(-rho * u2, Wb[0], fma(-wg2, Wb[4], vW));
  // 1/(gamma^2 K') and 1/(w gamma^2) from one division
  const double gK = g2 * Kp;
  const double t = recip_nr(gK * wg2);
  const double s = num * (t * wg2);
  const double iw = t * gK;
  const double yD = fma(-w_r * lor, s, Wb[0] * ilor);
  const double yE = fma(wPg2, s, -Wb[4]);
  const double c = fma(rho * g2 * lor, yD, 2.0 * wg2 * g2 * s);
  Ub[0] = yD + yE;
#pragma unroll
  for (int k = 0; k < 3; ++k) Ub[1 + k] = fma(-c, v[k], Wb[1 + k]) * iw;
  Ub[4] = yE;
}

}  // namespace dgsrhd
