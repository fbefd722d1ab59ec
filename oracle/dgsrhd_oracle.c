/*
 * Oracle for the DG special-relativistic hydrodynamics hot path
 * (arXiv 2205.00095, Glines et al.).  TEST INFRASTRUCTURE ONLY: this file is
 * the plain, slow FP64 CPU restatement of the method that the CUDA library is
 * checked against.  Only tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * Every routine follows the paper's equations in the paper's order, written as
 * loops over elements, nodes, lines and faces.  No blocking, fusion or
 * reordering.  Units c = 1.
 *
 * State layout (both here and at the library boundary):
 *   U[var][elem][node], var = (D, S_x, S_y, S_z, tau), tau = E - D,
 *   elem = ex + nx*(ey + ny*ez), node = a + N*(b + N*c), N = p + 1.
 * Primitive layout W[var][elem][node], var = (rho, v_x, v_y, v_z, P).
 *
 * Readings where the paper is silent, garbled or ambiguous are marked
 * "Reading:" in the comments.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NVAR 5
#define MAXN 8

/* ------------------------------------------------------------------------ */
/* Configuration (mirrors the user-facing problem description)              */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t dim;            /* 1..3 */
  int32_t degree;         /* p; N = p + 1 Gauss-Legendre nodes per axis */
  int64_t n_elem[3];
  double lo[3], hi[3];
  int32_t eos;            /* 0 ideal, 1 Taub-Matthews */
  double gamma_ad;        /* Gamma of the ideal EOS */
  int32_t c2p;            /* 0 analytic, 1 iterative, 2 default (ideal->analytic, TM->iterative) */
  int32_t c2p_max_iter;   /* <=0 : default (30 Newton, 100 Brent) */
  double c2p_rtol;        /* >0: the iterative solvers also stop at this relative step / bracket */
  int32_t flux;           /* 0 LLF, 1 HLL, 2 HLLC */
  int32_t rk_stages;      /* 1, 2, 3 */
  int32_t bc[3][2];       /* 0 periodic, 1 Dirichlet, 2 outflow, 3 reflecting wall */
  double bc_state[3][2][5]; /* Dirichlet primitive (rho, vx, vy, vz, P) */
  int32_t enforce;        /* physicality operator after every stage: 1 nodes, 2 nodes and face points */
  int32_t nodes;          /* 0 Gauss-Legendre, 1 Gauss-Lobatto-Legendre (degree >= 1) */
  int32_t limiter;        /* after every stage, before the operator: 1 scaling, 2 minmod */
  double limiter_alpha;   /* 1: bound relaxation limiter_alpha h^(3/2); 2: TVB constant M (M h^2) */
} or_config;

typedef struct {
  int64_t c2p_calls;
  int64_t c2p_iters_total;
  int64_t c2p_iters_max;
  int64_t c2p_nonconverged;
  int64_t c2p_invalid_input;
  int64_t face_guard_hits;
  int64_t enforced_cells;
  int64_t mean_inadmissible_cells;
  int64_t limited_cells;
} or_stats;

/* ------------------------------------------------------------------------ */
/* Basis (Sec. 2.3, Eq. interpolation): nodal Lagrange on Gauss-Legendre     */
/* ------------------------------------------------------------------------ */

/* Legendre P_n(x) and P_n'(x) by the three-term recurrence. */
static void legendre(int n, double x, double *pn, double *dpn) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *pn = 1.0; *dpn = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1; p1 = pk;
  }
  *pn = p1;
  *dpn = n * (x * p1 - p0) / (x * x - 1.0);
}

/* N Gauss-Legendre nodes (ascending) and weights on [-1, 1], by Newton's
 * method on P_N from the Chebyshev-like initial guess. */
int or_gauss_legendre(int N, double *x, double *w) {
  if (N < 1 || N > MAXN) return 1;
  if (N == 1) { x[0] = 0.0; w[0] = 2.0; return 0; }
  for (int i = 0; i < N; ++i) {
    double xi = -cos(M_PI * (i + 0.75) / (N + 0.5));
    for (int it = 0; it < 100; ++it) {
      double pn, dpn;
      legendre(N, xi, &pn, &dpn);
      double dx = pn / dpn;
      xi -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    double pn, dpn;
    legendre(N, xi, &pn, &dpn);
    x[i] = xi;
    w[i] = 2.0 / ((1.0 - xi * xi) * dpn * dpn);
  }
  return 0;
}

/* N >= 2 Gauss-Lobatto-Legendre nodes (ascending) and weights on [-1, 1]: the end points and
 * the N - 2 roots of P'_{N-1}, found by Newton's method with
 * P''_n = (2 x P'_n - n (n + 1) P_n) / (1 - x^2) from the Chebyshev-Lobatto guesses;
 * weights 2 / (N (N - 1) P_{N-1}(x_i)^2). */
int or_gauss_lobatto(int N, double *x, double *w) {
  if (N < 2 || N > MAXN) return 1;
  const int n = N - 1;
  for (int i = 0; i < N; ++i) {
    double xi = -cos(M_PI * i / (double)n);
    if (i > 0 && i < n) {
      for (int it = 0; it < 100; ++it) {
        double pn, dpn;
        legendre(n, xi, &pn, &dpn);
        double d2 = (2.0 * xi * dpn - n * (n + 1.0) * pn) / (1.0 - xi * xi);
        double dx = dpn / d2;
        xi -= dx;
        if (fabs(dx) < 1e-16) break;
      }
    }
    double pn, dpn;
    if (i == 0) xi = -1.0;
    if (i == n) xi = 1.0;
    legendre(n, xi, &pn, &dpn);
    /* P_n(+-1) = (+-1)^n; the derivative formula is not needed at the end points */
    if (i == 0) pn = (n % 2) ? -1.0 : 1.0;
    if (i == n) pn = 1.0;
    x[i] = xi;
    w[i] = 2.0 / (N * (N - 1.0) * pn * pn);
  }
  return 0;
}

/* Lagrange polynomial phi_i(t) through nodes x[0..N-1]. */
static double lagrange(int N, const double *x, int i, double t) {
  double v = 1.0;
  for (int j = 0; j < N; ++j)
    if (j != i) v *= (t - x[j]) / (x[i] - x[j]);
  return v;
}

/* phi_i'(t) as the sum over k of the product with factor k differentiated. */
static double lagrange_deriv(int N, const double *x, int i, double t) {
  double s = 0.0;
  for (int k = 0; k < N; ++k) {
    if (k == i) continue;
    double prod = 1.0 / (x[i] - x[k]);
    for (int j = 0; j < N; ++j)
      if (j != i && j != k) prod *= (t - x[j]) / (x[i] - x[j]);
    s += prod;
  }
  return s;
}

/* Basis tables for the collocated weak form (Eq. discrete_hyperbolic_
 * conservation_law with the quadratures Eqs. quad-vol-flux, quad-surface-flux
 * taken at the nodes):
 *   Dhat[i*N + a] = w_a phi_i'(x_a) / w_i   (volume term)
 *   em[i] = phi_i(-1), ep[i] = phi_i(+1)   (trace extrapolation)
 * The lifting coefficients are ep[i]/w_i and em[i]/w_i. */
int or_basis_family(int N, int family, double *x, double *w, double *Dhat, double *em,
                    double *ep) {
  if (family == 1 ? or_gauss_lobatto(N, x, w) : or_gauss_legendre(N, x, w)) return 1;
  for (int i = 0; i < N; ++i) {
    for (int a = 0; a < N; ++a)
      Dhat[i * N + a] = (N == 1) ? 0.0 : w[a] * lagrange_deriv(N, x, i, x[a]) / w[i];
    em[i] = lagrange(N, x, i, -1.0);
    ep[i] = lagrange(N, x, i, +1.0);
  }
  return 0;
}

int or_basis(int N, double *x, double *w, double *Dhat, double *em, double *ep) {
  return or_basis_family(N, 0, x, w, Dhat, em, ep);
}

/* ------------------------------------------------------------------------ */
/* Equations of state (Sec. 2.2)                                             */
/* ------------------------------------------------------------------------ */

/* Specific enthalpy minus rest mass, h - 1, as a function of (rho, P):
 * Eq. id_enthalpy gives Gamma/(Gamma-1) Theta (ideal); the Taub-Matthews
 * h = 5/2 Theta + 3/2 sqrt(Theta^2 + 4/9), Theta = P/rho, gives
 * h - 1 = 5/2 Theta + 3/2 Theta^2 / (sqrt(Theta^2 + 4/9) + 2/3).
 * Reading: h - 1 is formed without cancellation so that cold states keep
 * their internal energy; h = 1 + (h - 1). */
static double eos_hm1(const or_config *c, double rho, double P) {
  double th = P / rho;
  if (c->eos == 0) return c->gamma_ad / (c->gamma_ad - 1.0) * th;
  return 2.5 * th + 1.5 * th * th / (sqrt(th * th + 4.0 / 9.0) + 2.0 / 3.0);
}

static double eos_enthalpy(const or_config *c, double rho, double P) {
  return 1.0 + eos_hm1(c, rho, P);
}

/* Sound speed squared: Gamma Theta / h (ideal); the Taub-Matthews ratio
 * (3 Th^2 + 5 Th s) / (12 Th^2 + 2 + 12 Th s), s = sqrt(Th^2 + 4/9). */
static double eos_cs2(const or_config *c, double rho, double P) {
  double th = P / rho;
  if (c->eos == 0) return c->gamma_ad * th / eos_enthalpy(c, rho, P);
  double s = sqrt(th * th + 4.0 / 9.0);
  return (3.0 * th * th + 5.0 * th * s) / (12.0 * th * th + 2.0 + 12.0 * th * s);
}

/* ------------------------------------------------------------------------ */
/* prim -> cons (Eq. primitive_to_conserved), with tau = E - D               */
/* ------------------------------------------------------------------------ */
/* Reading: tau = gamma^2 rho h - P - gamma rho is evaluated as
 * D u^2/(gamma + 1) + gamma^2 rho (h - 1) - P (u = gamma v), the same value
 * without the cancellation of the rest-mass terms. */
static void prim2cons_point(const or_config *c, const double W[5], double U[5]) {
  double rho = W[0], vx = W[1], vy = W[2], vz = W[3], P = W[4];
  double v2 = vx * vx + vy * vy + vz * vz;
  double gam = 1.0 / sqrt(1.0 - v2);
  double hm1 = eos_hm1(c, rho, P);
  double D = gam * rho;
  double rhohg2 = gam * gam * rho * (1.0 + hm1);
  U[0] = D;
  U[1] = rhohg2 * vx;
  U[2] = rhohg2 * vy;
  U[3] = rhohg2 * vz;
  U[4] = D * gam * gam * v2 / (gam + 1.0) + gam * gam * rho * hm1 - P;
}

/* Same map from the interpolated primitive (rho, u, P), u = gamma v
 * (the vector the method interpolates, Sec. 2.3). */
static void prim_u_to_cons(const or_config *c, const double Wu[5], double U[5],
                           double *gam_out) {
  double ux = Wu[1], uy = Wu[2], uz = Wu[3];
  double gam = sqrt(1.0 + ux * ux + uy * uy + uz * uz);
  double W[5] = {Wu[0], ux / gam, uy / gam, uz / gam, Wu[4]};
  prim2cons_point(c, W, U);
  *gam_out = gam;
}

int or_prim2cons(const or_config *c, int64_t n, const double *W, double *U) {
  for (int64_t k = 0; k < n; ++k) {
    double w[5], u[5];
    for (int v = 0; v < 5; ++v) w[v] = W[v * n + k];
    prim2cons_point(c, w, u);
    for (int v = 0; v < 5; ++v) U[v * n + k] = u[v];
  }
  return 0;
}

static int admissible_parts(double D, double S2, double tau);

/* ------------------------------------------------------------------------ */
/* cons -> prim (Sec. 3)                                                     */
/* ------------------------------------------------------------------------ */

/* Ideal EOS, analytic: the quartic in beta (Sec. 3.1) solved by the
 * resolvent-cubic (Ferrari) route.
 * Reading: the quartic is monic, beta^4 + a3 beta^3 + a2 beta^2 + a1 beta
 * + a0 = 0, with the printed a3..a0; R uses 9 i1 i2; the T < 0 branch is
 * x = 2 (R^2 - T)^(1/6) cos(atan2(sqrt(-T), R)/3) - i1/3 (trigonometric
 * Cardano).  Returns beta, or NaN when the closed form breaks down. */
static double c2p_ideal_analytic_beta(double G, double xi, double eta) {
  double den = (G - 1.0) * (G - 1.0) * (xi * xi + 1.0);
  double a3 = -2.0 * G * (G - 1.0) * xi * eta / den;
  double a2 = (G * G * eta * eta + 2.0 * (G - 1.0) * xi * xi - (G - 1.0) * (G - 1.0)) / den;
  double a1 = -2.0 * G * xi * eta / den;
  double a0 = xi * xi / den;
  double i1 = -a2;
  double i2 = a3 * a1 - 4.0 * a0;
  double i3 = 4.0 * a2 * a0 - a1 * a1 - a3 * a3 * a0;
  double R = (9.0 * i1 * i2 - 27.0 * i3 - 2.0 * i1 * i1 * i1) / 54.0;
  double S = (3.0 * i2 - i1 * i1) / 9.0;
  double T = R * R + S * S * S;
  double x;
  if (T < 0.0)
    x = 2.0 * pow(R * R - T, 1.0 / 6.0) * cos(atan2(sqrt(-T), R) / 3.0) - i1 / 3.0;
  else
    x = cbrt(R + sqrt(T)) + cbrt(R - sqrt(T)) - i1 / 3.0;
  double B = 0.5 * (a3 + sqrt(a3 * a3 - 4.0 * a2 + 4.0 * x));
  double C = 0.5 * (x - sqrt(x * x - 4.0 * a0));
  return 0.5 * (-B + sqrt(B * B - 4.0 * C));
}

/* Ideal EOS, iterative: Newton-Raphson on the quartic P(w) of
 * Eq. iterative_quartic, beta = 2 w / (1 + w^2) (Eq. iterative_quartic_unknown;
 * Reading: the printed "u" there is beta = |v|), started from the small-xi
 * series of Eq. iterative_cubic_approximation.
 * Reading (stop rule, not printed): stop when |dw| <= 1e-14 w (Newton's
 * quadratic convergence then leaves the iterate at the rounding floor), or
 * |dw| <= rtol w for a caller's tolerance rtol > 1e-14; for xi < 1e-4 take the
 * series itself (its error is O(xi^5)).
 * Returns w; *iters gets the Newton iteration count, *conv 0/1. */
static double c2p_ideal_iterative_w(double G, double xi, double eta, int max_iter, double rtol,
                                    int *iters, int *conv) {
  double al = G / (G - 1.0);
  double k1 = al * eta - 1.0;
  double series = (al - 1.0) / (2.0 * k1) * xi
                + (al - 1.0) * (al - 1.0) / (8.0 * k1 * k1 * k1 * k1)
                  * ((al + 3.0) * (al * eta + 1.0) - 4.0 * (al + 1.0)) * xi * xi * xi;
  *iters = 0;
  *conv = 1;
  if (xi < 1e-4) return series;
  double w = series;
  if (!(w > 1e-300)) w = 1e-300;
  if (w > 1.0 - 1e-15) w = 1.0 - 1e-15;
  double c4 = (al - 1.0) * xi, c3 = -2.0 * (al * eta + 1.0), c2 = 2.0 * (al + 1.0) * xi,
         c1 = -2.0 * (al * eta - 1.0), c0 = (al - 1.0) * xi;
  /* Stop at |dw| <= 1e-14 w, or once the residual before the step is at the rounding level of
   * evaluating the quartic on (0, 1), |P(w)| <= 8 eps sum |c_k|: for xi ~ 1e3 that level keeps
   * the step near 1e-14 w and the first test alone would never end (reading R10). */
  const double pres = 8.0 * 2.220446049250313e-16 *
                      (fabs(c4) + fabs(c3) + fabs(c2) + fabs(c1) + fabs(c0));
  *conv = 0;
  for (int it = 1; it <= max_iter; ++it) {
    double P = (((c4 * w + c3) * w + c2) * w + c1) * w + c0;
    double dP = ((4.0 * c4 * w + 3.0 * c3) * w + 2.0 * c2) * w + c1;
    double dw = P / dP;
    w -= dw;
    *iters = it;
    if (fabs(dw) <= fmax(1e-14, rtol) * w || fabs(P) <= pres) { *conv = 1; break; }
  }
  return w;
}

/* Taub-Matthews cubic W^3 + c1 W^2 + c2 W + c3 = 0 in W = gamma^2 - 1
 * (Eq. synge_cubic). */
static void tm_cubic_coeffs(double xi, double eta, double *c1, double *c2, double *c3) {
  double e2 = eta * eta, x2 = xi * xi;
  double s = e2 + x2;
  double dmx = e2 - x2;
  double k = 4.0 * s - (x2 + 1.0);
  *c1 = (s * k - 14.0 * x2 * e2) / (2.0 * dmx * dmx);
  *c2 = (k * k - 57.0 * x2 * e2) / (16.0 * dmx * dmx);
  *c3 = -9.0 * x2 * e2 / (16.0 * dmx * dmx);
}

/* Taub-Matthews, analytic: discriminant d = Q^3 + R^2; trigonometric root
 * for d < 0, Cardano's real root otherwise (Sec. 3.2).
 * Reading: the root is clamped to W >= 0. */
static double c2p_tm_analytic_W(double xi, double eta) {
  double c1, c2, c3;
  tm_cubic_coeffs(xi, eta, &c1, &c2, &c3);
  double Q = (3.0 * c2 - c1 * c1) / 9.0;
  double R = (9.0 * c1 * c2 - 27.0 * c3 - 2.0 * c1 * c1 * c1) / 54.0;
  double d = Q * Q * Q + R * R;
  double W;
  if (d < 0.0) {
    double iota = acos(R / sqrt(-Q * Q * Q));
    W = 2.0 * sqrt(-Q) * cos(iota / 3.0) - c1 / 3.0;
  } else {
    W = -c1 / 3.0 + cbrt(R + sqrt(d)) + cbrt(R - sqrt(d));
  }
  if (W < 0.0) W = 0.0;
  return W;
}

static double tm_cubic(double c1, double c2, double c3, double W) {
  return ((W + c1) * W + c2) * W + c3;
}

/* Taub-Matthews, iterative: Brent's method (Brent 1973, "zero") on the cubic,
 * bracket gamma in [1, 200], i.e. W in [0, 200^2 - 1], upper end expanded
 * while there is no sign change (Sec. 3.2).
 * Reading: upper end x4 per expansion, at most 10 expansions; tolerance
 * max(2 eps, rtol) |b| + 1e-300 (rtol: a caller's relative tolerance); at
 * most max_iter iterations. */
static double c2p_tm_brent_W(double xi, double eta, int max_iter, double rtol, int *iters,
                             int *conv) {
  double c1, c2, c3;
  tm_cubic_coeffs(xi, eta, &c1, &c2, &c3);
  double a = 0.0, b = 200.0 * 200.0 - 1.0;
  double fa = tm_cubic(c1, c2, c3, a), fb = tm_cubic(c1, c2, c3, b);
  *iters = 0;
  *conv = 0;
  if (fa == 0.0) { *conv = 1; return 0.0; }
  for (int k = 0; k < 10 && fa * fb > 0.0; ++k) {
    b *= 4.0;
    fb = tm_cubic(c1, c2, c3, b);
  }
  if (fa * fb > 0.0) return NAN;
  double c = a, fc = fa, d = b - a, e = d;
  for (int it = 1; it <= max_iter; ++it) {
    *iters = it;
    if (fb * fc > 0.0) { c = a; fc = fa; d = b - a; e = d; }
    if (fabs(fc) < fabs(fb)) {
      a = b; b = c; c = a;
      fa = fb; fb = fc; fc = fa;
    }
    double tol = fmax(2.0 * 0x1p-52, rtol) * fabs(b) + 1e-300;
    double m = 0.5 * (c - b);
    if (fabs(m) <= tol || fb == 0.0) { *conv = 1; return b; }
    if (fabs(e) >= tol && fabs(fa) > fabs(fb)) {
      /* interpolation: secant when a == c, inverse quadratic otherwise */
      double s = fb / fa, p, q;
      if (a == c) {
        p = 2.0 * m * s;
        q = 1.0 - s;
      } else {
        double qq = fa / fc, r = fb / fc;
        p = s * (2.0 * m * qq * (qq - r) - (b - a) * (r - 1.0));
        q = (qq - 1.0) * (r - 1.0) * (s - 1.0);
      }
      if (p > 0.0) q = -q; else p = -p;
      if (2.0 * p < fmin(3.0 * m * q - fabs(tol * q), fabs(e * q))) {
        e = d; d = p / q;
      } else {
        d = m; e = m;
      }
    } else {
      d = m; e = m;
    }
    a = b; fa = fb;
    b += (fabs(d) > tol) ? d : (m > 0.0 ? tol : -tol);
    fb = tm_cubic(c1, c2, c3, b);
  }
  return b;
}

/* One point: U = (D, S_x, S_y, S_z, tau) -> W = (rho, v_x, v_y, v_z, P).
 * xi = |S|/D, eta = E/D (Sec. 3).  rho = D/gamma, v = beta S/|S| (Sec. 3.1).
 * Pressure: ideal P = (Gamma-1)(E - S.v - rho); Taub-Matthews
 * P = ((E - S.v)^2 - rho^2) / (3 (E - S.v)).
 * Reading: both are evaluated in the algebraically identical forms
 * E - S.v - rho = tau - S.v + D (1 - 1/gamma) and
 * (E - S.v)^2 - rho^2 = (E - S.v - rho)(E - S.v + rho), with 1 - 1/gamma
 * written without cancellation for each method (beta^2/(1 + sqrt(1-beta^2)),
 * 2 w^2/(1 + w^2), W/(gamma (gamma + 1))), so that cold states keep their
 * pressure.
 * Returns 0 ok, 1 invalid input (D <= 0, q <= 0 or not finite), 2 not
 * converged / closed form failed. */
static int con2prim_point(const or_config *c, const double U[5], double W[5], int *iters) {
  double D = U[0], Sx = U[1], Sy = U[2], Sz = U[3], tau = U[4];
  double E = tau + D;
  double S2 = Sx * Sx + Sy * Sy + Sz * Sz;
  *iters = 0;
  if (!admissible_parts(D, S2, tau) || !isfinite(S2) || !isfinite(tau)) {
    for (int v = 0; v < 5; ++v) W[v] = NAN;
    return 1;
  }
  double S = sqrt(S2);
  double xi = S / D, eta = E / D;
  int method = c->c2p;
  if (method == 2) method = (c->eos == 0) ? 0 : 1;
  int max_iter = c->c2p_max_iter;
  double beta, ginv, one_minus_ginv; /* |v|, 1/gamma, 1 - 1/gamma */
  int conv = 1;
  if (S2 == 0.0) {
    beta = 0.0; ginv = 1.0; one_minus_ginv = 0.0;
  } else if (c->eos == 0 && method == 0) {
    beta = c2p_ideal_analytic_beta(c->gamma_ad, xi, eta);
    if (!(beta >= 0.0 && beta < 1.0)) conv = 0;
    ginv = sqrt(1.0 - beta * beta);
    one_minus_ginv = beta * beta / (1.0 + ginv);
  } else if (c->eos == 0) {
    if (max_iter <= 0) max_iter = 30;
    double w = c2p_ideal_iterative_w(c->gamma_ad, xi, eta, max_iter, c->c2p_rtol, iters, &conv);
    beta = 2.0 * w / (1.0 + w * w);
    ginv = (1.0 - w * w) / (1.0 + w * w);
    one_minus_ginv = 2.0 * w * w / (1.0 + w * w);
    if (!(w > 0.0 && w < 1.0)) conv = 0;
  } else {
    double Wl;
    if (method == 0) {
      Wl = c2p_tm_analytic_W(xi, eta);
    } else {
      if (max_iter <= 0) max_iter = 100;
      Wl = c2p_tm_brent_W(xi, eta, max_iter, c->c2p_rtol, iters, &conv);
    }
    if (!(Wl >= 0.0) || !isfinite(Wl)) conv = 0;
    /* gamma = sqrt(W + 1), beta = sqrt(W / (W + 1)) */
    double gam = sqrt(Wl + 1.0);
    beta = sqrt(Wl / (Wl + 1.0));
    ginv = 1.0 / gam;
    one_minus_ginv = Wl / (gam * (gam + 1.0));
  }
  double rho = D * ginv;
  double vs = (S2 == 0.0) ? 0.0 : beta / S; /* v = beta S / |S| */
  double vx = vs * Sx, vy = vs * Sy, vz = vs * Sz;
  double Sv = Sx * vx + Sy * vy + Sz * vz;
  double e_minus_rho = tau - Sv + D * one_minus_ginv; /* E - S.v - rho */
  double P;
  if (c->eos == 0) {
    P = (c->gamma_ad - 1.0) * e_minus_rho;
  } else {
    double Ev = E - Sv;
    P = e_minus_rho * (Ev + rho) / (3.0 * Ev);
  }
  W[0] = rho; W[1] = vx; W[2] = vy; W[3] = vz; W[4] = P;
  return conv ? 0 : 2;
}

static void stats_c2p(or_stats *st, int status, int iters) {
  if (!st) return;
  st->c2p_calls++;
  st->c2p_iters_total += iters;
  if (iters > st->c2p_iters_max) st->c2p_iters_max = iters;
  if (status == 1) st->c2p_invalid_input++;
  if (status == 2) st->c2p_nonconverged++;
}

int or_con2prim(const or_config *c, int64_t n, const double *U, double *W, int32_t *iters,
                or_stats *st) {
  for (int64_t k = 0; k < n; ++k) {
    double u[5], w[5];
    int it;
    for (int v = 0; v < 5; ++v) u[v] = U[v * n + k];
    int status = con2prim_point(c, u, w, &it);
    stats_c2p(st, status, it);
    for (int v = 0; v < 5; ++v) W[v * n + k] = w[v];
    if (iters) iters[k] = it;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Flux, wavespeeds, numerical flux (Secs. 2.1, 2.4)                          */
/* ------------------------------------------------------------------------ */

/* Physical flux along direction d (Eq. srhd_flux) in the variables
 * (D, S, tau): F = (D v_d, S v_d + P e_d, (tau + P) v_d). */
static void phys_flux(const double U[5], const double W[5], int d, double F[5]) {
  double vd = W[1 + d], P = W[4];
  F[0] = U[0] * vd;
  F[1] = U[1] * vd;
  F[2] = U[2] * vd;
  F[3] = U[3] * vd;
  F[1 + d] += P;
  F[4] = (U[4] + P) * vd;
}

/* lambda_pm along d (Sec. 2.4): (v_d +- sqrt(sig (1 - v_d^2 + sig)))/(1 + sig),
 * sig = cs^2 / (gamma^2 (1 - cs^2)). */
static void wavespeeds(const or_config *c, const double W[5], double gam, int d,
                       double *lm, double *lp) {
  double cs2 = eos_cs2(c, W[0], W[4]);
  double sig = cs2 / (gam * gam * (1.0 - cs2));
  double vd = W[1 + d];
  double r = sqrt(sig * (1.0 - vd * vd + sig));
  *lm = (vd - r) / (1.0 + sig);
  *lp = (vd + r) / (1.0 + sig);
}

/* HLLC flux (the paper names the solver but prints no formula; this is the relativistic HLLC
 * construction of the literature it cites, restated in the variables (D, S, tau)).  With the
 * outer wavespeeds lamL < 0 < lamR, the HLL averages
 *   U_hll = (lamR U_R - lamL U_L - F_R + F_L) / (lamR - lamL),
 *   F_hll = (lamR F_L - lamL F_R + lamR lamL (U_R - U_L)) / (lamR - lamL)
 * give, with E = tau + D, its flux F_E = F_tau + F_D (= S_d) and m = S_d, the contact speed as
 * the root of F_E,hll x^2 - (E_hll + F_m,hll) x + m_hll = 0 that equals v_d for two equal
 * states, written without cancellation as x = 2 m / (b + sqrt(b^2 - 4 F_E m)), b = E + F_m;
 * the contact pressure p* = F_m,hll - x F_E,hll.  On the side K the contact faces (left when
 * x >= 0) the star state is
 *   D* = D (lam - v) / (lam - x),
 *   S*_d = (S_d (lam - v) + p* - p) / (lam - x),   S*_t = S_t (lam - v) / (lam - x),
 *   tau* = (tau (lam - v) + p* x - p v) / (lam - x)   (E* - D*, no cancellation),
 * with v = v_d, p the pressure and lam the outer speed of K, and F* = F_K + lam (U*_K - U_K).
 * lamL >= 0 gives F_L and lamR <= 0 gives F_R. */
static void hllc_flux(const double UL[5], const double UR[5], const double FL[5],
                      const double FR[5], const double WL[5], const double WR[5], double lamL,
                      double lamR, int d, double Fs[5]) {
  if (lamL >= 0.0) {
    for (int v = 0; v < 5; ++v) Fs[v] = FL[v];
    return;
  }
  if (lamR <= 0.0) {
    for (int v = 0; v < 5; ++v) Fs[v] = FR[v];
    return;
  }
  double Uh[5], Fh[5];
  for (int v = 0; v < 5; ++v) {
    Uh[v] = (lamR * UR[v] - lamL * UL[v] - FR[v] + FL[v]) / (lamR - lamL);
    Fh[v] = (lamR * FL[v] - lamL * FR[v] + lamR * lamL * (UR[v] - UL[v])) / (lamR - lamL);
  }
  const double Eh = Uh[4] + Uh[0], FEh = Fh[4] + Fh[0], mh = Uh[1 + d], Fmh = Fh[1 + d];
  const double b = Eh + Fmh;
  const double xs = 2.0 * mh / (b + sqrt(b * b - 4.0 * FEh * mh));
  const double ps = Fmh - xs * FEh;
  const int left = xs >= 0.0;
  const double *U = left ? UL : UR, *F = left ? FL : FR, *W = left ? WL : WR;
  const double lam = left ? lamL : lamR;
  const double v = W[1 + d], p = W[4];
  const double den = lam - xs;
  double Us[5];
  Us[0] = U[0] * (lam - v) / den;
  for (int k = 0; k < 3; ++k)
    Us[1 + k] = (k == d) ? (U[1 + d] * (lam - v) + ps - p) / den : U[1 + k] * (lam - v) / den;
  Us[4] = (U[4] * (lam - v) + ps * xs - p * v) / den;
  for (int k = 0; k < 5; ++k) Fs[k] = F[k] + lam * (Us[k] - U[k]);
}

/* Numerical flux between a left and right face state given as the
 * interpolated primitive (rho, u, P).
 * Reading (formulas not printed): HLL with S_L = min(lambda_L, 0),
 * S_R = max(lambda_R, 0), F = (S_R F_L - S_L F_R + S_L S_R (U_R - U_L))
 * / (S_R - S_L), the average when S_R = S_L = 0; LLF (Rusanov) with
 * a = max(|lambda_L|, |lambda_R|), F = (F_L + F_R)/2 - a (U_R - U_L)/2. */
static void numerical_flux(const or_config *c, const double WuL[5], const double WuR[5],
                           int d, double Fs[5]) {
  double UL[5], UR[5], gL, gR;
  prim_u_to_cons(c, WuL, UL, &gL);
  prim_u_to_cons(c, WuR, UR, &gR);
  double WL[5] = {WuL[0], WuL[1] / gL, WuL[2] / gL, WuL[3] / gL, WuL[4]};
  double WR[5] = {WuR[0], WuR[1] / gR, WuR[2] / gR, WuR[3] / gR, WuR[4]};
  double FL[5], FR[5];
  phys_flux(UL, WL, d, FL);
  phys_flux(UR, WR, d, FR);
  double lmL, lpL, lmR, lpR;
  wavespeeds(c, WL, gL, d, &lmL, &lpL);
  wavespeeds(c, WR, gR, d, &lmR, &lpR);
  double lamL = fmin(lmL, lmR), lamR = fmax(lpL, lpR);
  if (c->flux == 1) {
    double sL = fmin(lamL, 0.0), sR = fmax(lamR, 0.0);
    if (sR - sL == 0.0) {
      for (int v = 0; v < 5; ++v) Fs[v] = 0.5 * (FL[v] + FR[v]);
    } else {
      for (int v = 0; v < 5; ++v)
        Fs[v] = (sR * FL[v] - sL * FR[v] + sL * sR * (UR[v] - UL[v])) / (sR - sL);
    }
  } else if (c->flux == 2) {
    hllc_flux(UL, UR, FL, FR, WL, WR, lamL, lamR, d, Fs);
  } else {
    double a = fmax(fabs(lamL), fabs(lamR));
    for (int v = 0; v < 5; ++v) Fs[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * a * (UR[v] - UL[v]);
  }
}

/* ------------------------------------------------------------------------ */
/* Mesh helpers                                                              */
/* ------------------------------------------------------------------------ */
typedef struct {
  int dim, N, Nn;        /* Nn = N^dim nodes per element */
  int64_t n[3], E;
  double dx[3];
  double x[MAXN], w[MAXN], Dhat[MAXN * MAXN], em[MAXN], ep[MAXN];
} mesh;

static int mesh_init(const or_config *c, mesh *m) {
  if (c->dim < 1 || c->dim > 3 || c->degree < 0 || c->degree + 1 > MAXN) return 1;
  m->dim = c->dim;
  m->N = c->degree + 1;
  m->Nn = 1;
  m->E = 1;
  for (int d = 0; d < 3; ++d) {
    m->n[d] = (d < c->dim) ? c->n_elem[d] : 1;
    if (m->n[d] < 1) return 1;
    m->dx[d] = (d < c->dim) ? (c->hi[d] - c->lo[d]) / (double)m->n[d] : 1.0;
    m->E *= m->n[d];
    if (d < c->dim) m->Nn *= m->N;
  }
  if (c->nodes == 1 && m->N < 2) return 1;
  return or_basis_family(m->N, c->nodes, m->x, m->w, m->Dhat, m->em, m->ep);
}

static void node_ijk(const mesh *m, int node, int ijk[3]) {
  ijk[0] = node % m->N;
  ijk[1] = (m->dim > 1) ? (node / m->N) % m->N : 0;
  ijk[2] = (m->dim > 2) ? node / (m->N * m->N) : 0;
}

static int node_index(const mesh *m, const int ijk[3]) {
  int idx = ijk[0];
  if (m->dim > 1) idx += m->N * ijk[1];
  if (m->dim > 2) idx += m->N * m->N * ijk[2];
  return idx;
}

static void elem_coords(const mesh *m, int64_t e, int64_t ec[3]) {
  ec[0] = e % m->n[0];
  ec[1] = (e / m->n[0]) % m->n[1];
  ec[2] = e / (m->n[0] * m->n[1]);
}

static int64_t elem_index(const mesh *m, const int64_t ec[3]) {
  return ec[0] + m->n[0] * (ec[1] + m->n[1] * ec[2]);
}

static double node_weight(const mesh *m, int node) {
  int ijk[3];
  node_ijk(m, node, ijk);
  double w = 1.0;
  for (int d = 0; d < m->dim; ++d) w *= m->w[ijk[d]];
  return w;
}

int or_node_coords(const or_config *c, double *X) {
  mesh m;
  if (mesh_init(c, &m)) return 1;
  for (int64_t e = 0; e < m.E; ++e) {
    int64_t ec[3];
    elem_coords(&m, e, ec);
    for (int i = 0; i < m.Nn; ++i) {
      int ijk[3];
      node_ijk(&m, i, ijk);
      for (int d = 0; d < m.dim; ++d)
        X[((int64_t)d * m.E + e) * m.Nn + i] =
            c->lo[d] + (ec[d] + 0.5 * (1.0 + m.x[ijk[d]])) * m.dx[d];
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* DG right-hand side (Sec. 2.3)                                             */
/* ------------------------------------------------------------------------ */

/* Primitive (rho, u, P) with u = gamma v at every node (the interpolated
 * vector of Sec. 2.3), plus the nodal 3-velocity primitive. */
typedef struct {
  double *Wu; /* [5][E][Nn] : rho, u_x, u_y, u_z, P */
  double *Wv; /* [5][E][Nn] : rho, v_x, v_y, v_z, P */
} nodal_prims;

static void nodal_con2prim(const or_config *c, const mesh *m, const double *U, nodal_prims *np,
                           or_stats *st) {
  int64_t tot = m->E * m->Nn;
  or_stats loc;
  memset(&loc, 0, sizeof loc);
  for (int64_t k = 0; k < tot; ++k) {
    double u[5], w[5];
    int it;
    for (int v = 0; v < 5; ++v) u[v] = U[v * tot + k];
    int status = con2prim_point(c, u, w, &it);
    stats_c2p(&loc, status, it);
    double gam = 1.0 / sqrt(1.0 - (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]));
    for (int v = 0; v < 5; ++v) np->Wv[v * tot + k] = w[v];
    np->Wu[0 * tot + k] = w[0];
    np->Wu[1 * tot + k] = gam * w[1];
    np->Wu[2 * tot + k] = gam * w[2];
    np->Wu[3 * tot + k] = gam * w[3];
    np->Wu[4 * tot + k] = w[4];
  }
  if (st) {
    st->c2p_calls += loc.c2p_calls;
    st->c2p_iters_total += loc.c2p_iters_total;
    if (loc.c2p_iters_max > st->c2p_iters_max) st->c2p_iters_max = loc.c2p_iters_max;
    st->c2p_nonconverged += loc.c2p_nonconverged;
    st->c2p_invalid_input += loc.c2p_invalid_input;
  }
}

/* Trace of the interpolated primitive (rho, u, P) of element e on its face
 * in direction d, side (0 = low, 1 = high), at tangential node `tan` (the
 * node index with the d-th coordinate ignored): sum_i phi_i(+-1) W_i along
 * the normal line.
 * Reading (face guard): if the extrapolated rho or P is <= 0, the trace is
 * the primitive of the node on that line next to the face. */
static void face_trace(const mesh *m, const double *Wu, int64_t e, int d, int side,
                       const int tan_ijk[3], double out[5], int64_t *guard_hits) {
  int64_t tot = m->E * m->Nn;
  const double *coef = side ? m->ep : m->em;
  int ijk[3] = {tan_ijk[0], tan_ijk[1], tan_ijk[2]};
  for (int v = 0; v < 5; ++v) out[v] = 0.0;
  for (int a = 0; a < m->N; ++a) {
    ijk[d] = a;
    int node = node_index(m, ijk);
    for (int v = 0; v < 5; ++v) out[v] += coef[a] * Wu[v * tot + e * m->Nn + node];
  }
  if (!(out[0] > 0.0) || !(out[4] > 0.0)) {
    ijk[d] = side ? m->N - 1 : 0;
    int node = node_index(m, ijk);
    for (int v = 0; v < 5; ++v) out[v] = Wu[v * tot + e * m->Nn + node];
    if (guard_hits) (*guard_hits)++;
  }
}

/* Boundary ghost for a Dirichlet side: the fixed primitive (rho, v, P)
 * converted to (rho, u, P). */
static void dirichlet_ghost(const or_config *c, int d, int side, double out[5]) {
  const double *b = c->bc_state[d][side];
  double gam = 1.0 / sqrt(1.0 - (b[1] * b[1] + b[2] * b[2] + b[3] * b[3]));
  out[0] = b[0]; out[1] = gam * b[1]; out[2] = gam * b[2]; out[3] = gam * b[3]; out[4] = b[4];
}

/* R = dU/dt of the collocated nodal DG weak form:
 *   dU_i/dt = sum_d (2/dx_d) [ sum_a Dhat_{i_d a} F^d_a
 *                              - ep_{i_d}/w_{i_d} F*_{d,high}
 *                              + em_{i_d}/w_{i_d} F*_{d,low} ]
 * (Eq. discrete_hyperbolic_conservation_law with the node-collocated
 * quadratures Eqs. quad-vol-flux and quad-surface-flux).  Primitives are
 * recovered at the nodes and the primitive (rho, u, P) is interpolated to
 * the faces (Sec. 2.3). */
int or_rhs(const or_config *c, const double *U, double *R, or_stats *st) {
  mesh m;
  if (mesh_init(c, &m)) return 1;
  int64_t tot = m.E * m.Nn;
  nodal_prims np;
  np.Wu = (double *)malloc(sizeof(double) * 5 * tot);
  np.Wv = (double *)malloc(sizeof(double) * 5 * tot);
  if (!np.Wu || !np.Wv) { free(np.Wu); free(np.Wv); return 2; }
  nodal_con2prim(c, &m, U, &np, st);

  /* volume term */
  for (int64_t e = 0; e < m.E; ++e) {
    for (int i = 0; i < m.Nn; ++i) {
      int ijk[3];
      node_ijk(&m, i, ijk);
      double acc[5] = {0, 0, 0, 0, 0};
      for (int d = 0; d < m.dim; ++d) {
        double scale = 2.0 / m.dx[d];
        int jk[3] = {ijk[0], ijk[1], ijk[2]};
        for (int a = 0; a < m.N; ++a) {
          jk[d] = a;
          int node = node_index(&m, jk);
          double Ua[5], Wa[5], Fa[5];
          for (int v = 0; v < 5; ++v) {
            Ua[v] = U[v * tot + e * m.Nn + node];
            Wa[v] = np.Wv[v * tot + e * m.Nn + node];
          }
          phys_flux(Ua, Wa, d, Fa);
          for (int v = 0; v < 5; ++v) acc[v] += scale * m.Dhat[ijk[d] * m.N + a] * Fa[v];
        }
      }
      for (int v = 0; v < 5; ++v) R[v * tot + e * m.Nn + i] = acc[v];
    }
  }

  /* surface term: loop over every face of the mesh in each direction */
  int64_t guard = 0;
  int Nt = 1; /* tangential nodes per face */
  for (int d = 0; d < m.dim - 1; ++d) Nt *= m.N;
  for (int d = 0; d < m.dim; ++d) {
    double scale = 2.0 / m.dx[d];
    int64_t nf[3] = {m.n[0], m.n[1], m.n[2]};
    nf[d] += 1;
    int64_t nfaces = nf[0] * nf[1] * nf[2];
    for (int64_t f = 0; f < nfaces; ++f) {
      int64_t fc[3] = {f % nf[0], (f / nf[0]) % nf[1], f / (nf[0] * nf[1])};
      int64_t kd = fc[d];
      int periodic = (c->bc[d][0] == 0);
      /* neighbours: left element index (kd - 1), right element index kd */
      int64_t lc[3] = {fc[0], fc[1], fc[2]}, rc[3] = {fc[0], fc[1], fc[2]};
      lc[d] = kd - 1;
      rc[d] = kd;
      int has_left = kd > 0, has_right = kd < m.n[d];
      if (periodic) {
        if (!has_left) { lc[d] = m.n[d] - 1; has_left = 1; }
        if (!has_right) { rc[d] = 0; has_right = 1; }
        if (kd == m.n[d]) continue; /* same face as kd == 0 */
      }
      int64_t eL = has_left ? elem_index(&m, lc) : -1;
      int64_t eR = has_right ? elem_index(&m, rc) : -1;
      for (int t = 0; t < Nt; ++t) {
        /* tangential node coordinates in the other directions */
        int tan_ijk[3] = {0, 0, 0};
        int rem = t;
        for (int dd = 0; dd < m.dim; ++dd) {
          if (dd == d) continue;
          tan_ijk[dd] = rem % m.N;
          rem /= m.N;
        }
        double WL[5] = {0, 0, 0, 0, 0}, WR[5] = {0, 0, 0, 0, 0};
        if (eL >= 0) face_trace(&m, np.Wu, eL, d, 1, tan_ijk, WL, &guard);
        if (eR >= 0) face_trace(&m, np.Wu, eR, d, 0, tan_ijk, WR, &guard);
        /* ghosts: Dirichlet = fixed outer state; outflow = the interior trace; reflecting wall =
           the interior trace with its normal velocity reversed */
        if (eL < 0) {
          if (c->bc[d][0] == 1) dirichlet_ghost(c, d, 0, WL);
          else for (int v = 0; v < 5; ++v) WL[v] = WR[v];
          if (c->bc[d][0] == 3) WL[1 + d] = -WL[1 + d];
        }
        if (eR < 0) {
          if (c->bc[d][1] == 1) dirichlet_ghost(c, d, 1, WR);
          else for (int v = 0; v < 5; ++v) WR[v] = WL[v];
          if (c->bc[d][1] == 3) WR[1 + d] = -WR[1 + d];
        }
        double Fs[5];
        numerical_flux(c, WL, WR, d, Fs);
        /* lift onto the normal line in both neighbours */
        int ijk[3] = {tan_ijk[0], tan_ijk[1], tan_ijk[2]};
        for (int a = 0; a < m.N; ++a) {
          ijk[d] = a;
          int node = node_index(&m, ijk);
          if (eL >= 0)
            for (int v = 0; v < 5; ++v)
              R[v * tot + eL * m.Nn + node] -= scale * (m.ep[a] / m.w[a]) * Fs[v];
          if (eR >= 0)
            for (int v = 0; v < 5; ++v)
              R[v * tot + eR * m.Nn + node] += scale * (m.em[a] / m.w[a]) * Fs[v];
        }
      }
    }
  }
  if (st) st->face_guard_hits += guard;
  free(np.Wu);
  free(np.Wv);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Physicality-enforcing operator (Sec. 2.5)                                 */
/* ------------------------------------------------------------------------ */

/* Admissible set (Eq. physicality): D > 0 and q = E - sqrt(D^2 + |S|^2) > 0.
 * Readings: the sign under the root is the one of Eq. smoothed_state_physicality.  With
 * E = tau + D and D > 0, q > 0 holds exactly when E > 0 and E^2 > D^2 + |S|^2, i.e. when
 * tau > 0 and tau (tau + 2 D) > |S|^2; the test is made in that form (stored variables, no
 * cancellation of D against the root for cold states with tau << D, no root). */
static int admissible_parts(double D, double S2, double tau) {
  return D > 0.0 && tau > 0.0 && tau * (tau + 2.0 * D) > S2;
}

static int admissible(const double U[5]) {
  return admissible_parts(U[0], U[1] * U[1] + U[2] * U[2] + U[3] * U[3], U[4]);
}

/* Largest s in [0, 1] with s X + (1 - s) Xbar >= 0, for Xbar > 0. */
static double positivity_factor(double X, double Xbar) {
  if (X >= 0.0) return 1.0;
  return Xbar / (Xbar - X);
}

/* Largest factor s_i in [0, 1] for one point with conserved state Ui and admissible element mean
 * Ub: the two stages of Sec. 2.5 (Eqs. first_stage_positivity, first_stage_smoothed_state,
 * second_stage_quatratic, second_stage_coefficients, second_stage_solution).
 * Readings: the stage-2 coefficients with Delta = U~(1) - Ubar are
 *   a = dE^2 - dD^2 - |dS|^2, b = 2 (Ebar dE - Dbar dD - Sbar.dS),
 *   c0 = Ebar^2 - Dbar^2 - |Sbar|^2
 * and the root of Eq. second_stage_solution is evaluated in the equivalent
 * form 2 c0 / (-b + sqrt(b^2 - 4 a c0)), clamped to [0, 1]. */
static double point_factor(const double Ui[5], const double Ub[5]) {
  double Dbar = Ub[0], Ebar = Ub[4] + Ub[0];
  /* stage 1: positivity of D and E (Eq. first_stage_positivity) */
  double sD = positivity_factor(Ui[0], Dbar);
  double sE = positivity_factor(Ui[4] + Ui[0], Ebar);
  double s1 = fmin(sD, sE);
  double U1[5];
  for (int v = 0; v < 5; ++v) U1[v] = s1 * Ui[v] + (1.0 - s1) * Ub[v];
  if (admissible(U1)) return s1;
  /* stage 2: the quadratic of Eq. second_stage_quatratic */
  /* In the stored variables (E = tau + D):
   *   a  = dE^2 - dD^2 - |dS|^2          = dtau (dtau + 2 dD) - |dS|^2
   *   b  = 2 (Ebar dE - Dbar dD - Sbar.dS) = 2 (taubar (dtau + dD) + Dbar dtau - Sbar.dS)
   *   c0 = Ebar^2 - Dbar^2 - |Sbar|^2     = taubar (taubar + 2 Dbar) - |Sbar|^2 */
  double taubar = Ub[4];
  double dD = U1[0] - Ub[0];
  double dtau = U1[4] - Ub[4];
  double dS[3] = {U1[1] - Ub[1], U1[2] - Ub[2], U1[3] - Ub[3]};
  double a = dtau * (dtau + 2.0 * dD) - (dS[0] * dS[0] + dS[1] * dS[1] + dS[2] * dS[2]);
  double b = 2.0 * (taubar * (dtau + dD) + Dbar * dtau
                    - (Ub[1] * dS[0] + Ub[2] * dS[1] + Ub[3] * dS[2]));
  double c0 = taubar * (taubar + 2.0 * Dbar) - (Ub[1] * Ub[1] + Ub[2] * Ub[2] + Ub[3] * Ub[3]);
  double den = -b + sqrt(b * b - 4.0 * a * c0);
  double s2 = (den > 0.0) ? 2.0 * c0 / den : 1.0;
  if (s2 > 1.0) s2 = 1.0;
  if (s2 < 0.0) s2 = 0.0;
  return s1 * s2;
}

/* Conserved state of element e at face point `fp` (fp = (d * 2 + side) * Nt + t, t the
 * tangential node index with the d-th coordinate left out, the remaining axes in order):
 * the element's conserved polynomial sum_a phi_a(-+1) U_a along the normal line through t. */
static void face_point_state(const mesh *m, const double *U, int64_t e, int fp, double out[5]) {
  int64_t tot = m->E * m->Nn;
  int Nt = m->Nn / m->N;
  int d = fp / (2 * Nt), side = (fp / Nt) % 2, t = fp % Nt;
  int ijk[3] = {0, 0, 0}, k = 0;
  for (int a = 0; a < m->dim; ++a) {
    if (a == d) continue;
    ijk[a] = (k == 0) ? t % m->N : t / m->N;
    ++k;
  }
  const double *coef = (side == 1) ? m->ep : m->em;
  for (int v = 0; v < 5; ++v) out[v] = 0.0;
  for (int a = 0; a < m->N; ++a) {
    ijk[d] = a;
    int node = node_index(m, ijk);
    for (int v = 0; v < 5; ++v) out[v] += coef[a] * U[v * tot + e * m->Nn + node];
  }
}

/* The operator on one element, following the four-step procedure of
 * Sec. 2.5 (flag, check the mean, per-point s_i in two stages, s = min s_i,
 * smooth towards the mean, Eq. smoothed_states).
 * Readings: a flagged element uses s (1 - 1e-12) so that the smoothed points
 * are strictly inside the admissible set; an element whose mean is
 * inadmissible is left unchanged and counted.  With `faces` (the face-point
 * variant) the points are the nodes and the 2 dim N^(dim-1) face points of
 * the element's conserved polynomial: since the basis reproduces constants
 * (sum_a phi_a(-+1) = 1), smoothing the nodes smooths every face point by the
 * same s, so the minimum over both makes the polynomial admissible at the
 * faces too.  Returns the element's s. */
static double enforce_element(const mesh *m, double *U, int64_t e, or_stats *st, int faces) {
  int64_t tot = m->E * m->Nn;
  int nfp = faces ? 2 * m->dim * (m->Nn / m->N) : 0;
  int flagged = 0;
  for (int i = 0; i < m->Nn; ++i) {
    double Ui[5];
    for (int v = 0; v < 5; ++v) Ui[v] = U[v * tot + e * m->Nn + i];
    if (!admissible(Ui)) flagged = 1;
  }
  for (int fp = 0; fp < nfp; ++fp) {
    double Uf[5];
    face_point_state(m, U, e, fp, Uf);
    if (!admissible(Uf)) flagged = 1;
  }
  if (!flagged) return 1.0;
  double Ub[5] = {0, 0, 0, 0, 0}, wsum = 0.0;
  for (int i = 0; i < m->Nn; ++i) {
    double wi = node_weight(m, i);
    wsum += wi;
    for (int v = 0; v < 5; ++v) Ub[v] += wi * U[v * tot + e * m->Nn + i];
  }
  for (int v = 0; v < 5; ++v) Ub[v] /= wsum;
  if (!admissible(Ub)) {
    if (st) st->mean_inadmissible_cells++;
    return 1.0;
  }
  double s = 1.0;
  for (int i = 0; i < m->Nn; ++i) {
    double Ui[5];
    for (int v = 0; v < 5; ++v) Ui[v] = U[v * tot + e * m->Nn + i];
    double si = point_factor(Ui, Ub);
    if (si < s) s = si;
  }
  for (int fp = 0; fp < nfp; ++fp) {
    double Uf[5];
    face_point_state(m, U, e, fp, Uf);
    double si = point_factor(Uf, Ub);
    if (si < s) s = si;
  }
  s *= (1.0 - 1e-12);
  for (int i = 0; i < m->Nn; ++i)
    for (int v = 0; v < 5; ++v) {
      double *x = &U[v * tot + e * m->Nn + i];
      *x = s * (*x) + (1.0 - s) * Ub[v];
    }
  if (st) st->enforced_cells++;
  return s;
}

int or_enforce(const or_config *c, double *U, double *s_out, or_stats *st) {
  mesh m;
  if (mesh_init(c, &m)) return 1;
  for (int64_t e = 0; e < m.E; ++e) {
    double s = enforce_element(&m, U, e, st, c->enforce == 2);
    if (s_out) s_out[e] = s;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* SSP Runge-Kutta (Sec. 2.3; Shu & Osher 1989)                              */
/* Reading (coefficients not printed): Shu-Osher forms                       */
/*   RK1:    U^{n+1} = U + dt R(U)                                           */
/*   SSPRK2: U1 = U + dt R(U); U^{n+1} = 1/2 U + 1/2 (U1 + dt R(U1))         */
/*   SSPRK3: U1 = U + dt R(U); U2 = 3/4 U + 1/4 (U1 + dt R(U1));             */
/*           U^{n+1} = 1/3 U + 2/3 (U2 + dt R(U2))                           */
/* with the physicality operator after every stage.                         */
/* ------------------------------------------------------------------------ */
/* ------------------------------------------------------------------------ */
/* Slope limiter (reading: the paper adds the limiter of Moe et al. for p >= 1 */
/* but prints no formula; this is a scaling limiter of that kind).            */
/* For every element e with quadrature mean Ub_e and every conserved q: the   */
/* bounds M = max(Ub over e and its face neighbours) + alpha and              */
/* m = min(...) - alpha, alpha = limiter_alpha h^(3/2) (h the smallest dx);   */
/* the element's extremes M*, m* over its nodes and its face traces;          */
/* theta_q = min(1, (M - Ub)/(M* - Ub) if M* > M, (Ub - m)/(Ub - m*) if       */
/* m* < m); theta = min over q; U_i <- Ub + theta (U_i - Ub) (the mean is     */
/* kept and the state stays a convex combination of itself and its mean).    */
/* Non-periodic boundaries contribute no neighbour.                          */
/* ------------------------------------------------------------------------ */
static void limit_all(const or_config *c, const mesh *m, double *U, or_stats *st) {
  const int64_t tot = m->E * m->Nn;
  double wsum = 0.0, h = 1e300;
  for (int i = 0; i < m->Nn; ++i) wsum += node_weight(m, i);
  for (int d = 0; d < m->dim; ++d) h = fmin(h, m->dx[d]);
  const double alpha = c->limiter_alpha * pow(h, 1.5);
  double *mean = (double *)malloc(sizeof(double) * 5 * (size_t)m->E);
  if (!mean) return;
  for (int64_t e = 0; e < m->E; ++e)
    for (int v = 0; v < 5; ++v) {
      double acc = 0.0;
      for (int i = 0; i < m->Nn; ++i) acc += node_weight(m, i) * U[v * tot + e * m->Nn + i];
      mean[v * m->E + e] = acc / wsum;
    }
  int Nt = 1;
  for (int d = 0; d < m->dim - 1; ++d) Nt *= m->N;
  for (int64_t e = 0; e < m->E; ++e) {
    int64_t ec[3];
    elem_coords(m, e, ec);
    double theta = 1.0;
    for (int v = 0; v < 5; ++v) {
      const double ub = mean[v * m->E + e];
      double M = ub, mn = ub;
      for (int d = 0; d < m->dim; ++d)
        for (int side = 0; side < 2; ++side) {
          int64_t nc[3] = {ec[0], ec[1], ec[2]};
          nc[d] += side ? 1 : -1;
          if (nc[d] < 0 || nc[d] >= m->n[d]) {
            if (c->bc[d][side] != 0) continue;
            nc[d] = (nc[d] + m->n[d]) % m->n[d];
          }
          const double un = mean[v * m->E + elem_index(m, nc)];
          M = fmax(M, un);
          mn = fmin(mn, un);
        }
      M += alpha;
      mn -= alpha;
      /* extremes over the nodes and the face traces */
      double hi = -1e300, lo = 1e300;
      for (int i = 0; i < m->Nn; ++i) {
        const double q = U[v * tot + e * m->Nn + i];
        hi = fmax(hi, q);
        lo = fmin(lo, q);
      }
      for (int d = 0; d < m->dim; ++d)
        for (int side = 0; side < 2; ++side)
          for (int t = 0; t < Nt; ++t) {
            int ijk[3] = {0, 0, 0}, rem = t;
            for (int dd = 0; dd < m->dim; ++dd) {
              if (dd == d) continue;
              ijk[dd] = rem % m->N;
              rem /= m->N;
            }
            double q = 0.0;
            for (int a = 0; a < m->N; ++a) {
              ijk[d] = a;
              q += (side ? m->ep[a] : m->em[a]) * U[v * tot + e * m->Nn + node_index(m, ijk)];
            }
            hi = fmax(hi, q);
            lo = fmin(lo, q);
          }
      if (hi > M) theta = fmin(theta, (M - ub) / (hi - ub));
      if (lo < mn) theta = fmin(theta, (ub - mn) / (ub - lo));
    }
    if (theta < 1.0) {
      if (st) st->limited_cells += 1;
      for (int v = 0; v < 5; ++v) {
        const double ub = mean[v * m->E + e];
        for (int i = 0; i < m->Nn; ++i) {
          double *q = &U[v * tot + e * m->Nn + i];
          *q = ub + theta * (*q - ub);
        }
      }
    }
  }
  free(mean);
}

/* ------------------------------------------------------------------------ */
/* Minmod limiter (reading: Sec. 2.3 names the minmod limiter after van      */
/* Leer but prints no formula).  The minmod bound of Cockburn and Shu on the */
/* face deviations, applied through one factor per element so that every    */
/* node stays a convex combination of itself and the element mean (applied  */
/* to each conserved variable's slope on its own, it lost admissible means   */
/* on every strong blast of Sec. 4.2 at p = 1).  For element e, conserved q  */
/* and axis d:                                                                */
/*   ub   the element's quadrature mean of q,                                */
/*   a+_d = (quadrature mean of q's trace on the +d face) - ub,              */
/*   a-_d = ub - (the same on the -d face),                                  */
/*   D+_d = ub(+d neighbour) - ub, D-_d = ub - ub(-d neighbour)              */
/*          (a non-periodic boundary contributes no difference),             */
/*   mm(x, D+, D-) = x if |x| <= M h^2 + 2^-40 (|ub_D| + |ub_tau|) (h the    */
/*          smallest dx: the TVB threshold, plus a floor at the rounding of  */
/*          the element's energy scale, which bounds |S| as well),           */
/*          else s min(|x|, |D+|, |D-|) if all share the sign s, else 0;     */
/* theta = min(1, mm(a, D+_d, D-_d) / a over q, d and a in {a+_d, a-_d});    */
/* U_i <- ub + theta (U_i - ub).  The mean is kept; linear data pass         */
/* untouched; an element holding a strict extremum is flattened (theta = 0). */
/* ------------------------------------------------------------------------ */
static double minmod3(double x, const double *D, int nD, double thr) {
  if (fabs(x) <= thr) return x;
  double mag = fabs(x);
  for (int k = 0; k < nD; ++k) {
    if ((D[k] > 0.0) != (x > 0.0) || D[k] == 0.0) return 0.0;
    mag = fmin(mag, fabs(D[k]));
  }
  return x > 0.0 ? mag : -mag;
}

static void minmod_all(const or_config *c, const mesh *m, double *U, or_stats *st) {
  const int64_t tot = m->E * m->Nn;
  double wsum = 0.0, h = 1e300;
  for (int i = 0; i < m->Nn; ++i) wsum += node_weight(m, i);
  for (int d = 0; d < m->dim; ++d) h = fmin(h, m->dx[d]);
  const double thr = c->limiter_alpha * h * h;
  double *mean = (double *)malloc(sizeof(double) * 5 * (size_t)m->E);
  if (!mean) return;
  for (int64_t e = 0; e < m->E; ++e)
    for (int v = 0; v < 5; ++v) {
      double acc = 0.0;
      for (int i = 0; i < m->Nn; ++i) acc += node_weight(m, i) * U[v * tot + e * m->Nn + i];
      mean[v * m->E + e] = acc / wsum;
    }
  int Nt = 1;
  for (int d = 0; d < m->dim - 1; ++d) Nt *= m->N;
  const double face_wsum = wsum / 2.0; /* the tangential weights sum to 2^(dim-1) */
  for (int64_t e = 0; e < m->E; ++e) {
    int64_t ec[3];
    elem_coords(m, e, ec);
    const double thr_e = thr + 0x1p-40 * (fabs(mean[e]) + fabs(mean[4 * m->E + e]));
    double theta = 1.0;
    for (int v = 0; v < 5; ++v) {
      const double *q = &U[v * tot + e * m->Nn];
      const double ub = mean[v * m->E + e];
      for (int d = 0; d < m->dim; ++d) {
        double D[2];
        int nD = 0;
        for (int side = 1; side >= 0; --side) {
          int64_t nc[3] = {ec[0], ec[1], ec[2]};
          nc[d] += side ? 1 : -1;
          if (nc[d] < 0 || nc[d] >= m->n[d]) {
            if (c->bc[d][side] != 0) continue;
            nc[d] = (nc[d] + m->n[d]) % m->n[d];
          }
          const double un = mean[v * m->E + elem_index(m, nc)];
          D[nD++] = side ? un - ub : ub - un;
        }
        double fm[2] = {0.0, 0.0};
        for (int side = 0; side < 2; ++side)
          for (int t = 0; t < Nt; ++t) {
            int ijk[3] = {0, 0, 0}, rem = t;
            double wt = 1.0;
            for (int dd = 0; dd < m->dim; ++dd) {
              if (dd == d) continue;
              ijk[dd] = rem % m->N;
              rem /= m->N;
              wt *= m->w[ijk[dd]];
            }
            double tr = 0.0;
            for (int a = 0; a < m->N; ++a) {
              ijk[d] = a;
              tr += (side ? m->ep[a] : m->em[a]) * q[node_index(m, ijk)];
            }
            fm[side] += wt * tr;
          }
        const double dev[2] = {fm[1] / face_wsum - ub, ub - fm[0] / face_wsum};
        for (int k = 0; k < 2; ++k) {
          const double mmv = minmod3(dev[k], D, nD, thr_e);
          if (mmv != dev[k]) theta = fmin(theta, mmv / dev[k]);
        }
      }
    }
    if (theta < 1.0) {
      if (st) st->limited_cells += 1;
      for (int v = 0; v < 5; ++v) {
        const double ub = mean[v * m->E + e];
        for (int i = 0; i < m->Nn; ++i) {
          double *q = &U[v * tot + e * m->Nn + i];
          *q = ub + theta * (*q - ub);
        }
      }
    }
  }
  free(mean);
}

int or_step(const or_config *c, double *U, double dt, int nsteps, or_stats *st) {
  mesh m;
  if (mesh_init(c, &m)) return 1;
  if (c->rk_stages < 1 || c->rk_stages > 3) return 1;
  int64_t n = 5 * m.E * m.Nn;
  double *U0 = (double *)malloc(sizeof(double) * n);
  double *Uk = (double *)malloc(sizeof(double) * n);
  double *R = (double *)malloc(sizeof(double) * n);
  if (!U0 || !Uk || !R) { free(U0); free(Uk); free(R); return 2; }
  static const double a_n[3][3] = {{0.0, 0, 0}, {0.0, 0.5, 0}, {0.0, 0.75, 1.0 / 3.0}};
  static const double b_k[3][3] = {{1.0, 0, 0}, {1.0, 0.5, 0}, {1.0, 0.25, 2.0 / 3.0}};
  int ns = c->rk_stages;
  for (int step = 0; step < nsteps; ++step) {
    memcpy(U0, U, sizeof(double) * n);
    memcpy(Uk, U, sizeof(double) * n);
    for (int k = 0; k < ns; ++k) {
      int rc = or_rhs(c, Uk, R, st);
      if (rc) { free(U0); free(Uk); free(R); return rc; }
      double a = a_n[ns - 1][k], b = b_k[ns - 1][k];
      for (int64_t j = 0; j < n; ++j) Uk[j] = a * U0[j] + b * (Uk[j] + dt * R[j]);
      if (c->limiter == 1) limit_all(c, &m, Uk, st);
      if (c->limiter == 2) minmod_all(c, &m, Uk, st);
      if (c->enforce) or_enforce(c, Uk, NULL, st);
    }
    memcpy(U, Uk, sizeof(double) * n);
  }
  free(U0); free(Uk); free(R);
  return 0;
}

/* Reading (CFL rule not printed): dt = C / ((2p + 1) sum_d 1/dx_d), with
 * every characteristic speed bounded by c = 1. */
double or_cfl_dt(const or_config *c, double cfl) {
  mesh m;
  if (mesh_init(c, &m)) return -1.0;
  double s = 0.0;
  for (int d = 0; d < m.dim; ++d) s += 1.0 / m.dx[d];
  return cfl / ((2.0 * c->degree + 1.0) * s);
}

/* Single-point helpers for tests. */
int or_wavespeeds(const or_config *c, const double *Wv, int d, double *lm, double *lp) {
  double gam = 1.0 / sqrt(1.0 - (Wv[1] * Wv[1] + Wv[2] * Wv[2] + Wv[3] * Wv[3]));
  wavespeeds(c, Wv, gam, d, lm, lp);
  return 0;
}

int or_numerical_flux(const or_config *c, const double *WvL, const double *WvR, int d,
                      double *Fs) {
  double gL = 1.0 / sqrt(1.0 - (WvL[1] * WvL[1] + WvL[2] * WvL[2] + WvL[3] * WvL[3]));
  double gR = 1.0 / sqrt(1.0 - (WvR[1] * WvR[1] + WvR[2] * WvR[2] + WvR[3] * WvR[3]));
  double uL[5] = {WvL[0], gL * WvL[1], gL * WvL[2], gL * WvL[3], WvL[4]};
  double uR[5] = {WvR[0], gR * WvR[1], gR * WvR[2], gR * WvR[3], WvR[4]};
  numerical_flux(c, uL, uR, d, Fs);
  return 0;
}

int or_phys_flux(const or_config *c, const double *Wv, int d, double *F) {
  double U[5];
  prim2cons_point(c, Wv, U);
  phys_flux(U, Wv, d, F);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Diagnostic of the Kelvin-Helmholtz study (Sec. 4.5): the spatial mean of  */
/* the squared velocity component `axis`, <v_a^2> = (1/|Omega|) int v_a^2 dV, */
/* by the nodal quadrature of the basis: sum over elements and nodes of      */
/* (prod_d dx_d / 2) w_node v_a^2 with v from con2prim at the node.          */
/* ------------------------------------------------------------------------ */
double or_mean_square_velocity(const or_config *c, const double *U, int axis) {
  mesh m;
  if (mesh_init(c, &m) || axis < 0 || axis > 2) return NAN;
  const int64_t n = m.E * m.Nn;
  double *W = (double *)malloc(sizeof(double) * 5 * (size_t)n);
  int32_t *it = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  if (!W || !it) { free(W); free(it); return NAN; }
  or_stats st;
  memset(&st, 0, sizeof st);
  or_con2prim(c, n, U, W, it, &st);
  double jac = 1.0, vol = 1.0;
  for (int d = 0; d < m.dim; ++d) {
    jac *= 0.5 * m.dx[d];
    vol *= c->hi[d] - c->lo[d];
  }
  double sum = 0.0;
  for (int64_t e = 0; e < m.E; ++e)
    for (int i = 0; i < m.Nn; ++i) {
      const double v = W[(int64_t)(1 + axis) * n + e * m.Nn + i];
      sum += jac * node_weight(&m, i) * v * v;
    }
  free(W);
  free(it);
  return sum / vol;
}

double or_enthalpy(const or_config *c, double rho, double P) { return eos_enthalpy(c, rho, P); }
double or_cs2(const or_config *c, double rho, double P) { return eos_cs2(c, rho, P); }
