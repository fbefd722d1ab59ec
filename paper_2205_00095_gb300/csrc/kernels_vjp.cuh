// Vector-Jacobian product of the DG right-hand side, U_bar = (dR/dU)^T R_bar, and of the
// physicality operator with frozen smoothing factors.
//
// The forward RHS is R = Dhat-volume(F(U, W(U))) - lift(F*(traces(W(U)))).  Its reverse sweep:
//   face_vjp_kernel : per face point, F*_bar = (2/dx)(sum_a l-_a R_bar_right - sum_a l+_a R_bar_left)
//                     (transposed lift), then the reverse of the LLF/HLL flux with its branch
//                     choices (min/max of the wavespeeds, the clamps to 0, |lambda|) frozen at
//                     their forward values, giving the adjoints of the two face traces.
//   node_vjp_kernel : per node, the transposed volume contraction F_bar = (2/dx) Dhat^T R_bar, the
//                     transposed trace extrapolation (face guard as decided in the forward pass),
//                     the transposed flux Jacobians, and the con2prim adjoint by the
//                     implicit-function theorem: W(U) inverts U = prim2cons(W) (Eq.
//                     primitive_to_conserved), so U_bar = (dU/dW)^{-T} W_bar, a 5 x 5 solve at the
//                     converged root.
// Inputs kept from the forward pass: the nodal (rho, u, P), the face traces, the face-guard
// flags and, when the forward face kernel was asked for it, the face-state tape (the roots and
// reciprocals of every face state), which leaves the face reverse sweep without a root or a
// division.
#pragma once

#include "kernels.cuh"
#include "split.cuh"

namespace dgsrhd {

// ---------------------------------------------------------------------------------------
// One face state: forward with its intermediates, then its reverse.
// ---------------------------------------------------------------------------------------
struct FaceFwd : FaceState {
  double Wu[5];
  double H, rhoh_lor;
  double F[5];
  double X, r, ir, lm, lp;
};

// The forward face state with the intermediates of its reverse.  `t` (kFaceTape values at
// stride ts, or null) is the tape the forward face kernel wrote for this face state: with it only the flux
// and two sums are formed here; without it the state is evaluated in full.  Both give the same
// bits, since the tape holds what the same functions compute.
template <int D>
__device__ __forceinline__ void face_fwd(const Params& p, const double Wu[5],
                                         const double* __restrict__ t, long long ts, FaceFwd& f) {
#pragma unroll
  for (int k = 0; k < 5; ++k) f.Wu[k] = Wu[k];
  if (t) {
    f.ilor = t[0], f.isg = t[ts], f.iZ = t[2 * ts], f.id1 = t[3 * ts], f.i = t[4 * ts];
    f.ir = t[5 * ts], f.u2 = t[6 * ts], f.lor = t[7 * ts], f.sg = t[8 * ts], f.A = t[9 * ts];
    f.B = t[10 * ts], f.K = t[11 * ts], f.rho_hm1 = t[12 * ts];
#pragma unroll
    for (int k = 0; k < 5; ++k) f.U[k] = t[(13 + k) * ts];
    f.r = t[18 * ts], f.lm = t[19 * ts], f.lp = t[20 * ts];
#pragma unroll
    for (int k = 0; k < 5; ++k) f.F[k] = t[(21 + k) * ts];
    f.q = __dadd_rn(1.0, f.u2);
    f.P = Wu[4];
    f.v[0] = Wu[1] * f.ilor;
    f.v[1] = Wu[2] * f.ilor;
    f.v[2] = Wu[3] * f.ilor;
  } else {
    face_state_core(p, Wu, f, nullptr);
    wavespeeds_full<D>(f, f.lm, f.lp, f.X, f.r, f.ir, nullptr);
    phys_flux_dir<D>(f.U, f.v, f.P, f.F);
  }
  f.H = __dadd_rn(Wu[0], f.rho_hm1);
  f.rhoh_lor = f.H * f.lor;
}

// Reverse of face_fwd from the adjoints of its conserved state and normal flux already
// contracted with the flux map (Db, Sb, taub: the adjoints reaching D, S and tau; Pb, vdb: those
// reaching P and v_d through the flux) and of its wavespeeds (lmb, lpb) -> adjoint of the face
// primitive (rho, u, P).
template <int D>
__device__ __forceinline__ void face_rev_state(const Params& p, const FaceFwd& f, double Db,
                                               const double Sb[3], double taub, double Pb,
                                               double vdb, double lmb, double lpb,
                                               double Wb[5]) {
  const double rho = f.Wu[0], P = f.Wu[4];
  const double vd = f.v[D];
  // wavespeeds
  const double ib = lmb * (vd * f.B - f.r) + lpb * (vd * f.B + f.r);
  vdb = fma((lmb + lpb) * f.B, f.i, vdb);
  double Bb = (lmb + lpb) * vd * f.i - ib * f.i * f.i;
  double Ab = -ib * f.i * f.i;
  const double rb = (lpb - lmb) * f.i;
  const double Xb = 0.5 * rb * f.ir;
  Ab += Xb * (f.B * (1.0 - vd * vd) + 2.0 * f.A);
  Bb += Xb * f.A * (1.0 - vd * vd);
  vdb += Xb * f.A * f.B * (-2.0 * vd);
  // v_k = u_k / gamma
  double ub[3] = {0.0, 0.0, 0.0};
  ub[D] = vdb * f.ilor;
  double ilorb = vdb * f.Wu[1 + D];
  // tau = D u2/(gamma + 1) + q rho(h-1) - P
  Db += taub * f.u2 * f.id1;
  double u2b = taub * f.U[0] * f.id1;
  double lorb = -taub * f.U[0] * f.u2 * f.id1 * f.id1;
  double qb = taub * f.rho_hm1;
  double rhm1b = taub * f.q;
  Pb -= taub;
  // S_k = rho h gamma u_k
  const double rhlb = Sb[0] * f.Wu[1] + Sb[1] * f.Wu[2] + Sb[2] * f.Wu[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) ub[k] += Sb[k] * f.rhoh_lor;
  const double Hb = rhlb * f.lor;
  lorb += rhlb * f.H;
  double rhob = Hb;
  rhm1b += Hb;
  // D = gamma rho
  lorb += Db * rho;
  rhob += Db * f.lor;
  // equation of state
  if (p.eos == 0) {
    qb += Bb * f.K;  // B = q K, K = rho + (alpha - Gamma) P
    rhob += Bb * f.q;
    rhm1b += Bb * f.q;
    Ab -= Bb * f.q;
    Pb += Ab * p.gamma_ad + rhm1b * p.alpha;
  } else {
    qb += Bb * f.K;
    const double Kb = Bb * f.q;
    // K = 9 P^2 + 7 P s + 2 rho^2 and A = P (3 P + 5 s), s = sqrt(P^2 + 4 rho^2 / 9)
    Pb += fma(Kb, fma(18.0, P, 7.0 * f.sg), Ab * fma(6.0, P, 5.0 * f.sg));
    double sgb = P * fma(7.0, Kb, 5.0 * Ab);
    rhob += Kb * 4.0 * rho;
    Pb += rhm1b * (2.5 + 3.0 * P * f.iZ);
    const double Zb = -rhm1b * 1.5 * P * P * f.iZ * f.iZ;
    sgb += Zb;
    rhob += Zb * (2.0 / 3.0);
    Pb += sgb * P * f.isg;
    rhob += sgb * (4.0 / 9.0) * rho * f.isg;
  }
  // gamma = q^(1/2), 1/gamma = q^(-1/2), q = 1 + u2
  qb += 0.5 * f.ilor * (lorb - ilorb * f.ilor * f.ilor);
  const double u2b2 = 2.0 * (u2b + qb);  // u2 = |u|^2
  Wb[0] = rhob;
  Wb[1] = fma(f.Wu[1], u2b2, ub[0]);
  Wb[2] = fma(f.Wu[2], u2b2, ub[1]);
  Wb[3] = fma(f.Wu[3], u2b2, ub[2]);
  Wb[4] = Pb;
}

// Reverse of face_fwd: adjoints of its outputs (flux Fb, conserved state Ub, wavespeeds lmb,
// lpb) -> adjoint of the face primitive (rho, u, P).  vdb_in, Pb_in: direct uses of v_D and P
// (HLLC).
template <int D>
__device__ __forceinline__ void face_rev(const Params& p, const FaceFwd& f, const double Fb[5],
                                         const double Ub[5], double lmb, double lpb, double Wb[5],
                                         double vdb_in = 0.0, double Pb_in = 0.0) {
  const double vd = f.v[D], P = f.Wu[4];
  // flux along D: F = (D v_d, S v_d + P e_d, (tau + P) v_d)
  const double Sb[3] = {Ub[1] + Fb[1] * vd, Ub[2] + Fb[2] * vd, Ub[3] + Fb[3] * vd};
  const double vdb = vdb_in + (Fb[0] * f.U[0] + Fb[1] * f.U[1] + Fb[2] * f.U[2] +
                               Fb[3] * f.U[3] + Fb[4] * (f.U[4] + P));
  face_rev_state<D>(p, f, Ub[0] + Fb[0] * vd, Sb, Ub[4] + Fb[4] * vd,
                    Fb[1 + D] + fma(Fb[4], vd, Pb_in), vdb, lmb, lpb, Wb);
}

// face_rev for adjoints of the form Fb = alpha g, Ub = beta g (LLF and HLL: g = F*_bar per
// side, alpha and beta the side's weights): the flux map contracts to one factor
// kappa = alpha v_d + beta on (D, S, tau), and alpha on P and v_d.
template <int D>
__device__ __forceinline__ void face_rev_scaled(const Params& p, const FaceFwd& f, const double g[5],
                                                double alpha, double beta, double lmb, double lpb,
                                                double Wb[5]) {
  const double vd = f.v[D], P = f.Wu[4];
  const double kappa = fma(alpha, vd, beta);
  const double Sb[3] = {g[1] * kappa, g[2] * kappa, g[3] * kappa};
  const double gU = fma(g[0], f.U[0], fma(g[1], f.U[1], fma(g[2], f.U[2],
                    fma(g[3], f.U[3], g[4] * (f.U[4] + P)))));
  face_rev_state<D>(p, f, g[0] * kappa, Sb, g[4] * kappa, alpha * fma(g[4], vd, g[1 + D]),
                    alpha * gU, lmb, lpb, Wb);
}

// Reverse of hllc_flux<D> (the forward is re-evaluated here with the same formulas), with the
// choice of the contact's side and of the supersonic cases frozen.  Outputs: adjoints of the two
// face states' U and F, of lamL and lamR, and of the normal velocity and pressure of the side K
// the star state is built from (vKb, PKb, left = K is the left state).
template <int D>
__device__ __forceinline__ void hllc_flux_vjp(const FaceFwd& L, const FaceFwd& R, double lamL,
                                              double lamR, const double Fsb[5], double FLb[5],
                                              double FRb[5], double ULb[5], double URb[5],
                                              double& lamLb, double& lamRb, double& vKb,
                                              double& PKb, bool& left) {
#pragma unroll
  for (int k = 0; k < 5; ++k) FLb[k] = FRb[k] = ULb[k] = URb[k] = 0.0;
  lamLb = lamRb = vKb = PKb = 0.0;
  left = true;
  if (lamL >= 0.0 || lamR <= 0.0) {  // supersonic: the upwind physical flux
    const bool useL = lamL >= 0.0;
    left = useL;
#pragma unroll
    for (int k = 0; k < 5; ++k) (useL ? FLb : FRb)[k] = Fsb[k];
    return;
  }
  constexpr int m = 1 + D;
  const double idl = recip_nr(lamR - lamL), lrl = lamR * lamL;
  auto NU = [&](int c) { return lamR * R.U[c] - lamL * L.U[c] - R.F[c] + L.F[c]; };
  auto NF = [&](int c) { return lamR * L.F[c] - lamL * R.F[c] + lrl * (R.U[c] - L.U[c]); };
  const double Uh0 = NU(0) * idl, Uh4 = NU(4) * idl, Uhm = NU(m) * idl;
  const double Fh0 = NF(0) * idl, Fh4 = NF(4) * idl, Fhm = NF(m) * idl;
  const double Eh = Uh4 + Uh0, FEh = Fh4 + Fh0, mh = Uhm, Fmh = Fhm;
  const double b = Eh + Fmh;
  const double sq = sqrt(fma(b, b, -4.0 * FEh * mh));
  const double id1 = recip_nr(b + sq);
  const double xs = 2.0 * mh * id1;
  const double ps = fma(-xs, FEh, Fmh);
  left = xs >= 0.0;
  const FaceFwd& K = left ? L : R;
  const double lam = left ? lamL : lamR, v = K.v[D], P = K.P;
  const double lv = lam - v, di = recip_nr(lam - xs);
  double Num[5];
  Num[0] = K.U[0] * lv;
#pragma unroll
  for (int k = 0; k < 3; ++k) Num[1 + k] = (k == D) ? K.U[m] * lv + ps - P : K.U[1 + k] * lv;
  Num[4] = K.U[4] * lv + ps * xs - P * v;
  // F* = F_K + lam (Num di - U_K)
  double lamb = 0.0, dib = 0.0, lvb = 0.0, psb = 0.0, xsb = 0.0;
  double* UKb = left ? ULb : URb;
  double* FKb = left ? FLb : FRb;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    FKb[k] += Fsb[k];
    lamb = fma(Fsb[k], Num[k] * di - K.U[k], lamb);
    const double Usb = lam * Fsb[k];
    UKb[k] -= Usb;
    dib = fma(Usb, Num[k], dib);
    const double Nb = Usb * di;
    UKb[k] = fma(Nb, lv, UKb[k]);
    lvb = fma(Nb, K.U[k], lvb);
    if (k == m) {
      psb += Nb;
      PKb -= Nb;
    }
    if (k == 4) {
      psb = fma(Nb, xs, psb);
      xsb = fma(Nb, ps, xsb);
      PKb = fma(-Nb, v, PKb);
      vKb = fma(-Nb, P, vKb);
    }
  }
  // di = 1/(lam - xs)
  lamb = fma(-dib * di, di, lamb);
  xsb = fma(dib * di, di, xsb);
  lamb += lvb;
  vKb -= lvb;
  // ps = Fmh - xs FEh
  double Fmhb = psb, FEhb = -psb * xs;
  xsb = fma(-psb, FEh, xsb);
  // xs = 2 mh / (b + sq), sq = sqrt(b^2 - 4 FEh mh)
  double mhb = 2.0 * xsb * id1;
  const double d1b = -xsb * xs * id1;
  double bb = d1b;
  const double discb = 0.5 * d1b / sq;
  bb = fma(2.0 * b, discb, bb);
  FEhb = fma(-4.0 * mh, discb, FEhb);
  mhb = fma(-4.0 * FEh, discb, mhb);
  const double Ehb = bb;
  Fmhb += bb;
  // the HLL averages of components 0, m, 4
  double Uhb[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, Fhb[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  Uhb[0] = Ehb;
  Uhb[4] = Ehb;
  Uhb[m] += mhb;
  Fhb[0] = FEhb;
  Fhb[4] = FEhb;
  Fhb[m] += Fmhb;
  double idlb = 0.0;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    if (c != 0 && c != 4 && c != m) continue;
    const double gu = Uhb[c] * idl, gf = Fhb[c] * idl;
    URb[c] = fma(gu, lamR, URb[c]);
    ULb[c] = fma(-gu, lamL, ULb[c]);
    FRb[c] -= gu;
    FLb[c] += gu;
    lamRb = fma(gu, R.U[c], lamRb);
    lamLb = fma(-gu, L.U[c], lamLb);
    const double dU = R.U[c] - L.U[c];
    FLb[c] = fma(gf, lamR, FLb[c]);
    FRb[c] = fma(-gf, lamL, FRb[c]);
    URb[c] = fma(gf, lrl, URb[c]);
    ULb[c] = fma(-gf, lrl, ULb[c]);
    lamRb = fma(gf, fma(lamL, dU, L.F[c]), lamRb);
    lamLb = fma(gf, fma(lamR, dU, -R.F[c]), lamLb);
    idlb = fma(Uhb[c], NU(c), fma(Fhb[c], NF(c), idlb));
  }
  // idl = 1/(lamR - lamL)
  lamRb = fma(-idlb * idl, idl, lamRb);
  lamLb = fma(idlb * idl, idl, lamLb);
  (left ? lamLb : lamRb) += lamb;
}

// Reverse of numerical_flux<D>: Fsb -> adjoints of the left and right face primitives.
template <int D>
__device__ __forceinline__ void numerical_flux_vjp(const Params& p, const double WL[5],
                                                   const double WR[5], const double* tL,
                                                   const double* tR, long long ts,
                                                   const double Fsb[5], double WLb[5],
                                                   double WRb[5]) {
  FaceFwd L, R;
  face_fwd<D>(p, WL, tL, ts, L);
  face_fwd<D>(p, WR, tR, ts, R);
  // the forward's selections, on the bit patterns (integer pipe) as min_bits / max_bits take them
  const bool selL_from_L = order_key(L.lm) <= order_key(R.lm);  // lambda_L = min(lm_L, lm_R)
  const bool selR_from_L = order_key(L.lp) >= order_key(R.lp);  // lambda_R = max(lp_L, lp_R)
  const double lamL = selL_from_L ? L.lm : R.lm, lamR = selR_from_L ? L.lp : R.lp;
  double lamLb = 0.0, lamRb = 0.0;
  auto wavespeed_adjoints = [&](double& lmLb, double& lpLb, double& lmRb, double& lpRb) {
    lmLb = selL_from_L ? lamLb : 0.0;
    lmRb = selL_from_L ? 0.0 : lamLb;
    lpLb = selR_from_L ? lamRb : 0.0;
    lpRb = selR_from_L ? 0.0 : lamRb;
  };
  double lmLb, lpLb, lmRb, lpRb;
  if (p.flux == 2) {
    double FLb[5], FRb[5], ULb[5], URb[5];
    double vLb = 0.0, PLb = 0.0, vRb = 0.0, PRb = 0.0;  // direct uses of v_D and P
    double vKb, PKb;
    bool left;
    hllc_flux_vjp<D>(L, R, lamL, lamR, Fsb, FLb, FRb, ULb, URb, lamLb, lamRb, vKb, PKb, left);
    (left ? vLb : vRb) = vKb;
    (left ? PLb : PRb) = PKb;
    wavespeed_adjoints(lmLb, lpLb, lmRb, lpRb);
    face_rev<D>(p, L, FLb, ULb, lmLb, lpLb, WLb, vLb, PLb);
    face_rev<D>(p, R, FRb, URb, lmRb, lpRb, WRb, vRb, PRb);
    return;
  }
  // LLF and HLL: F_L_bar = aL Fsb, U_L_bar = bL Fsb, and likewise on the right
  double aL, bL, aR, bR;
  if (p.flux == 1) {
    const bool actL = dbits(lamL) < 0, actR = pos_bits(lamR);  // as the forward's S_L, S_R
    const double sL = actL ? lamL : 0.0, sR = actR ? lamR : 0.0;
    const double den = sR - sL;
    if ((dbits(den) << 1) == 0) {  // den = +-0
      aL = aR = 0.5;
      bL = bR = 0.0;
    } else {
      // F* = (sR F_L - sL F_R + sL sR dU) / den, den = sR - sL, so
      // dF*/dsR = sL (dF - sL dU) / den^2 and dF*/dsL = -sR (dF - sR dU) / den^2
      // (dU = U_R - U_L, dF = F_R - F_L; differences unfused so that they round alike however
      // their operands were formed)
      const double id = recip_nr(den);
      const double sRid = sR * id, sLid = sL * id, sLsRid = sL * sRid;
      double gF = 0.0, gU = 0.0;  // Fsb . dF and Fsb . dU
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        gF = fma(Fsb[v], __dsub_rn(R.F[v], L.F[v]), gF);
        gU = fma(Fsb[v], __dsub_rn(R.U[v], L.U[v]), gU);
      }
      aL = sRid;
      bL = -sLsRid;
      aR = -sLid;
      bR = sLsRid;
      const double sRb = sLid * id * fma(-sL, gU, gF), sLb = -sRid * id * fma(-sR, gU, gF);
      lamLb = actL ? sLb : 0.0;
      lamRb = actR ? sRb : 0.0;
    }
  } else {
    // a = max(|lambda_L|, |lambda_R|), chosen on the bit patterns as the forward chooses it
    const bool useL = order_key(abs_bits(lamL)) >= order_key(abs_bits(lamR));
    const double a = useL ? abs_bits(lamL) : abs_bits(lamR);
    double gU = 0.0;
#pragma unroll
    for (int v = 0; v < 5; ++v) gU = fma(Fsb[v], __dsub_rn(R.U[v], L.U[v]), gU);
    const double ab = -0.5 * gU;
    aL = aR = 0.5;
    bL = 0.5 * a;
    bR = -0.5 * a;
    if (useL)
      lamLb = dbits(lamL) >= 0 ? ab : -ab;
    else
      lamRb = dbits(lamR) >= 0 ? ab : -ab;
  }
  wavespeed_adjoints(lmLb, lpLb, lmRb, lpRb);
  face_rev_scaled<D>(p, L, Fsb, aL, bL, lmLb, lpLb, WLb);
  face_rev_scaled<D>(p, R, Fsb, aR, bR, lmRb, lpRb, WRb);
}

// ---------------------------------------------------------------------------------------
// Face kernel of the VJP: adjoints of the face traces, TrB in the layout of Tr.
// ---------------------------------------------------------------------------------------
template <int DIM, int N, int D>
__device__ __forceinline__ void face_vjp_point(const Params& p, const double* __restrict__ Tr,
                                               const double* __restrict__ tape,
                                               const double* __restrict__ Rb,
                                               double* __restrict__ TrB, long long k) {
  constexpr int Nn = Shape<DIM, N>::Nn, Nt = Shape<DIM, N>::Nt;
  const long long nf = p.nface[D];
  if (k >= nf * Nt) return;
  const long long f = k / Nt;
  const int t = (int)(k - f * Nt);
  long long eL, eR;
  if (f < p.E) {
    eR = f;
    const long long c = elem_coord(p, f, D);
    if (c > 0)
      eL = f - p.stride[D];
    else if (p.bc[D][0] == 0)
      eL = f + (p.n[D] - 1) * p.stride[D];
    else
      eL = -1;
  } else {
    const long long j = f - p.E;
    if (D == 0) {
      eL = (p.n[0] - 1) + p.n[0] * j;
    } else if (D == 1) {
      const unsigned q0 = fdiv((unsigned)j, p.ndiv[0]);
      eL = (long long)((unsigned)j - q0 * (unsigned)p.n[0]) +
           p.n[0] * ((p.n[1] - 1) + p.n[1] * (long long)q0);
    } else {
      eL = j + p.n[0] * p.n[1] * (p.n[2] - 1);
    }
    eR = -1;
  }
  const long long tot = p.E * Nn;
  const long long side_stride = 5 * p.E * Nt;
  const double* trL = Tr + ((long long)D * 2 + 1) * side_stride;
  const double* trR = Tr + ((long long)D * 2 + 0) * side_stride;
  double WL[5], WR[5], Fsb[5];
  if (eL >= 0) {
#pragma unroll
    for (int v = 0; v < 5; ++v) WL[v] = trL[(v * p.E + eL) * Nt + t];
  }
  if (eR >= 0) {
#pragma unroll
    for (int v = 0; v < 5; ++v) WR[v] = trR[(v * p.E + eR) * Nt + t];
  }
  // ghosts: Dirichlet = fixed outer state; outflow = the interior trace; reflecting wall =
  // the interior trace with its normal velocity reversed
  if (eL < 0) {
#pragma unroll
    for (int v = 0; v < 5; ++v) WL[v] = (p.bc[D][0] == 1) ? p.ghost[D][0][v] : WR[v];
    if (p.bc[D][0] == 3) WL[1 + D] = -WL[1 + D];
  }
  if (eR < 0) {
#pragma unroll
    for (int v = 0; v < 5; ++v) WR[v] = (p.bc[D][1] == 1) ? p.ghost[D][1][v] : WL[v];
    if (p.bc[D][1] == 3) WR[1 + D] = -WR[1 + D];
  }
  // transposed lift: R_left -= s l+ F*, R_right += s l- F* (s = 2/dx_D, in the tables)
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < N; ++a) {
      const int node = line_node<DIM, N>(D, t, a);
      if (eR >= 0) acc = fma(p.slm[D][a], Rb[v * tot + eR * Nn + node], acc);
      if (eL >= 0) acc = fma(-p.slp[D][a], Rb[v * tot + eL * Nn + node], acc);
    }
    Fsb[v] = acc;
  }
  double WLb[5], WRb[5];
  if (tape) {
    const long long ts = nf * Nt;
    const double* tp = tape + tape_base(p, D) + k;
    numerical_flux_vjp<D>(p, WL, WR, tp, tp + kFaceTape * ts, ts, Fsb, WLb, WRb);
  } else {
    numerical_flux_vjp<D>(p, WL, WR, nullptr, nullptr, 0, Fsb, WLb, WRb);
  }
  // ghost states: Dirichlet ghosts are constant, outflow ghosts copy the interior trace,
  // reflecting ghosts copy it with the normal velocity reversed
  if (eL < 0 && p.bc[D][0] >= 2) {
    if (p.bc[D][0] == 3) WLb[1 + D] = -WLb[1 + D];
#pragma unroll
    for (int v = 0; v < 5; ++v) WRb[v] += WLb[v];
  }
  if (eR < 0 && p.bc[D][1] >= 2) {
    if (p.bc[D][1] == 3) WRb[1 + D] = -WRb[1 + D];
#pragma unroll
    for (int v = 0; v < 5; ++v) WLb[v] += WRb[v];
  }
  double* tbL = TrB + ((long long)D * 2 + 1) * side_stride;
  double* tbR = TrB + ((long long)D * 2 + 0) * side_stride;
  if (eL >= 0)
#pragma unroll
    for (int v = 0; v < 5; ++v) tbL[(v * p.E + eL) * Nt + t] = WLb[v];
  if (eR >= 0)
#pragma unroll
    for (int v = 0; v < 5; ++v) tbR[(v * p.E + eR) * Nt + t] = WRb[v];
}

template <int DIM, int N>
__global__ void __launch_bounds__(128) face_vjp_kernel(Params p, const double* __restrict__ Tr,
                                                       const double* __restrict__ tape,
                                                       const double* __restrict__ Rb,
                                                       double* __restrict__ TrB) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.y == 0) face_vjp_point<DIM, N, 0>(p, Tr, tape, Rb, TrB, k);
  if (DIM > 1 && blockIdx.y == 1) face_vjp_point<DIM, N, (DIM > 1 ? 1 : 0)>(p, Tr, tape, Rb, TrB, k);
  if (DIM > 2 && blockIdx.y == 2) face_vjp_point<DIM, N, (DIM > 2 ? 2 : 0)>(p, Tr, tape, Rb, TrB, k);
}

// ---------------------------------------------------------------------------------------
// Nodal adjoint: U_bar = (dF/dU|_W)^T F_bar + (dU/dW)^{-T} W_bar, W = (rho, v, P).
// ---------------------------------------------------------------------------------------

// Given the node state (U, rho, u, P), the adjoint of its nodal fluxes (Fb[d][5]) and of its
// interpolated primitive (Wub = adjoint of (rho, u, P)), return U_bar.
template <int DIM>
__device__ __forceinline__ void node_adjoint(const Params& p, const double U[5], const double Wu[5],
                                             double lor, double ilor, const double Fb[DIM][5],
                                             const double Wub[5], double Ub[5]) {
  const double rho = Wu[0], P = Wu[4];
  const double u2 = fma(Wu[1], Wu[1], fma(Wu[2], Wu[2], Wu[3] * Wu[3]));
  const double q = 1.0 + u2;
  const double v[3] = {Wu[1] * ilor, Wu[2] * ilor, Wu[3] * ilor};
  double Wb[5] = {Wub[0], 0.0, 0.0, 0.0, Wub[4]};  // adjoint of (rho, v, P)
  // u = gamma v: du/dv = gamma I + gamma^3 v v^T (symmetric)
  const double vu = v[0] * Wub[1] + v[1] * Wub[2] + v[2] * Wub[3];
  const double l3vu = lor * q * vu;
#pragma unroll
  for (int k = 0; k < 3; ++k) Wb[1 + k] = fma(lor, Wub[1 + k], l3vu * v[k]);
  // fluxes F^d = (D v_d, S v_d + P e_d, (tau + P) v_d)
#pragma unroll
  for (int k = 0; k < 5; ++k) Ub[k] = 0.0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const double vd = v[d];
#pragma unroll
    for (int k = 0; k < 5; ++k) Ub[k] = fma(vd, Fb[d][k], Ub[k]);
    Wb[1 + d] += Fb[d][0] * U[0] + Fb[d][1] * U[1] + Fb[d][2] * U[2] + Fb[d][3] * U[3] +
                 Fb[d][4] * (U[4] + P);
    Wb[4] += fma(Fb[d][4], vd, Fb[d][1 + d]);
  }
  double x[5];
  c2p_adjoint(p, rho, v, P, lor, ilor, q, u2, Wb, x);
#pragma unroll
  for (int k = 0; k < 5; ++k) Ub[k] += x[k];
}

// With Ukb null: Ub = U_bar.  Otherwise the stage combination of the SSP-RK reverse sweep is
// fused in: Unb += a_n R_bar and Ukb += b_k (R_bar + dt U_bar) (Unb and Ukb may be the same).
// Three resident 256-thread blocks per SM in 1D and 2D (at most 85 registers per thread); in 3D
// that bound would spill, and two are asked for.
template <int DIM, int N>
__global__ void __launch_bounds__(Shape<DIM, N>::BLOCK, DIM == 3 ? 2 : 3)
    node_vjp_kernel(Params p, const double* __restrict__ U, const double* __restrict__ Wst,
                    const unsigned char* __restrict__ guard, const double* __restrict__ Rb,
                    const double* __restrict__ TrB, double* __restrict__ Ub, double* Unb,
                    double* Ukb, double a_n, double b_k, double dt) {
  using S = Shape<DIM, N>;
  constexpr int Nn = S::Nn, Nt = S::Nt, BLOCK = S::BLOCK;
  // The transposed volume term runs in FP32 head-and-tail pair arithmetic (products by Dekker's
  // two-product, sums by Knuth's two-sum), within about 2^-44 of the FP64 contraction relative
  // to its terms, on the FP32 pipe instead of the FP64 one.  FP32 spans far fewer binades than
  // FP64: when every |R_bar| of the block is zero or inside [2^-100, 2^100] the pairs hold it in
  // full; otherwise (a block-uniform branch) each element's R_bar is first scaled by the power
  // of two that brings its largest component into [1, 2) (exact), and the sums are scaled back
  // in FP64, where components below 2^-100 of the element's largest lose digits, a negligible
  // share of every sum they enter.
  __shared__ F32Pair shR[5][BLOCK];
  __shared__ F32Pair shD[DIM][N * N];  // (2/dx_d) Dhat per axis
  __shared__ int shX[S::EPB];          // largest biased FP64 exponent of R_bar per element
  const int tid = threadIdx.x;
  if (tid < DIM * N * N)
    shD[tid / (N * N)][tid % (N * N)] = f32_pair(p.inv_half_dx[tid / (N * N)] * p.Dhat[tid % (N * N)]);
  if (tid < S::EPB) shX[tid] = 0;
  const int le = tid / Nn, li = tid - le * Nn;
  const long long e = (long long)blockIdx.x * S::EPB + le;
  const bool valid = e < p.E;
  const long long tot = p.E * Nn;
  const long long g = e * Nn + li;
  double y[5];  // this node's R_bar, for the fused stage combination
  int ex = 0;
  bool inside = true;
  if (valid) {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      y[v] = Rb[v * tot + g];
      const int b = (__double2hiint(y[v]) >> 20) & 0x7ff;
      ex = max(ex, b);
      inside = inside && ((__double_as_longlong(y[v]) << 1) == 0 || (b >= 1023 - 100 && b <= 1023 + 100));
    }
  }
  const bool whole = __syncthreads_and(inside);  // also orders the tables' set-up
  int X = 1023;
  if (!whole) {
    if (valid && ex > 0) atomicMax(&shX[le], ex);
    __syncthreads();
    X = valid ? shX[le] : 1023;
  }
  if (valid) {
#pragma unroll
    for (int v = 0; v < 5; ++v) shR[v][tid] = f32_pair(whole ? y[v] : scale_pow2(y[v], 1023 - X));
  }
  __syncthreads();
  if (!valid) return;
  int ijk[3];
  node_ijk<DIM, N>(li, ijk);
  // transposed volume term: F_bar^d[a] = (2/dx_d) sum_i Dhat[i][a] R_bar[i]
  double Fb[DIM][5];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int ns = node_stride<N>(d);
    const int base = tid - ijk[d] * ns;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      F32Pair acc = mul_pair(shD[d][ijk[d]], shR[v][base]);
#pragma unroll
      for (int i = 1; i < N; ++i) acc = add_pair(acc, mul_pair(shD[d][i * N + ijk[d]], shR[v][base + i * ns]));
      Fb[d][v] = f32_to_f64_bits(acc.hi) + f32_to_f64_bits(acc.lo);
    }
  }
  if (!whole) {
#pragma unroll
    for (int d = 0; d < DIM; ++d)
#pragma unroll
      for (int v = 0; v < 5; ++v) Fb[d][v] = scale_pow2(Fb[d][v], X - 1023);
  }
  // transposed trace extrapolation; a guarded face point took the end node's primitive
  double Wub[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int t = tan_index<DIM, N>(ijk, d);
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const bool guarded = guard[e * S::NFP + (d * 2 + side) * Nt + t] != 0;
      const double w = guarded ? ((ijk[d] == (side ? N - 1 : 0)) ? 1.0 : 0.0)
                               : (side ? p.ep[ijk[d]] : p.em[ijk[d]]);
      if ((dbits(w) << 1) != 0) {  // w != 0, on the integer pipe
#pragma unroll
        for (int v = 0; v < 5; ++v)
          Wub[v] = fma(w, TrB[((((long long)d * 2 + side) * 5 + v) * p.E + e) * Nt + t], Wub[v]);
      }
    }
  }
  double u[5], Wu[5], out[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    u[v] = U[v * tot + g];
    Wu[v] = Wst[v * tot + g];
  }
  // gamma and 1/gamma as the forward con2prim found them
  node_adjoint<DIM>(p, u, Wu, Wst[5 * tot + g], Wst[6 * tot + g], Fb, Wub, out);
  if (!Ukb) {
#pragma unroll
    for (int v = 0; v < 5; ++v) Ub[v * tot + g] = out[v];
  } else {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      if (a_n != 0.0) Unb[v * tot + g] += a_n * y[v];
      Ukb[v * tot + g] += b_k * fma(dt, out[v], y[v]);  // re-read: Ukb may be Unb
    }
  }
}

// ---------------------------------------------------------------------------------------
// Physicality operator with frozen factors: U~_i = s U_i + (1 - s) mean(U), so
// U_bar_i = s Ut_bar_i + (1 - s) (w_i / sum w) sum_j Ut_bar_j.
// ---------------------------------------------------------------------------------------
template <int DIM, int N>
__global__ void __launch_bounds__(Shape<DIM, N>::BLOCK)
    enforce_vjp_kernel(Params p, const double* __restrict__ s, const double* __restrict__ Tb,
                       double* __restrict__ Ub) {
  using S = Shape<DIM, N>;
  constexpr int Nn = S::Nn;
  __shared__ double sh[5][S::BLOCK];
  __shared__ double sum[S::EPB][5];
  const int tid = threadIdx.x;
  const int le = tid / Nn, li = tid - le * Nn;
  const long long e = (long long)blockIdx.x * S::EPB + le;
  const bool valid = e < p.E;
  const long long tot = p.E * Nn;
  const long long g = e * Nn + li;
  double t[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const double se = valid ? s[e] : 1.0;
  if (valid)
#pragma unroll
    for (int v = 0; v < 5; ++v) t[v] = Tb[v * tot + g];
  const bool any = __syncthreads_or(valid && se != 1.0);
  if (any) {
#pragma unroll
    for (int v = 0; v < 5; ++v) sh[v][tid] = t[v];
    __syncthreads();
    if (valid && li == 0 && se != 1.0) {
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        double acc = 0.0;
        for (int j = 0; j < Nn; ++j) acc += sh[v][le * Nn + j];
        sum[le][v] = acc;
      }
    }
    __syncthreads();
  }
  if (!valid) return;
  if (se == 1.0) {
#pragma unroll
    for (int v = 0; v < 5; ++v) Ub[v * tot + g] = t[v];
    return;
  }
  int ijk[3];
  node_ijk<DIM, N>(li, ijk);
  double wi = 1.0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) wi *= p.w[ijk[d]];
  const double c = (1.0 - se) * wi / p.wsum;
#pragma unroll
  for (int v = 0; v < 5; ++v) Ub[v * tot + g] = se * t[v] + c * sum[le][v];
}

}  // namespace dgsrhd
