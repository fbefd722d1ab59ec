// Launch parameters shared by the host API and the kernels (passed by value).
#pragma once

#include <stdint.h>

namespace dgsrhd {

constexpr int kMaxN = 5;  // degree <= 4
// Values per face state that the forward sweep can save for the reverse one: the roots and
// reciprocals 1/gamma, 1/sigma, 1/Z, 1/(gamma + 1), 1/(A + B), 1/r (the first six), then u^2,
// gamma, sigma, A, B, K, rho (h - 1), the conserved state U[5], r, the wavespeeds lambda-+ and
// the physical flux F[5] along the face normal.
constexpr int kFaceTape = 26;
// Planes of the saved nodal primitive: (rho, u_x, u_y, u_z, P, gamma, 1/gamma).
constexpr int kNodePrim = 7;
constexpr int kFaceTapeRecips = 6;

// Indices into the device counter array (unsigned long long).
enum StatSlot {
  kStatC2pCalls = 0,
  kStatItersTotal,
  kStatItersMax,
  kStatNonConv,
  kStatInvalid,
  kStatFaceGuard,
  kStatEnforced,
  kStatMeanBad,
  kStatLimited,
  kStatCount
};

// Division of a 32-bit index x by an invariant divisor d >= 1 without an integer division
// instruction sequence: q = umulhi(x, m) >> s with s = floor(log2 d) and m = ceil(2^(32+s) / d)
// (m = 0 when d is a power of two: q = x >> s).  Exact for x < 2^31: writing
// m = 2^(32+s)/d + eps with 0 <= eps < 1, x m / 2^(32+s) = x/d + delta with
// 0 <= delta < 2^31 / 2^(32+s) = 2^(-1-s) < 1/d, which cannot carry x/d past the next integer
// (the method of Granlund & Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994).  Element and face indices stay below 2^31 because a
// configuration has fewer than 2^30 elements.
struct FastDiv {
  unsigned m, s;
};

struct Params {
  int dim, N, Nn, Nt;        // nodes per axis, per element (N^dim), per face (N^(dim-1))
  long long n[3];            // elements per axis (1 for unused axes)
  long long stride[3];       // element index stride per axis: 1, n0, n0 n1
  FastDiv ndiv[3], sdiv[3];  // dividers for n[d] and stride[d]
  long long E;               // elements
  long long nface[3];        // faces per axis: E (+ E/n_d boundary faces if not periodic)
  long long fs_off[3];       // offset of axis d in the face-flux buffer
  double inv_half_dx[3];     // 2 / dx_d
  int eos;                   // 0 ideal, 1 Taub-Matthews
  double gamma_ad, alpha;    // Gamma, Gamma / (Gamma - 1)
  // constants of the ideal EOS formed once on the host: Gamma - 1, (Gamma - 1)^2, -2 Gamma,
  // -2 Gamma (Gamma - 1), Gamma^2, 2 (Gamma - 1), alpha - Gamma
  double gm1, gm1sq, m2G, m2Ggm1, G2, tgm1, amG;
  int c2p;                   // 0 closed form, 1 iterative (resolved)
  int max_iter;
  double c2p_rtol;           // > 0: the iterative solvers also stop at this relative step
  int flux;                  // 0 LLF, 1 HLL
  int bc[3][2];              // 0 periodic, 1 Dirichlet, 2 outflow
  double ghost[3][2][5];     // Dirichlet ghost as (rho, u, P)
  // basis tables (Gauss-Legendre nodal Lagrange basis on [-1, 1])
  double w[kMaxN];           // quadrature weights
  double Dhat[kMaxN * kMaxN];// Dhat[i*N + a] = w_a phi_i'(x_a) / w_i
  double em[kMaxN], ep[kMaxN];   // phi_i(-1), phi_i(+1)
  double lm[kMaxN], lp[kMaxN];   // phi_i(-1)/w_i, phi_i(+1)/w_i
  double slm[3][kMaxN], slp[3][kMaxN];  // (2/dx_d) lm, (2/dx_d) lp: the transposed lift per axis
  double wsum;               // sum of tensor weights = 2^dim
  unsigned long long* stats; // device counters [kStatCount]
  int enforce_faces;         // physicality operator over the nodes and the face points
  int limiter;               // 1: scaling limiter after every stage
  double lim_alpha;          // its bound relaxation (already times h^(3/2))
};

}  // namespace dgsrhd
