// Element kernels of the nodal DG right-hand side and the SSP-RK stage (FP64 path).
//
// One RK stage is three kernels:
//   volume_kernel : per element, one thread per node.  con2prim at every node (Sec. 3), nodal
//                   fluxes (Eq. srhd_flux), the sum-factorised volume term
//                   R_vol[i] = sum_d (2/dx_d) sum_a Dhat[i_d][a] F^d[.. a ..] (Eq. quad-vol-flux at
//                   the nodes), and the primitive (rho, u, P) extrapolated to the 2 dim faces of the
//                   element, sum_i phi_i(+-1) W_i along each normal line (Sec. 2.3).
//   face_kernel   : one thread per face point; LLF/HLL flux of the two traces (Sec. 2.4), stored
//                   doubled (2 F*; the lift tables carry the 1/2).
//   update_kernel : per element, one thread per node; R = R_vol - lift of the face fluxes
//                   (Eq. quad-surface-flux), the Shu-Osher combination, and the physicality
//                   operator of Sec. 2.5.
// Face fluxes are computed once per face point and read by both neighbours.
#pragma once

#include "device_math.cuh"
#include "launch.h"

namespace dgsrhd {

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

template <int DIM, int N>
struct Shape {
  static constexpr int Nn = ipow(N, DIM);        // nodes per element
  static constexpr int Nt = ipow(N, DIM - 1);    // nodes per face
  static constexpr int EPB = Nn >= 256 ? 1 : 256 / Nn;  // elements per block
  static constexpr int BLOCK = EPB * Nn;
  static constexpr int NFP = 2 * DIM * Nt;       // face points per element
};

// node index -> (a, b, c), x fastest
template <int DIM, int N>
__device__ __forceinline__ void node_ijk(int i, int ijk[3]) {
  ijk[0] = i % N;
  ijk[1] = DIM > 1 ? (i / N) % N : 0;
  ijk[2] = DIM > 2 ? i / (N * N) : 0;
}

// stride of axis d inside the element's node index
template <int N>
__device__ __forceinline__ int node_stride(int d) {
  return d == 0 ? 1 : (d == 1 ? N : N * N);
}

// tangential index of a node on the faces normal to d (other axes in order, x fastest)
template <int DIM, int N>
__device__ __forceinline__ int tan_index(const int ijk[3], int d) {
  if (DIM == 1) return 0;
  if (DIM == 2) return d == 0 ? ijk[1] : ijk[0];
  return d == 0 ? ijk[1] + N * ijk[2] : (d == 1 ? ijk[0] + N * ijk[2] : ijk[0] + N * ijk[1]);
}

// node index of tangential point t on the line normal to d at normal coordinate a
template <int DIM, int N>
__device__ __forceinline__ int line_node(int d, int t, int a) {
  if (DIM == 1) return a;
  if (DIM == 2) return d == 0 ? a + N * t : t + N * a;
  const int t0 = t % N, t1 = t / N;
  return d == 0 ? a + N * (t0 + N * t1) : (d == 1 ? t0 + N * (a + N * t1) : t0 + N * (t1 + N * a));
}

__device__ __forceinline__ unsigned fdiv(unsigned x, FastDiv f) {
  return f.m ? __umulhi(x, f.m) >> f.s : x >> f.s;
}

__device__ __forceinline__ long long elem_coord(const Params& p, long long e, int d) {
  const unsigned q = fdiv((unsigned)e, p.sdiv[d]);
  return (long long)(q - fdiv(q, p.ndiv[d]) * (unsigned)p.n[d]);
}

// index of the face flux on the high side of element e along d
__device__ __forceinline__ long long high_face(const Params& p, long long e, int d) {
  const long long c = elem_coord(p, e, d);
  if (c < p.n[d] - 1) return e + p.stride[d];
  if (p.bc[d][1] == 0) return e - (p.n[d] - 1) * p.stride[d];
  // boundary face: enumerate the elements with c = n_d - 1 by their other coordinates
  const unsigned ue = (unsigned)e;
  long long j;
  if (d == 0) {
    j = fdiv(ue, p.ndiv[0]);
  } else if (d == 1) {
    const unsigned q0 = fdiv(ue, p.ndiv[0]);
    j = (long long)(ue - q0 * (unsigned)p.n[0]) + p.n[0] * (long long)fdiv(ue, p.sdiv[2]);
  } else {
    j = (long long)(ue - fdiv(ue, p.sdiv[2]) * (unsigned)p.stride[2]);
  }
  return p.E + j;
}

// block-level reduction of con2prim statistics into 64 slots of each counter
__device__ __forceinline__ void block_stats(const Params& p, int iters, int status, int* shred) {
  // blocks need not be a multiple of 32 threads: the last warp may be partial
  const int in_warp = min(32, (int)blockDim.x - (int)(threadIdx.x & ~31u));
  const unsigned full = in_warp == 32 ? 0xffffffffu : ((1u << in_warp) - 1u);
  unsigned it = (unsigned)iters;
  unsigned sum = __reduce_add_sync(full, it);
  unsigned mx = __reduce_max_sync(full, it);
  unsigned nc = __popc(__ballot_sync(full, status == 2));
  unsigned inv = __popc(__ballot_sync(full, status == 1));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < 4 * 32) shred[threadIdx.x] = 0;
  __syncthreads();
  if (lane == 0) {
    atomicAdd(&shred[0], (int)sum);
    atomicMax(&shred[1], (int)mx);
    atomicAdd(&shred[2], (int)nc);
    atomicAdd(&shred[3], (int)inv);
  }
  __syncthreads();
  (void)warp;
  if (threadIdx.x == 0) {
    unsigned long long* st = p.stats;
    const int slot = blockIdx.x & 63;
    if (shred[0]) atomicAdd(&st[kStatItersTotal * 64 + slot], (unsigned long long)shred[0]);
    if (shred[1]) atomicMax(&st[kStatItersMax * 64 + slot], (unsigned long long)shred[1]);
    if (shred[2]) atomicAdd(&st[kStatNonConv * 64 + slot], (unsigned long long)shred[2]);
    if (shred[3]) atomicAdd(&st[kStatInvalid * 64 + slot], (unsigned long long)shred[3]);
  }
}

// ---------------------------------------------------------------------------------------
// Volume kernel
// ---------------------------------------------------------------------------------------
template <int DIM, int N>
__global__ void __launch_bounds__(Shape<DIM, N>::BLOCK)
    volume_kernel(Params p, const double* __restrict__ U, double* __restrict__ Rvol,
                  double* __restrict__ Tr, double* __restrict__ Wout,
                  unsigned char* __restrict__ guard_out, double* __restrict__ Ucopy,
                  double rscale) {
  using S = Shape<DIM, N>;
  constexpr int Nn = S::Nn, Nt = S::Nt, BLOCK = S::BLOCK;
  __shared__ double shF[DIM][5][BLOCK];
  __shared__ double shW[5][BLOCK];
  __shared__ double shD[DIM][N * N];  // (2/dx_d) Dhat per axis, times rscale when it is nonzero
  __shared__ int shred[4 * 32];
  const int tid = threadIdx.x;
  if (tid < DIM * N * N) {
    const double c = p.inv_half_dx[tid / (N * N)] * p.Dhat[tid % (N * N)];
    shD[tid / (N * N)][tid % (N * N)] = rscale != 0.0 ? c * rscale : c;
  }
  const int le = tid / Nn, li = tid - le * Nn;
  const long long e = (long long)blockIdx.x * S::EPB + le;
  const bool valid = e < p.E;
  const long long tot = p.E * Nn;
  const long long g = e * Nn + li;

  int iters = 0, status = 0;
  if (valid) {
    double u[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = U[v * tot + g];
    if (Ucopy) {  // the input state, kept on the device (it may have been read from the host)
#pragma unroll
      for (int v = 0; v < 5; ++v) Ucopy[v * tot + g] = u[v];
    }
    Prim W;
    status = con2prim(p, u, W, iters);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      double F[5];
      phys_flux(u, W.v, W.P, d, F);
#pragma unroll
      for (int v = 0; v < 5; ++v) shF[d][v][tid] = F[v];
    }
    shW[0][tid] = W.rho;
    shW[1][tid] = W.lor * W.v[0];
    shW[2][tid] = W.lor * W.v[1];
    shW[3][tid] = W.lor * W.v[2];
    shW[4][tid] = W.P;
    if (Wout) {  // (rho, u, P, gamma, 1/gamma) kept for the vector-Jacobian product
#pragma unroll
      for (int v = 0; v < 5; ++v) Wout[v * tot + g] = shW[v][tid];
      Wout[5 * tot + g] = W.lor;
      Wout[6 * tot + g] = W.ginv;
    }
  }
  block_stats(p, iters, status, shred);  // contains __syncthreads

  if (valid) {
    int ijk[3];
    node_ijk<DIM, N>(li, ijk);
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const int ns = node_stride<N>(d);
      const int base = tid - ijk[d] * ns;
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const double c = shD[d][ijk[d] * N + a];
#pragma unroll
        for (int v = 0; v < 5; ++v) acc[v] = fma(c, shF[d][v][base + a * ns], acc[v]);
      }
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) Rvol[v * tot + g] = acc[v];

    // face traces of (rho, u, P)
    int guard = 0;
    for (int fp = li; fp < S::NFP; fp += Nn) {
      const int d = fp / (2 * Nt);
      const int side = (fp / Nt) & 1;
      const int t = fp % Nt;
      double out[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const int node = le * Nn + line_node<DIM, N>(d, t, a);
        const double c = side ? p.ep[a] : p.em[a];
#pragma unroll
        for (int v = 0; v < 5; ++v) out[v] = fma(c, shW[v][node], out[v]);
      }
      const bool guarded = !pos_bits(out[0]) || !pos_bits(out[4]);
      if (guarded) {
        const int node = le * Nn + line_node<DIM, N>(d, t, side ? N - 1 : 0);
#pragma unroll
        for (int v = 0; v < 5; ++v) out[v] = shW[v][node];
        ++guard;
      }
      // the guard decision per face point, kept with the primitives for the reverse sweep
      if (guard_out) guard_out[e * S::NFP + fp] = guarded ? 1 : 0;
#pragma unroll
      for (int v = 0; v < 5; ++v) Tr[((((long long)d * 2 + side) * 5 + v) * p.E + e) * Nt + t] = out[v];
    }
    if (guard) atomicAdd(&p.stats[kStatFaceGuard * 64 + (blockIdx.x & 63)], (unsigned long long)guard);
  }
}

// ---------------------------------------------------------------------------------------
// Face kernel: blockIdx.y = axis; each axis runs its own instantiation of the face point so
// that every index into the state is known at compile time.
// ---------------------------------------------------------------------------------------
// Face-state tape: kFaceTape values per side (left, then right) per face point, plane j of axis
// D at (fs_off[D] / 5) * 2 kFaceTape + j nface[D] Nt.
__device__ __forceinline__ long long tape_base(const Params& p, int D) {
  return (p.fs_off[D] / 5) * (2 * kFaceTape);
}

// PAIRS: store each flux as its FP32 head and tail (float2, same footprint) for the split update
template <int DIM, int N, int D, bool SAVE, bool PAIRS>
__device__ __forceinline__ void face_point(const Params& p, const double* __restrict__ Tr,
                                           double* __restrict__ Fs, double* __restrict__ tape,
                                           long long k) {
  constexpr int Nt = Shape<DIM, N>::Nt;
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
  double WL[5], WR[5];
  const long long side_stride = 5 * p.E * Nt;
  const double* trL = Tr + ((long long)D * 2 + 1) * side_stride;  // high side of the left elem
  const double* trR = Tr + ((long long)D * 2 + 0) * side_stride;  // low side of the right elem
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
  double* out = Fs + p.fs_off[D];
  if (PAIRS) {
    F32Pair Fp[5];
    numerical_flux<D, false, F32Pair>(p, WL, WR, Fp, nullptr, nullptr);  // Fp = 2 F*
    float2* outp = reinterpret_cast<float2*>(out);
#pragma unroll
    for (int v = 0; v < 5; ++v) outp[(v * nf + f) * Nt + t] = make_float2(Fp[v].hi, Fp[v].lo);
    return;
  }
  double F[5], rec[2][kFaceTape];
  numerical_flux<D, SAVE>(p, WL, WR, F, rec[0], rec[1]);  // F = 2 F*
#pragma unroll
  for (int v = 0; v < 5; ++v) out[(v * nf + f) * Nt + t] = F[v];
  if (SAVE) {
    double* tp = tape + tape_base(p, D);
#pragma unroll
    for (int j = 0; j < 2 * kFaceTape; ++j) tp[j * nf * Nt + k] = rec[j / kFaceTape][j % kFaceTape];
  }
}

// SAVE: also write the face-state tape for the reverse sweep.  PAIRS (never with SAVE): write
// the fluxes as FP32 head and tail for the split update.
template <int DIM, int N, bool SAVE, bool PAIRS = false>
__global__ void __launch_bounds__(128) face_kernel(Params p, const double* __restrict__ Tr,
                                                   double* __restrict__ Fs,
                                                   double* __restrict__ tape) {
  static_assert(!(SAVE && PAIRS), "the tape is written by the FP64 face kernel only");
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.y == 0) face_point<DIM, N, 0, SAVE, PAIRS>(p, Tr, Fs, tape, k);
  if (DIM > 1 && blockIdx.y == 1)
    face_point<DIM, N, (DIM > 1 ? 1 : 0), SAVE, PAIRS>(p, Tr, Fs, tape, k);
  if (DIM > 2 && blockIdx.y == 2)
    face_point<DIM, N, (DIM > 2 ? 2 : 0), SAVE, PAIRS>(p, Tr, Fs, tape, k);
}

// ---------------------------------------------------------------------------------------
// Physicality operator on the elements of one block (Sec. 2.5).  u holds this thread's node
// state; on return it holds the smoothed state.  Every thread of the block must call it.  With
// p.enforce_faces the element's points are its nodes and the face points of its conserved
// polynomial (sum_a phi_a(-+1) U_a along each normal line): smoothing the nodes by s smooths
// every face point by the same s (the basis reproduces constants), so the minimum over both
// leaves the polynomial admissible at the faces too.
// ---------------------------------------------------------------------------------------
template <int DIM, int N, int BLOCKSZ = Shape<DIM, N>::BLOCK>
struct EnforceShared {
  double a[5][BLOCKSZ];
  double u[5][BLOCKSZ];  // the nodal states themselves (face-point variant)
  double mean[Shape<DIM, N>::EPB][5];
  double s[Shape<DIM, N>::EPB];
  int flag[Shape<DIM, N>::EPB];
};

// Largest factor s_i in [0, 1] for one point with conserved state X and admissible element
// mean m: the two stages of Sec. 2.5 (Eqs. first_stage_positivity, first_stage_smoothed_state,
// second_stage_quatratic with the coefficients of Eq. second_stage_coefficients in the stored
// variables, the root of Eq. second_stage_solution as 2 c0 / (-b + sqrt(b^2 - 4 a c0)) clamped to
// [0, 1]).
__device__ __forceinline__ double point_factor(const double X[5], const double m[5]) {
  const double Db = m[0], taub = m[4], Eb = m[4] + m[0];
  // stage 1: largest factors keeping D and E positive (Eq. first_stage_positivity)
  const double sD = X[0] >= 0.0 ? 1.0 : Db / (Db - X[0]);
  const double Ei = X[4] + X[0];
  const double sE = Ei >= 0.0 ? 1.0 : Eb / (Eb - Ei);
  const double s1 = fmin(sD, sE);
  double U1[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) U1[v] = s1 * X[v] + (1.0 - s1) * m[v];
  if (admissible(U1)) return s1;
  // stage 2 quadratic a s^2 + b s + c0 > 0 in the stored variables (Eq.
  // second_stage_coefficients with E = tau + D)
  const double dD = U1[0] - Db, dtau = U1[4] - taub;
  const double d1 = U1[1] - m[1], d2 = U1[2] - m[2], d3 = U1[3] - m[3];
  const double qa = dtau * (dtau + 2.0 * dD) - (d1 * d1 + d2 * d2 + d3 * d3);
  const double qb = 2.0 * (taub * (dtau + dD) + Db * dtau - (m[1] * d1 + m[2] * d2 + m[3] * d3));
  const double qc = taub * (taub + 2.0 * Db) - (m[1] * m[1] + m[2] * m[2] + m[3] * m[3]);
  const double den = -qb + sqrt(qb * qb - 4.0 * qa * qc);
  double s2 = den > 0.0 ? 2.0 * qc / den : 1.0;
  s2 = fmin(fmax(s2, 0.0), 1.0);
  return s1 * s2;
}

// Conserved state of the block-local element le at its face point fp (= (d 2 + side) Nt + t),
// from the nodal states in shared memory.
template <int DIM, int N, int BLOCKSZ>
__device__ __forceinline__ void face_point_state(const Params& p, const double (&su)[5][BLOCKSZ],
                                                 int le, int fp, double out[5]) {
  constexpr int Nn = Shape<DIM, N>::Nn, Nt = Shape<DIM, N>::Nt;
  const int d = fp / (2 * Nt), side = (fp / Nt) & 1, t = fp % Nt;
#pragma unroll
  for (int v = 0; v < 5; ++v) out[v] = 0.0;
#pragma unroll
  for (int a = 0; a < N; ++a) {
    const int node = le * Nn + line_node<DIM, N>(d, t, a);
    const double c = side ? p.ep[a] : p.em[a];
#pragma unroll
    for (int v = 0; v < 5; ++v) out[v] = fma(c, su[v][node], out[v]);
  }
}

// FACES: the face-point variant (p.enforce_faces), a template parameter so that the nodal
// operator's kernels carry none of its registers.
template <bool FACES, int DIM, int N, int BLOCKSZ>
__device__ __forceinline__ void enforce_block(const Params& p, double u[5], bool valid, int le,
                                              int li, long long e, double* s_out,
                                              EnforceShared<DIM, N, BLOCKSZ>& sh) {
  constexpr int Nn = Shape<DIM, N>::Nn, NFP = Shape<DIM, N>::NFP;
  const int tid = threadIdx.x;
  bool bad = valid && !admissible_screen(u);
  if (FACES) {
#pragma unroll
    for (int v = 0; v < 5; ++v) sh.u[v][tid] = valid ? u[v] : 0.0;
    __syncthreads();
    if (valid) {
      for (int fp = li; fp < NFP; fp += Nn) {
        double X[5];
        face_point_state<DIM, N, BLOCKSZ>(p, sh.u, le, fp, X);
        if (!admissible_screen(X)) bad = true;
      }
    }
  }
  if (!__syncthreads_or(bad)) {
    if (valid && li == 0 && s_out) s_out[e] = 1.0;
    return;
  }
  if (li == 0) sh.flag[le] = 0;
  __syncthreads();
  if (bad) sh.flag[le] = 1;
  int ijk[3];
  node_ijk<DIM, N>(li, ijk);
  double wi = 1.0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) wi *= p.w[ijk[d]];
#pragma unroll
  for (int v = 0; v < 5; ++v) sh.a[v][tid] = valid ? wi * u[v] : 0.0;
  __syncthreads();
  if (li == 0 && valid && sh.flag[le]) {
    double m[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int j = 0; j < Nn; ++j)
#pragma unroll
      for (int v = 0; v < 5; ++v) m[v] += sh.a[v][le * Nn + j];
#pragma unroll
    for (int v = 0; v < 5; ++v) sh.mean[le][v] = m[v] / p.wsum;
    sh.flag[le] = admissible(sh.mean[le]) ? 2 : 3;
  }
  __syncthreads();
  const int fl = valid ? sh.flag[le] : 0;
  double si = 1.0;
  if (fl == 2) {
    si = point_factor(u, sh.mean[le]);
    if (FACES) {
      for (int fp = li; fp < NFP; fp += Nn) {
        double X[5];
        face_point_state<DIM, N, BLOCKSZ>(p, sh.u, le, fp, X);
        si = fmin(si, point_factor(X, sh.mean[le]));
      }
    }
  }
  sh.a[0][tid] = si;
  __syncthreads();
  if (li == 0 && valid) {
    double s = 1.0;
    if (fl == 2) {
      for (int j = 0; j < Nn; ++j) s = fmin(s, sh.a[0][le * Nn + j]);
      s *= (1.0 - 1e-12);
      atomicAdd(&p.stats[kStatEnforced * 64 + (blockIdx.x & 63)], 1ull);
    } else if (fl == 3) {
      atomicAdd(&p.stats[kStatMeanBad * 64 + (blockIdx.x & 63)], 1ull);
    }
    sh.s[le] = s;
    if (s_out) s_out[e] = s;
  }
  __syncthreads();
  if (fl == 2) {
    const double s = sh.s[le];
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = s * u[v] + (1.0 - s) * sh.mean[le][v];
  }
}

// ---------------------------------------------------------------------------------------
// Update kernel: R = R_vol - lift; mode 0 writes R, mode 1 writes the RK stage
// Uout = a_n Un + b_k (Uk + dt R) followed (if enforce) by the physicality operator.  With
// rscale nonzero (mode 1 only), R_vol arrives times rscale = b_k dt and the lift is scaled the
// same way, so the stage is a_n Un + b_k Uk + R: one fused multiply-add per variable fewer.
// Uout may alias Uk or Un (each thread reads its own node before the block writes).
// ---------------------------------------------------------------------------------------
template <int DIM, int N, bool FACES>
__global__ void __launch_bounds__(Shape<DIM, N>::BLOCK)
    update_kernel(Params p, const double* __restrict__ Rvol, const double* __restrict__ Fs,
                  const double* Un, const double* Uk, double* Uout, double a_n, double b_k,
                  double dt, int mode, int enforce, double* __restrict__ s_out, double rscale) {
  using S = Shape<DIM, N>;
  constexpr int Nn = S::Nn;
  __shared__ EnforceShared<DIM, N> sh;
  // (2/dx_d) phi_i(-+1)/w_i per axis, halved (the face kernel stores 2 F*), times rscale when
  // it is nonzero
  __shared__ double shl[DIM][2][N];
  const int tid = threadIdx.x;
  if (tid < DIM * N) {
    const int d = tid / N, i = tid % N;
    const double cm = 0.5 * p.inv_half_dx[d] * p.lm[i], cp = 0.5 * p.inv_half_dx[d] * p.lp[i];
    shl[d][0][i] = rscale != 0.0 ? cm * rscale : cm;
    shl[d][1][i] = rscale != 0.0 ? cp * rscale : cp;
  }
  __syncthreads();
  const int le = tid / Nn, li = tid - le * Nn;
  const long long e = (long long)blockIdx.x * S::EPB + le;
  const bool valid = e < p.E;
  const long long tot = p.E * Nn;
  const long long g = e * Nn + li;
  double u[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (valid) {
    int ijk[3];
    node_ijk<DIM, N>(li, ijk);
    double R[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) R[v] = Rvol[v * tot + g];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const int t = tan_index<DIM, N>(ijk, d);
      const long long nf = p.nface[d];
      const double* fs = Fs + p.fs_off[d];
      const long long flo = e, fhi = high_face(p, e, d);
      const double cp = shl[d][1][ijk[d]];
      const double cm = shl[d][0][ijk[d]];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double Fhi = fs[(v * nf + fhi) * S::Nt + t];
        const double Flo = fs[(v * nf + flo) * S::Nt + t];
        R[v] = R[v] - cp * Fhi + cm * Flo;
      }
    }
    if (mode == 0) {
#pragma unroll
      for (int v = 0; v < 5; ++v) Uout[v * tot + g] = R[v];
    } else if ((dbits(rscale) << 1) != 0) {  // R = b_k dt (R_vol - lift)
      // the branches are uniform, and their tests read the bit patterns (integer pipe)
      if ((dbits(a_n) << 1) != 0) {
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = fma(a_n, Un[v * tot + g], fma(b_k, Uk[v * tot + g], R[v]));
      } else if (dbits(b_k) == dbits(1.0)) {
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = Uk[v * tot + g] + R[v];
      } else {
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = fma(b_k, Uk[v * tot + g], R[v]);
      }
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double x = fma(dt, R[v], Uk[v * tot + g]);
        u[v] = (a_n != 0.0) ? fma(a_n, Un[v * tot + g], b_k * x) : (b_k == 1.0 ? x : b_k * x);
      }
    }
  }
  if (mode == 0) return;  // uniform over the grid
  if (enforce) enforce_block<FACES>(p, u, valid, le, li, e, s_out, sh);
  if (valid) {
#pragma unroll
    for (int v = 0; v < 5; ++v) Uout[v * tot + g] = u[v];
  }
}

// Stand-alone physicality operator, in place.
template <int DIM, int N>
__global__ void __launch_bounds__(Shape<DIM, N>::BLOCK)
    enforce_kernel(Params p, double* U, double* __restrict__ s_out) {
  using S = Shape<DIM, N>;
  constexpr int Nn = S::Nn;
  __shared__ EnforceShared<DIM, N> sh;
  const int tid = threadIdx.x;
  const int le = tid / Nn, li = tid - le * Nn;
  const long long e = (long long)blockIdx.x * S::EPB + le;
  const bool valid = e < p.E;
  const long long tot = p.E * Nn;
  const long long g = e * Nn + li;
  double u[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (valid)
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = U[v * tot + g];
  if (p.enforce_faces)
    enforce_block<true>(p, u, valid, le, li, e, s_out, sh);
  else
    enforce_block<false>(p, u, valid, le, li, e, s_out, sh);
  if (valid)
#pragma unroll
    for (int v = 0; v < 5; ++v) U[v * tot + g] = u[v];
}

// ---------------------------------------------------------------------------------------
// Limiters (Sec. 2.3 names the limiters of Moe et al. and the minmod limiter, printing neither).
// means_kernel: the quadrature mean of every element.  limit_kernel: one factor theta per
// element, U_i <- mean + theta (U_i - mean), then the physicality operator when enabled.
//   scaling (limiter 1): bounds M = max(own and face-neighbour means) + alpha and
//     m = min(...) - alpha per conserved variable; the element's extremes over its nodes and
//     face traces; theta = min over the variables of (M - mean)/(max - mean) and
//     (mean - m)/(mean - min) where exceeded;
//   minmod (limiter 2): per variable and axis the face-mean deviations a+ = (mean of the +d
//     face traces) - mean and a- = mean - (the same on the -d face), the neighbour-mean
//     differences D+ and D-, mm(a) = a if |a| <= M h^2 + 2^-40 (|mean D| + |mean tau|), else
//     s min(|a|, |D+|, |D-|) if all share the sign s, else 0; theta = min of mm(a) / a.
// Non-periodic boundaries add no neighbour.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double minmod_bound(double x, const double* D, int nD, double thr) {
  if (fabs(x) <= thr) return x;
  double mag = fabs(x);
  for (int k = 0; k < nD; ++k) {
    if ((D[k] > 0.0) != (x > 0.0) || D[k] == 0.0) return 0.0;
    mag = fmin(mag, fabs(D[k]));
  }
  return x > 0.0 ? mag : -mag;
}

template <int DIM, int N>
__global__ void __launch_bounds__(Shape<DIM, N>::BLOCK)
    means_kernel(Params p, const double* __restrict__ U, double* __restrict__ means) {
  using S = Shape<DIM, N>;
  constexpr int Nn = S::Nn;
  __shared__ double sh[5][S::BLOCK];
  const int tid = threadIdx.x;
  const int le = tid / Nn, li = tid - le * Nn;
  const long long e = (long long)blockIdx.x * S::EPB + le;
  const bool valid = e < p.E;
  const long long tot = p.E * Nn;
  if (valid) {
    int ijk[3];
    node_ijk<DIM, N>(li, ijk);
    double wi = 1.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) wi *= p.w[ijk[d]];
#pragma unroll
    for (int v = 0; v < 5; ++v) sh[v][tid] = wi * U[v * tot + e * Nn + li];
  }
  __syncthreads();
  if (valid) {
    for (int v = li; v < 5; v += Nn) {  // elements of fewer than 5 nodes take several rounds
      double acc = 0.0;
      for (int j = 0; j < Nn; ++j) acc += sh[v][le * Nn + j];
      means[v * p.E + e] = acc / p.wsum;
    }
  }
}

template <int DIM, int N>
__global__ void __launch_bounds__(Shape<DIM, N>::BLOCK)
    limit_kernel(Params p, double* U, const double* __restrict__ means, int enforce,
                 double* __restrict__ s_out, double* __restrict__ theta_out) {
  using S = Shape<DIM, N>;
  constexpr int Nn = S::Nn, Nt = S::Nt, NFP = S::NFP, EPB = S::EPB;
  __shared__ EnforceShared<DIM, N> sh;  // sh.a holds the nodal state first
  __shared__ double tr[EPB][NFP][5];     // face traces of the conserved variables
  __shared__ double th[EPB];
  const int tid = threadIdx.x;
  const int le = tid / Nn, li = tid - le * Nn;
  const long long e = (long long)blockIdx.x * EPB + le;
  const bool valid = e < p.E;
  const long long tot = p.E * Nn;
  const long long g = e * Nn + li;
  double u[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (valid) {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      u[v] = U[v * tot + g];
      sh.a[v][tid] = u[v];
    }
  }
  __syncthreads();
  if (valid) {
    for (int fp = li; fp < NFP; fp += Nn) {
      const int d = fp / (2 * Nt), side = (fp / Nt) & 1, t = fp % Nt;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        double q = 0.0;
#pragma unroll
        for (int a = 0; a < N; ++a)
          q = fma(side ? p.ep[a] : p.em[a], sh.a[v][le * Nn + line_node<DIM, N>(d, t, a)], q);
        tr[le][fp][v] = q;
      }
    }
  }
  __syncthreads();
  if (valid && li == 0 && p.limiter == 2) {
    // minmod: tangential quadrature weights of the face points, summing to 2^(dim-1)
    double theta = 1.0;
    const double thr = p.lim_alpha + 0x1p-40 * (fabs(means[e]) + fabs(means[4 * p.E + e]));
    const double face_wsum = 0.5 * p.wsum;
    for (int v = 0; v < 5; ++v) {
      const double ub = means[v * p.E + e];
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const long long c = elem_coord(p, e, d);
        double D[2];
        int nD = 0;
        for (int side = 1; side >= 0; --side) {
          long long ne;
          if (side == 0)
            ne = (c > 0) ? e - p.stride[d] : (p.bc[d][0] == 0 ? e + (p.n[d] - 1) * p.stride[d] : -1);
          else
            ne = (c < p.n[d] - 1) ? e + p.stride[d] : (p.bc[d][1] == 0 ? e - (p.n[d] - 1) * p.stride[d] : -1);
          if (ne < 0) continue;
          const double un = means[v * p.E + ne];
          D[nD++] = side ? un - ub : ub - un;
        }
        double fm[2] = {0.0, 0.0};
        for (int side = 0; side < 2; ++side)
          for (int t = 0; t < Nt; ++t) {
            int ijk[3];
            node_ijk<DIM, N>(line_node<DIM, N>(d, t, 0), ijk);
            double wt = 1.0;
#pragma unroll
            for (int dd = 0; dd < DIM; ++dd)
              if (dd != d) wt *= p.w[ijk[dd]];
            fm[side] += wt * tr[le][(d * 2 + side) * Nt + t][v];
          }
        const double dev[2] = {fm[1] / face_wsum - ub, ub - fm[0] / face_wsum};
        for (int k = 0; k < 2; ++k) {
          const double mmv = minmod_bound(dev[k], D, nD, thr);
          if (mmv != dev[k]) theta = fmin(theta, mmv / dev[k]);
        }
      }
    }
    th[le] = theta;
    if (theta < 1.0) atomicAdd(&p.stats[kStatLimited * 64 + (blockIdx.x & 63)], 1ULL);
  } else if (valid && li == 0) {
    double theta = 1.0;
    for (int v = 0; v < 5; ++v) {
      const double ub = means[v * p.E + e];
      double M = ub, m = ub;
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const long long c = elem_coord(p, e, d);
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          long long ne;
          if (side == 0)
            ne = (c > 0) ? e - p.stride[d] : (p.bc[d][0] == 0 ? e + (p.n[d] - 1) * p.stride[d] : -1);
          else
            ne = (c < p.n[d] - 1) ? e + p.stride[d] : (p.bc[d][1] == 0 ? e - (p.n[d] - 1) * p.stride[d] : -1);
          if (ne < 0) continue;
          const double un = means[v * p.E + ne];
          M = fmax(M, un);
          m = fmin(m, un);
        }
      }
      M += p.lim_alpha;
      m -= p.lim_alpha;
      double hi = -1e300, lo = 1e300;
      for (int i = 0; i < Nn; ++i) {
        hi = fmax(hi, sh.a[v][le * Nn + i]);
        lo = fmin(lo, sh.a[v][le * Nn + i]);
      }
      for (int fp = 0; fp < NFP; ++fp) {
        hi = fmax(hi, tr[le][fp][v]);
        lo = fmin(lo, tr[le][fp][v]);
      }
      if (hi > M) theta = fmin(theta, (M - ub) / (hi - ub));
      if (lo < m) theta = fmin(theta, (ub - m) / (ub - lo));
    }
    th[le] = theta;
    if (theta < 1.0) atomicAdd(&p.stats[kStatLimited * 64 + (blockIdx.x & 63)], 1ULL);
  }
  __syncthreads();
  if (theta_out && valid && li == 0) theta_out[e] = th[le];  // kept for the reverse sweep
  if (valid && th[le] < 1.0) {
    const double t = th[le];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double ub = means[v * p.E + e];
      u[v] = fma(t, u[v] - ub, ub);
    }
  }
  if (enforce && p.enforce_faces)
    enforce_block<true>(p, u, valid, le, li, e, s_out, sh);
  else if (enforce)
    enforce_block<false>(p, u, valid, le, li, e, s_out, sh);
  if (valid)
#pragma unroll
    for (int v = 0; v < 5; ++v) U[v * tot + g] = u[v];
}

// ---------------------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------------------
template <int DIM, int N>
static cudaError_t launch_stage_kernels(const StageArgs& a);

}  // namespace dgsrhd

#include "kernels_split.cuh"
#include "kernels_vjp.cuh"

namespace dgsrhd {

template <int DIM, int N>
static cudaError_t launch_stage_kernels(const StageArgs& a) {
  using S = Shape<DIM, N>;
  const Params& p = *a.p;
  const unsigned eblocks = (unsigned)((p.E + S::EPB - 1) / S::EPB);
  if (a.split && (a.op == Op::Volume || a.op == Op::Update)) {
    constexpr int SB = SplitShape<DIM, N>::BLOCK;
    if (a.op == Op::Volume) {
      const size_t smem = VolSmem<DIM, N>::TOTAL;
      cudaFuncSetAttribute(volume_kernel_split<DIM, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      // the split pair keeps R_vol as FP32 and the reference fluxes as FP32 head and tail in
      // the FP64 buffers
      volume_kernel_split<DIM, N><<<eblocks, SB, smem, a.stream>>>(
          p, a.U, reinterpret_cast<float*>(a.Rvol), a.Tr, reinterpret_cast<float2*>(a.Fref));
    } else {
      auto kern = p.enforce_faces ? update_kernel_split<DIM, N, true> : update_kernel_split<DIM, N, false>;
      kern<<<eblocks, S::BLOCK, 0, a.stream>>>(
          p, reinterpret_cast<const float*>(a.Rvol), reinterpret_cast<const float2*>(a.Fs),
          reinterpret_cast<const float2*>(a.Fref),
          a.Un, a.Uk, a.Uout, a.a_n, a.b_k, a.dt, a.mode, a.enforce, a.s_out);
    }
    return cudaGetLastError();
  }
  switch (a.op) {
    case Op::Volume:
      volume_kernel<DIM, N><<<eblocks, S::BLOCK, 0, a.stream>>>(p, a.U, a.Rvol, a.Tr, a.Wstore,
                                                                 a.guard, a.Ucopy, a.rscale);
      break;
    case Op::Face: {
      long long mx = 0;
      for (int d = 0; d < DIM; ++d) mx = p.nface[d] > mx ? p.nface[d] : mx;
      const long long nthreads = mx * S::Nt;
      dim3 grid((unsigned)((nthreads + 127) / 128), DIM);
      // the split update consumes the fluxes as FP32 head and tail
      if (a.tape)
        face_kernel<DIM, N, true><<<grid, 128, 0, a.stream>>>(p, a.Tr, a.Fs, a.tape);
      else if (a.split)
        face_kernel<DIM, N, false, true><<<grid, 128, 0, a.stream>>>(p, a.Tr, a.Fs, nullptr);
      else
        face_kernel<DIM, N, false><<<grid, 128, 0, a.stream>>>(p, a.Tr, a.Fs, nullptr);
      break;
    }
    case Op::Update: {
      auto kern = p.enforce_faces ? update_kernel<DIM, N, true> : update_kernel<DIM, N, false>;
      kern<<<eblocks, S::BLOCK, 0, a.stream>>>(p, a.Rvol, a.Fs, a.Un, a.Uk, a.Uout, a.a_n, a.b_k,
                                               a.dt, a.mode, a.enforce, a.s_out,
                                               a.mode == 1 ? a.rscale : 0.0);
      break;
    }
    case Op::Enforce:
      enforce_kernel<DIM, N><<<eblocks, S::BLOCK, 0, a.stream>>>(p, a.Uout, a.s_out);
      break;
    case Op::VjpFace: {
      long long mx = 0;
      for (int d = 0; d < DIM; ++d) mx = p.nface[d] > mx ? p.nface[d] : mx;
      const long long nthreads = mx * S::Nt;
      dim3 grid((unsigned)((nthreads + 127) / 128), DIM);
      face_vjp_kernel<DIM, N><<<grid, 128, 0, a.stream>>>(p, a.Tr, a.tape, a.Rbar, a.TrBar);
      break;
    }
    case Op::VjpNode:
      if (!a.guard) return cudaErrorInvalidValue;
      node_vjp_kernel<DIM, N><<<eblocks, S::BLOCK, 0, a.stream>>>(
          p, a.U, a.Wstore, a.guard, a.Rbar, a.TrBar, a.Ubar, a.Unb, a.Ukb, a.a_n, a.b_k, a.dt);
      break;
    case Op::EnforceVjp:
      enforce_vjp_kernel<DIM, N><<<eblocks, S::BLOCK, 0, a.stream>>>(p, a.s_in, a.Tbar, a.Ubar);
      break;
    case Op::Means:
      means_kernel<DIM, N><<<eblocks, S::BLOCK, 0, a.stream>>>(p, a.Uout, a.means);
      break;
    case Op::Limit:
      limit_kernel<DIM, N><<<eblocks, S::BLOCK, 0, a.stream>>>(p, a.Uout, a.means, a.enforce,
                                                               a.s_out, a.theta_out);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int DIM>
cudaError_t dispatch_stage(int N, const StageArgs& a) {
  switch (N) {
    case 1: return launch_stage_kernels<DIM, 1>(a);
    case 2: return launch_stage_kernels<DIM, 2>(a);
    case 3: return launch_stage_kernels<DIM, 3>(a);
    case 4: return launch_stage_kernels<DIM, 4>(a);
    case 5: return launch_stage_kernels<DIM, 5>(a);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dgsrhd
