// Split-precision variants of the volume and update kernels.  The volume term and the
// face-trace extrapolation run on tensor cores (3xTF32, FP32 accumulation, see split.cuh); the
// lift, a rank-2 update per line, runs as FP32 FMAs.  The nodal flux, which enters only the
// volume contraction, is formed as FP32 head-and-tail pairs from those of U, v and P (within
// about 2^-46 of the FP64 flux).  con2prim, the numerical flux, the Lorentz factors, the RK
// combination, the element means and the physicality operator stay in FP64.
//
// The contractions act on deviations from a per-element reference (the values at the element's
// first node).  The DG operator annihilates constants (summation by parts:
// sum_a Dhat[i][a] = phi_i(+1)/w_i - phi_i(-1)/w_i, the lift of a constant flux on both faces),
// so with the same reference flux F_ref in the volume term and in the lift
//   R = Dhat (F - F_ref) - lift(F* - F_ref)
// exactly, and the traces are W_ref + sum_i phi_i(+-1) (W_i - W_ref) (partition of unity).  The
// FP32 and TF32 parts then carry only the variation inside an element, O(dx |grad F|), instead
// of |F| itself, which keeps their rounding below the cancellation between volume and surface
// terms.  A deviation is formed in FP32 from the FP32 heads and tails of the value and of the
// reference (split.cuh: dev_f32), as accurate as the FP32 truncation of the exact FP64
// difference and without an FP64 operation.  R_vol leaves the volume kernel as FP32 and the
// update adds the FP32 lift to it before widening R to FP64 for the RK combination.
#pragma once

#include "kernels.cuh"
#include "split.cuh"

namespace dgsrhd {

template <int DIM, int N>
struct SplitShape {
  using S = Shape<DIM, N>;
  static constexpr int BLOCK = (S::BLOCK + 31) / 32 * 32;  // whole warps for mma.sync
  static constexpr int WARPS = BLOCK / 32;
  static constexpr int LINES = S::EPB * S::Nt;              // lines per axis in a block
  static constexpr int TILES = (LINES + 15) / 16;           // 16-line row tiles
  // resident blocks per SM asked of the register allocator for the volume kernel: its shared
  // memory admits at least three 256-thread blocks, which 85 registers per thread keep
  static constexpr int VOL_MIN_BLOCKS = 3;
};

// Byte offsets of the dynamic shared memory of the split volume kernel.
template <int DIM, int N>
struct VolSmem {
  using Q = SplitShape<DIM, N>;
  static constexpr int BLOCK = Q::BLOCK, LINES = Q::LINES;
  static constexpr size_t F = 0;                                          // uint2 [DIM][5][BLOCK]
  static constexpr size_t W = F + sizeof(uint2) * DIM * 5 * BLOCK;        // uint2 [5][BLOCK]
  static constexpr size_t BV = W + sizeof(uint2) * 5 * BLOCK;             // uint2 [DIM][8][8]
  static constexpr size_t BT = BV + sizeof(uint2) * DIM * 64;             // uint2 [8][8]
  static constexpr size_t OV = BT + sizeof(uint2) * 64;                   // float [DIM][5][BLOCK]
  static constexpr size_t OT = OV + sizeof(float) * DIM * 5 * BLOCK;      // float [DIM][2][5][LINES]
  static constexpr size_t FR = OT + sizeof(float) * DIM * 2 * 5 * LINES;  // F32Pair [EPB][DIM][5]
  static constexpr size_t WR = FR + sizeof(F32Pair) * Shape<DIM, N>::EPB * DIM * 5;  // double [EPB][5]
  static constexpr size_t WRP = WR + sizeof(double) * Shape<DIM, N>::EPB * 5;  // F32Pair [EPB][5]
  static constexpr size_t RED = WRP + sizeof(F32Pair) * Shape<DIM, N>::EPB * 5;  // int [128]
  static constexpr size_t TOTAL = RED + sizeof(int) * 128;
};

__device__ __forceinline__ uint2 as_u2(Tf32Pair p) { return make_uint2(p.hi, p.lo); }

// One 16-line tile of the contraction along axis d for variable plane `src` (uint2 hi/lo per
// node of the block): A[row][k] = src[node(row, k)], B = coef (uint2 [8][8], B[k][n]).
// Calls `store(row, n, value)` for every valid output of the tile.
template <int DIM, int N, class Store>
__device__ __forceinline__ void contract_tile(const uint2* __restrict__ src, const uint2* __restrict__ coef,
                                              int d, int tile, int ncols, Store&& store) {
  constexpr int Nn = Shape<DIM, N>::Nn, Nt = Shape<DIM, N>::Nt;
  constexpr int LINES = SplitShape<DIM, N>::LINES;
  const int lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
  const int r0 = tile * 16 + g, r1 = r0 + 8;
  unsigned ahi[4], alo[4], bhi[2], blo[2];
  const int rows[2] = {r0, r1};
  const int ks[2] = {tig, tig + 4};
#pragma unroll
  for (int kk = 0; kk < 2; ++kk)
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      const int r = rows[rr], k = ks[kk];
      uint2 v = make_uint2(0u, 0u);
      if (r < LINES && k < N) {
        const int le = r / Nt, t = r - le * Nt;
        v = src[le * Nn + line_node<DIM, N>(d, t, k)];
      }
      ahi[kk * 2 + rr] = v.x;
      alo[kk * 2 + rr] = v.y;
    }
  const uint2 b0 = coef[tig * 8 + g], b1 = coef[(tig + 4) * 8 + g];
  bhi[0] = b0.x;
  blo[0] = b0.y;
  bhi[1] = b1.x;
  blo[1] = b1.y;
  float c[4] = {0.f, 0.f, 0.f, 0.f};
  mma_3xtf32(c, ahi, alo, bhi, blo);
  const int n0 = 2 * tig, n1 = 2 * tig + 1;
  if (r0 < LINES) {
    if (n0 < ncols) store(r0, n0, c[0]);
    if (n1 < ncols) store(r0, n1, c[1]);
  }
  if (r1 < LINES) {
    if (n0 < ncols) store(r1, n0, c[2]);
    if (n1 < ncols) store(r1, n1, c[3]);
  }
}

template <int DIM, int N>
__global__ void __launch_bounds__(SplitShape<DIM, N>::BLOCK, SplitShape<DIM, N>::VOL_MIN_BLOCKS)
    volume_kernel_split(Params p, const double* __restrict__ U, float* __restrict__ Rvol,
                        double* __restrict__ Tr, float2* __restrict__ Fref) {
  using S = Shape<DIM, N>;
  using Q = SplitShape<DIM, N>;
  using L = VolSmem<DIM, N>;
  constexpr int Nn = S::Nn, Nt = S::Nt, BLOCK = Q::BLOCK, LINES = Q::LINES;
  extern __shared__ __align__(16) unsigned char smem[];
  uint2* shF = reinterpret_cast<uint2*>(smem + L::F);
  uint2* shW = reinterpret_cast<uint2*>(smem + L::W);
  uint2* shBV = reinterpret_cast<uint2*>(smem + L::BV);
  uint2* shBT = reinterpret_cast<uint2*>(smem + L::BT);
  float* outV = reinterpret_cast<float*>(smem + L::OV);
  float* outT = reinterpret_cast<float*>(smem + L::OT);
  F32Pair* shFR = reinterpret_cast<F32Pair*>(smem + L::FR);
  double* shWR = reinterpret_cast<double*>(smem + L::WR);
  F32Pair* shWRp = reinterpret_cast<F32Pair*>(smem + L::WRP);
  int* shred = reinterpret_cast<int*>(smem + L::RED);

  const int tid = threadIdx.x;
  // coefficient matrices B[k][n]: volume (2/dx_d) Dhat[n][k]; traces phi_k(-1), phi_k(+1)
  for (int j = tid; j < DIM * 64; j += BLOCK) {
    const int d = j / 64, k = (j / 8) % 8, n = j % 8;
    const double v = (k < N && n < N) ? p.inv_half_dx[d] * p.Dhat[n * N + k] : 0.0;
    shBV[j] = as_u2(split_tf32_f64(v));
  }
  if (tid < 64) {
    const int k = tid / 8, n = tid % 8;
    const double v = (k < N && n < 2) ? (n == 0 ? p.em[k] : p.ep[k]) : 0.0;
    shBT[tid] = as_u2(split_tf32_f64(v));
  }
  const int le = tid / Nn, li = tid - le * Nn;
  const long long e = (long long)blockIdx.x * S::EPB + le;
  const bool valid = tid < S::BLOCK && e < p.E;
  const long long tot = p.E * Nn;
  const long long g = e * Nn + li;

  int iters = 0, status = 0;
  if (valid) {
    double u[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = U[v * tot + g];
    Prim W;
    status = con2prim(p, u, W, iters);
    // nodal flux (D v_d, S v_d + P e_d, (tau + P) v_d) as FP32 pairs (its terms share one sign),
    // parked in the node's slots of shF until the element's reference is known
    F32Pair up[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      // an empty statement that reads con2prim's result: the pair of u[v] is formed after the
      // recovery, so that it does not hold registers through it
      double uv = u[v];
      asm("" : "+d"(uv) : "d"(W.P));
      up[v] = f32_pair(uv);
    }
    const F32Pair Pp = f32_pair(W.P);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const F32Pair vp = f32_pair(W.v[d]);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        F32Pair F;
        if (v < 4) {
          F = mul_pair(up[v], vp);
          if (v == 1 + d) F = add_pair(F, Pp);
        } else {
          F = add_pair(mul_pair(up[4], vp), mul_pair(Pp, vp));
        }
        shF[(d * 5 + v) * BLOCK + tid] = make_uint2(__float_as_uint(F.hi), __float_as_uint(F.lo));
        if (li == 0) {  // the element's first node is its reference
          shFR[(le * DIM + d) * 5 + v] = F;
          // doubled for the update kernel, which lifts 2 F* - 2 F_ref (exact scaling)
          Fref[((long long)d * 5 + v) * p.E + e] = make_float2(2.0f * F.hi, 2.0f * F.lo);
        }
      }
    }
    const double Wu[5] = {W.rho, W.lor * W.v[0], W.lor * W.v[1], W.lor * W.v[2], W.P};
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      // (rho, u, P) as FP32 head and tail, parked in the node's slot of shW like the fluxes
      const F32Pair w = f32_pair(Wu[v]);
      shW[v * BLOCK + tid] = make_uint2(__float_as_uint(w.hi), __float_as_uint(w.lo));
      if (li == 0) {  // the element's first node is its reference
        shWR[le * 5 + v] = Wu[v];
        shWRp[le * 5 + v] = w;
      }
    }
  }
  block_stats(p, iters, status, shred);  // contains __syncthreads
  if (valid) {
#pragma unroll
    for (int d = 0; d < DIM; ++d)
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const uint2 f = shF[(d * 5 + v) * BLOCK + tid];  // this thread's own slot
        shF[(d * 5 + v) * BLOCK + tid] = as_u2(split_tf32(
            dev_f32(F32Pair{__uint_as_float(f.x), __uint_as_float(f.y)}, shFR[(le * DIM + d) * 5 + v])));
      }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const uint2 w = shW[v * BLOCK + tid];  // this thread's own slot
      shW[v * BLOCK + tid] = as_u2(split_tf32(
          dev_f32(F32Pair{__uint_as_float(w.x), __uint_as_float(w.y)}, shWRp[le * 5 + v])));
    }
  } else {
#pragma unroll
    for (int d = 0; d < DIM; ++d)
#pragma unroll
      for (int v = 0; v < 5; ++v) shF[(d * 5 + v) * BLOCK + tid] = make_uint2(0u, 0u);
#pragma unroll
    for (int v = 0; v < 5; ++v) shW[v * BLOCK + tid] = make_uint2(0u, 0u);
  }
  __syncthreads();

  // tensor-core contractions: volume term (DIM x 5 x TILES tasks) and traces (same count)
  const int warp = tid >> 5;
  constexpr int TASKS = DIM * 5 * Q::TILES;
  for (int task = warp; task < 2 * TASKS; task += Q::WARPS) {
    const bool trace = task >= TASKS;
    const int tk = trace ? task - TASKS : task;
    const int d = tk / (5 * Q::TILES), v = (tk / Q::TILES) % 5, tile = tk % Q::TILES;
    if (!trace) {
      contract_tile<DIM, N>(shF + (d * 5 + v) * BLOCK, shBV + d * 64, d, tile, N,
                            [&](int row, int n, float val) {
                              const int lr = row / Nt, t = row - lr * Nt;
                              outV[(d * 5 + v) * BLOCK + lr * Nn + line_node<DIM, N>(d, t, n)] = val;
                            });
    } else {
      contract_tile<DIM, N>(shW + v * BLOCK, shBT, d, tile, 2, [&](int row, int n, float val) {
        outT[((d * 2 + n) * 5 + v) * LINES + row] = val;
      });
    }
  }
  __syncthreads();

  if (valid) {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      float acc = 0.f;
#pragma unroll
      for (int d = 0; d < DIM; ++d) acc += outV[(d * 5 + v) * BLOCK + tid];
      Rvol[v * tot + g] = acc;  // FP32: the update adds the FP32 lift before widening
    }
    int guard = 0;
    for (int fp = li; fp < S::NFP; fp += Nn) {
      const int d = fp / (2 * Nt);
      const int side = (fp / Nt) & 1;
      const int t = fp % Nt;
      double out[5];
#pragma unroll
      for (int v = 0; v < 5; ++v)
        out[v] = shWR[le * 5 + v] + f32_to_f64_bits(outT[((d * 2 + side) * 5 + v) * LINES + le * Nt + t]);
      if (!pos_bits(out[0]) || !pos_bits(out[4])) {
        const int node = le * Nn + line_node<DIM, N>(d, t, side ? N - 1 : 0);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const uint2 w = shW[v * BLOCK + node];
          out[v] = shWR[le * 5 + v] + f32_to_f64_bits(__uint_as_float(w.x) + __uint_as_float(w.y));
        }
        ++guard;
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) Tr[((((long long)d * 2 + side) * 5 + v) * p.E + e) * Nt + t] = out[v];
    }
    if (guard) atomicAdd(&p.stats[kStatFaceGuard * 64 + (blockIdx.x & 63)], (unsigned long long)guard);
  }
}

// Split update: R = R_vol + lift in FP32, widened once; then the SSP-RK combination and the
// physicality operator in FP64, as in update_kernel.  The lift is a rank-2 update per line
// (K = 2: the line's two face fluxes), far below a tensor-core tile, so it runs as FP32 FMAs on
// the FP32 deviations F* - F_ref (exact products and one rounding each: at least the accuracy
// of the 3xTF32 products).  The face fluxes arrive as FP32 head and tail (face_kernel with
// pairs), the reference fluxes likewise (volume_kernel_split).  The kernel waits on its loads
// (few FP64 instructions per node hide little), so it is held to 48 registers for five resident
// blocks per SM (three with the face points, which need more registers).
template <int DIM, int N, bool FACES>
__global__ void __launch_bounds__(Shape<DIM, N>::BLOCK, FACES ? 3 : 5)
    update_kernel_split(Params p, const float* __restrict__ Rvol, const float2* __restrict__ Fs,
                        const float2* __restrict__ Fref, const double* Un, const double* Uk,
                        double* Uout, double a_n, double b_k, double dt, int mode, int enforce,
                        double* __restrict__ s_out) {
  using S = Shape<DIM, N>;
  constexpr int Nn = S::Nn;
  __shared__ EnforceShared<DIM, N> sh;
  // (2/dx_d) phi_i(-+1)/w_i per axis, rounded to FP32 and halved: the face kernel stores 2 F*
  // and the volume kernel 2 F_ref
  __shared__ float shl[DIM][2][N];
  // the element's reference fluxes, read once per element rather than once per node
  __shared__ float2 shref[S::EPB][DIM * 5];
  const int tid = threadIdx.x;
  if (tid < DIM * N) {
    const int d = tid / N, i = tid % N;
    shl[d][0][i] = 0.5f * f64_to_f32_bits(p.inv_half_dx[d] * p.lm[i]);
    shl[d][1][i] = 0.5f * f64_to_f32_bits(p.inv_half_dx[d] * p.lp[i]);
  }
  const int le = tid / Nn, li = tid - le * Nn;
  const long long e = (long long)blockIdx.x * S::EPB + le;
  const bool valid = e < p.E;
  const long long tot = p.E * Nn;
  const long long g = e * Nn + li;
  if (valid)
    for (int j = li; j < DIM * 5; j += Nn) shref[le][j] = Fref[(long long)j * p.E + e];
  __syncthreads();
  double u[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (valid) {
    int ijk[3];
    node_ijk<DIM, N>(li, ijk);
    float lift[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const int t = tan_index<DIM, N>(ijk, d);
      const long long nf = p.nface[d];
      const float2* fs = Fs + p.fs_off[d];
      const long long flo = e, fhi = high_face(p, e, d);
      const float cp = shl[d][1][ijk[d]];
      const float cm = shl[d][0][ijk[d]];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const float2 r = shref[le][d * 5 + v];
        const float2 xh = fs[(v * nf + fhi) * S::Nt + t];
        const float2 xl = fs[(v * nf + flo) * S::Nt + t];
        const F32Pair rp{r.x, r.y};
        lift[v] = fmaf(cm, dev_f32(F32Pair{xl.x, xl.y}, rp), lift[v]);
        lift[v] = fmaf(-cp, dev_f32(F32Pair{xh.x, xh.y}, rp), lift[v]);
      }
    }
    double R[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) R[v] = f32_to_f64_bits(__fadd_rn(Rvol[v * tot + g], lift[v]));
    if (mode == 0) {
#pragma unroll
      for (int v = 0; v < 5; ++v) Uout[v * tot + g] = R[v];
    } else if ((dbits(a_n) << 1) != 0) {  // uniform branches on the bit patterns; no b_k x
      // is formed where b_k = 1
#pragma unroll
      for (int v = 0; v < 5; ++v)
        u[v] = fma(a_n, Un[v * tot + g], b_k * fma(dt, R[v], Uk[v * tot + g]));
    } else if (dbits(b_k) == dbits(1.0)) {
#pragma unroll
      for (int v = 0; v < 5; ++v) u[v] = fma(dt, R[v], Uk[v * tot + g]);
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) u[v] = b_k * fma(dt, R[v], Uk[v * tot + g]);
    }
  }
  if (mode == 0) return;  // uniform over the grid
  if (enforce) enforce_block<FACES>(p, u, valid, le, li, e, s_out, sh);
  if (valid) {
#pragma unroll
    for (int v = 0; v < 5; ++v) Uout[v * tot + g] = u[v];
  }
}

}  // namespace dgsrhd
