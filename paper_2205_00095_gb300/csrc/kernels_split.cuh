// Split-precision variants of the volume and update kernels: the volume term, the face-trace
// extrapolation and the lift run on tensor cores (3xTF32, FP32 accumulation, see split.cuh);
// con2prim, the nodal and numerical fluxes, the Lorentz factors, the RK combination, the
// element means and the physicality operator stay in FP64.
//
// The contractions act on deviations from a per-element reference (the values at the element's
// first node).  A deviation is formed in FP32 from the FP32 heads and tails of the value and of
// the reference (split.cuh: dev_f32), as accurate as the FP32 truncation of the exact FP64
// difference and without an FP64 operation.  R_vol leaves the volume kernel as FP32 and the
// update adds the FP32 lift to it before widening R to FP64 for the RK combination.  The DG operator annihilates constants
// (summation by parts: sum_a Dhat[i][a] = phi_i(+1)/w_i - phi_i(-1)/w_i, the lift of a constant
// flux on both faces), so with the same reference flux F_ref in the volume term and in the lift
//   R = Dhat (F - F_ref) - lift(F* - F_ref)
// exactly, and the traces are W_ref + sum_i phi_i(+-1) (W_i - W_ref) (partition of unity).  The
// TF32 parts then carry only the variation inside an element, O(dx |grad F|), instead of
// |F| itself, which keeps the rounding of the split below the cancellation between volume and
// surface terms.
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
__global__ void __launch_bounds__(SplitShape<DIM, N>::BLOCK)
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
  double F[DIM][5], Wu[5];
  if (valid) {
    double u[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = U[v * tot + g];
    Prim W;
    status = con2prim(p, u, W, iters);
#pragma unroll
    for (int d = 0; d < DIM; ++d) phys_flux(u, W.v, W.P, d, F[d]);
    Wu[0] = W.rho;
    Wu[1] = W.lor * W.v[0];
    Wu[2] = W.lor * W.v[1];
    Wu[3] = W.lor * W.v[2];
    Wu[4] = W.P;
    if (li == 0) {  // the element's first node is its reference, kept as FP32 head and tail
#pragma unroll
      for (int d = 0; d < DIM; ++d)
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const F32Pair r = f32_pair(F[d][v]);
          shFR[(le * DIM + d) * 5 + v] = r;
          Fref[((long long)d * 5 + v) * p.E + e] = make_float2(r.hi, r.lo);
        }
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        shWR[le * 5 + v] = Wu[v];
        shWRp[le * 5 + v] = f32_pair(Wu[v]);
      }
    }
  }
  block_stats(p, iters, status, shred);  // contains __syncthreads
  if (valid) {
#pragma unroll
    for (int d = 0; d < DIM; ++d)
#pragma unroll
      for (int v = 0; v < 5; ++v)
        shF[(d * 5 + v) * BLOCK + tid] =
            as_u2(split_tf32(dev_f32(f32_pair(F[d][v]), shFR[(le * DIM + d) * 5 + v])));
#pragma unroll
    for (int v = 0; v < 5; ++v)
      shW[v * BLOCK + tid] = as_u2(split_tf32(dev_f32(f32_pair(Wu[v]), shWRp[le * 5 + v])));
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

// Byte offsets of the dynamic shared memory of the split update kernel.
template <int DIM, int N>
struct UpdSmem {
  using Q = SplitShape<DIM, N>;
  static constexpr int BLOCK = Q::BLOCK;
  using Enf = EnforceShared<DIM, N, BLOCK>;
  static constexpr size_t E = 0;                                         // Enf
  static constexpr size_t BL = (sizeof(Enf) + 15) / 16 * 16;             // uint2 [DIM][8][8]
  static constexpr size_t OL = BL + sizeof(uint2) * DIM * 64;            // float [DIM][5][BLOCK]
  static constexpr size_t FS = OL + sizeof(float) * DIM * 5 * BLOCK;     // uint2 [DIM][2][5][LINES]
  static constexpr size_t TOTAL = FS + sizeof(uint2) * DIM * 2 * 5 * Q::LINES;
};

template <int DIM, int N>
__global__ void __launch_bounds__(SplitShape<DIM, N>::BLOCK)
    update_kernel_split(Params p, const float* __restrict__ Rvol, const double* __restrict__ Fs,
                        const float2* __restrict__ Fref, const double* Un, const double* Uk,
                        double* Uout, double a_n, double b_k, double dt, int mode, int enforce,
                        double* __restrict__ s_out) {
  using S = Shape<DIM, N>;
  using Q = SplitShape<DIM, N>;
  using L = UpdSmem<DIM, N>;
  constexpr int Nn = S::Nn, Nt = S::Nt, BLOCK = Q::BLOCK, LINES = Q::LINES;
  extern __shared__ __align__(16) unsigned char smem[];
  typename L::Enf& sh = *reinterpret_cast<typename L::Enf*>(smem + L::E);
  uint2* shBL = reinterpret_cast<uint2*>(smem + L::BL);
  float* outL = reinterpret_cast<float*>(smem + L::OL);
  uint2* shFs = reinterpret_cast<uint2*>(smem + L::FS);
  const int tid = threadIdx.x;
  // lift coefficients B[k][n]: k = 0 low-face flux (+ (2/dx) phi_n(-1)/w_n),
  // k = 1 high-face flux (- (2/dx) phi_n(+1)/w_n)
  for (int j = tid; j < DIM * 64; j += BLOCK) {
    const int d = j / 64, k = (j / 8) % 8, n = j % 8;
    double v = 0.0;
    if (n < N && k == 0) v = p.inv_half_dx[d] * p.lm[n];
    if (n < N && k == 1) v = -p.inv_half_dx[d] * p.lp[n];
    shBL[j] = as_u2(split_tf32_f64(v));
  }
  __syncthreads();

  // stage the block's face fluxes minus the reference flux, TF32-split, in shared memory:
  // shFs[d][side][v][line], side 0 = low face, 1 = high face; lines run fastest so that
  // consecutive threads read consecutive face points
  for (int j = tid; j < DIM * 2 * 5 * LINES; j += BLOCK) {
    const int r = j % LINES;
    const int v = (j / LINES) % 5;
    const int side = (j / (5 * LINES)) % 2;
    const int d = j / (10 * LINES);
    const int lr = r / Nt, t = r - lr * Nt;
    const long long e = (long long)blockIdx.x * S::EPB + lr;
    uint2 val = make_uint2(0u, 0u);
    if (e < p.E) {
      const long long f = side == 0 ? e : high_face(p, e, d);
      const float2 r = Fref[((long long)d * 5 + v) * p.E + e];
      const F32Pair rp = {r.x, r.y};
      val = as_u2(split_tf32(dev_f32(f32_pair(Fs[p.fs_off[d] + (v * p.nface[d] + f) * Nt + t]), rp)));
    }
    shFs[j] = val;
  }
  __syncthreads();

  // lift on tensor cores: rows are the block's lines, k selects the low / high face flux
  const int warp = tid >> 5, lane = tid & 31, gq = lane >> 2, tig = lane & 3;
  constexpr int TASKS = DIM * 5 * Q::TILES;
  for (int task = warp; task < TASKS; task += Q::WARPS) {
    const int d = task / (5 * Q::TILES), v = (task / Q::TILES) % 5, tile = task % Q::TILES;
    unsigned ahi[4] = {0u, 0u, 0u, 0u}, alo[4] = {0u, 0u, 0u, 0u};
    if (tig < 2) {  // k = tig in {0, 1}; k = tig + 4 is padding
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const int r = tile * 16 + gq + 8 * rr;
        if (r < LINES) {
          const uint2 q = shFs[((d * 2 + tig) * 5 + v) * LINES + r];
          ahi[rr] = q.x;
          alo[rr] = q.y;
        }
      }
    }
    const uint2 b0 = shBL[d * 64 + tig * 8 + gq], b1 = shBL[d * 64 + (tig + 4) * 8 + gq];
    const unsigned bhi[2] = {b0.x, b1.x}, blo[2] = {b0.y, b1.y};
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    mma_3xtf32(c, ahi, alo, bhi, blo);
    const int rows[2] = {tile * 16 + gq, tile * 16 + gq + 8};
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int r = rows[rr], n = 2 * tig + cc;
        if (r < LINES && n < N) {
          const int lr = r / Nt, t = r - lr * Nt;
          outL[(d * 5 + v) * BLOCK + lr * Nn + line_node<DIM, N>(d, t, n)] = c[rr * 2 + cc];
        }
      }
  }
  __syncthreads();

  const int le = tid / Nn, li = tid - le * Nn;
  const long long e = (long long)blockIdx.x * S::EPB + le;
  const bool valid = tid < S::BLOCK && e < p.E;
  const long long tot = p.E * Nn;
  const long long g = e * Nn + li;
  double u[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (valid) {
    double R[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      float lift = 0.f;
#pragma unroll
      for (int d = 0; d < DIM; ++d) lift += outL[(d * 5 + v) * BLOCK + tid];
      // R_vol and the lift are FP32 sums of deviation products: their sum in FP32 keeps that
      // accuracy and is widened once
      R[v] = f32_to_f64_bits(__fadd_rn(Rvol[v * tot + g], lift));
    }
    if (mode == 0) {
#pragma unroll
      for (int v = 0; v < 5; ++v) Uout[v * tot + g] = R[v];
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double x = fma(dt, R[v], Uk[v * tot + g]);
        u[v] = (a_n != 0.0) ? fma(a_n, Un[v * tot + g], b_k * x) : b_k * x;
      }
    }
  }
  if (mode == 0) return;
  // enforce_block expects le/li of the FP64 layout; threads past S::BLOCK carry no node
  if (enforce) enforce_block(p, u, valid, valid ? le : 0, valid ? li : 1, e, s_out, sh);
  if (valid) {
#pragma unroll
    for (int v = 0; v < 5; ++v) Uout[v * tot + g] = u[v];
  }
}

}  // namespace dgsrhd
