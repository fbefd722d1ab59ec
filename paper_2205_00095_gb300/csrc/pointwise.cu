// Point-wise kernels: prim -> cons and cons -> prim at every node (any dimension).
#include "device_math.cuh"
#include "launch.h"

namespace dgsrhd {

__global__ void __launch_bounds__(256) prim2cons_kernel(Params p, long long n,
                                                         const double* __restrict__ W,
                                                         double* __restrict__ U) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    double w[5], u[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) w[v] = W[v * n + k];
    prim_v_to_cons(p, w, u);
#pragma unroll
    for (int v = 0; v < 5; ++v) U[v * n + k] = u[v];
  }
}

__global__ void __launch_bounds__(256) con2prim_kernel(Params p, long long n,
                                                        const double* __restrict__ U,
                                                        double* __restrict__ W,
                                                        int* __restrict__ iters_out) {
  __shared__ int shred[4];
  if (threadIdx.x < 4) shred[threadIdx.x] = 0;
  __syncthreads();
  int it_sum = 0, it_max = 0, nc = 0, inv = 0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    double u[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = U[v * n + k];
    Prim w;
    int it;
    const int st = con2prim(p, u, w, it);
    W[0 * n + k] = w.rho;
    W[1 * n + k] = w.v[0];
    W[2 * n + k] = w.v[1];
    W[3 * n + k] = w.v[2];
    W[4 * n + k] = w.P;
    if (iters_out) iters_out[k] = it;
    it_sum += it;
    it_max = max(it_max, it);
    nc += (st == 2);
    inv += (st == 1);
  }
  atomicAdd(&shred[0], it_sum);
  atomicMax(&shred[1], it_max);
  atomicAdd(&shred[2], nc);
  atomicAdd(&shred[3], inv);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int slot = blockIdx.x & 63;
    if (shred[0]) atomicAdd(&p.stats[kStatItersTotal * 64 + slot], (unsigned long long)shred[0]);
    if (shred[1]) atomicMax(&p.stats[kStatItersMax * 64 + slot], (unsigned long long)shred[1]);
    if (shred[2]) atomicAdd(&p.stats[kStatNonConv * 64 + slot], (unsigned long long)shred[2]);
    if (shred[3]) atomicAdd(&p.stats[kStatInvalid * 64 + slot], (unsigned long long)shred[3]);
  }
}

// U_bar = (dW/dU)^T W_bar for W = con2prim(U), W = (rho, v, P): con2prim at the node, then the
// implicit-function-theorem solve (dU/dW)^T U_bar = W_bar.
__global__ void __launch_bounds__(256) con2prim_vjp_kernel(Params p, long long n,
                                                            const double* __restrict__ U,
                                                            const double* __restrict__ Wb,
                                                            double* __restrict__ Ub) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    double u[5], wb[5], out[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      u[v] = U[v * n + k];
      wb[v] = Wb[v * n + k];
    }
    Prim w;
    int it;
    con2prim(p, u, w, it);
    const double g2 = w.lor * w.lor;
    const double v2 = w.v[0] * w.v[0] + w.v[1] * w.v[1] + w.v[2] * w.v[2];
    c2p_adjoint(p, w.rho, w.v, w.P, w.lor, 1.0 / w.lor, g2, g2 * v2, wb, out);
#pragma unroll
    for (int v = 0; v < 5; ++v) Ub[v * n + k] = out[v];
  }
}

// Partial sums of the quadrature of v_axis^2 (the Kelvin-Helmholtz diagnostic of Sec. 4.5):
// con2prim at every node, weight prod_d w[node index along d]; one partial per block (fixed
// assignment of nodes to threads and fixed reduction tree, so the sums are reproducible).
__global__ void __launch_bounds__(256) velocity_square_kernel(Params p, long long n, int Nn,
                                                              const double* __restrict__ U,
                                                              int axis,
                                                              double* __restrict__ partial) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    double u[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = U[v * n + k];
    Prim w;
    int it;
    con2prim(p, u, w, it);
    int node = (int)(k % Nn);
    double wq = 1.0;
    for (int d = 0; d < p.dim; ++d) {
      wq *= p.w[node % p.N];
      node /= p.N;
    }
    acc = fma(wq * w.v[axis], w.v[axis], acc);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// The library's reciprocal and roots next to CUDA's, for the diagnostic entry point.
__global__ void __launch_bounds__(256) math_check_kernel(long long n, const double* __restrict__ x,
                                                         double* __restrict__ out) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const double v = x[k];
    out[k] = recip_nr(v);
    out[n + k] = 1.0 / v;
    out[2 * n + k] = sqrt_nr(v);
    out[3 * n + k] = sqrt(v);
    out[4 * n + k] = v == 0.0 ? 0.0 : rcbrt_nr(v);
    out[5 * n + k] = v == 0.0 ? 0.0 : rcbrt(v);
    out[6 * n + k] = rsqrt_nr(v);
    out[7 * n + k] = rsqrt(v);
  }
}

// Throughput probe of one arithmetic operation: every thread runs four independent chains of
// `iters` applications, x <- op(x), so that enough operations are in flight to keep the
// operation's pipe busy; the chains' sum is stored so that none is removed.  kind: 0 FP64 FMA
// x <- fma(x, a, b); 1 FP64 division x <- b / x; 2 sqrt; 3 rsqrt; 4 rcbrt; the library's
// 5 reciprocal (recip_nr), 6 square root (sqrt_nr), 7 reciprocal cube root (rcbrt_nr); 8 FP32
// FMA; 9 the library's reciprocal square root (rsqrt_nr).  a and b are kernel arguments (not constants
// the compiler could fold); every chain stays bounded.
template <int KIND>
__device__ __forceinline__ double probe_op(double x, double a, double b) {
  if (KIND == 0) return fma(x, a, b);
  if (KIND == 1) return b / x;
  if (KIND == 2) return sqrt(x);
  if (KIND == 3) return rsqrt(x);
  if (KIND == 4) return rcbrt(x);
  if (KIND == 5) return recip_nr(x);
  if (KIND == 6) return sqrt_nr(x);
  if (KIND == 9) return rsqrt_nr(x);
  return rcbrt_nr(x);
}

template <int KIND>
__global__ void __launch_bounds__(256) fp64_probe_kernel(long long iters, double a, double b,
                                                         double* __restrict__ sink) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double x0 = 1.0 + 1e-7 * (double)(t & 1023), x1 = x0 + 0.25, x2 = x0 + 0.5, x3 = x0 + 0.75;
  for (long long k = 0; k < iters; ++k) {
    x0 = probe_op<KIND>(x0, a, b);
    x1 = probe_op<KIND>(x1, a, b);
    x2 = probe_op<KIND>(x2, a, b);
    x3 = probe_op<KIND>(x3, a, b);
  }
  sink[t] = (x0 + x1) + (x2 + x3);
}

__global__ void __launch_bounds__(256) fp32_probe_kernel(long long iters, float a, float b,
                                                         double* __restrict__ sink) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float x0 = 1.0f + 1e-4f * (float)(t & 1023), x1 = x0 + 0.25f, x2 = x0 + 0.5f, x3 = x0 + 0.75f;
  for (long long k = 0; k < iters; ++k) {
    x0 = fmaf(x0, a, b);
    x1 = fmaf(x1, a, b);
    x2 = fmaf(x2, a, b);
    x3 = fmaf(x3, a, b);
  }
  sink[t] = (double)((x0 + x1) + (x2 + x3));
}

cudaError_t launch_fp64_probe(cudaStream_t s, int kind, long long iters, long long threads,
                              double* sink) {
  const unsigned blocks = (unsigned)(threads / 256);
  const double a = 0.999999, b = 1e-6;
  switch (kind) {
    case 0: fp64_probe_kernel<0><<<blocks, 256, 0, s>>>(iters, a, b, sink); break;
    case 1: fp64_probe_kernel<1><<<blocks, 256, 0, s>>>(iters, a, 1.5, sink); break;
    case 2: fp64_probe_kernel<2><<<blocks, 256, 0, s>>>(iters, a, b, sink); break;
    case 3: fp64_probe_kernel<3><<<blocks, 256, 0, s>>>(iters, a, b, sink); break;
    case 4: fp64_probe_kernel<4><<<blocks, 256, 0, s>>>(iters, a, b, sink); break;
    case 5: fp64_probe_kernel<5><<<blocks, 256, 0, s>>>(iters, a, b, sink); break;
    case 6: fp64_probe_kernel<6><<<blocks, 256, 0, s>>>(iters, a, b, sink); break;
    case 7: fp64_probe_kernel<7><<<blocks, 256, 0, s>>>(iters, a, b, sink); break;
    case 8: fp32_probe_kernel<<<blocks, 256, 0, s>>>(iters, 0.999999f, 1e-6f, sink); break;
    case 9: fp64_probe_kernel<9><<<blocks, 256, 0, s>>>(iters, a, b, sink); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

static unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  const long long cap = 152LL * 16;  // enough resident blocks to fill the GPU
  return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

cudaError_t launch_prim2cons(const Params& p, cudaStream_t s, long long n, const double* W,
                             double* U) {
  prim2cons_kernel<<<grid_for(n), 256, 0, s>>>(p, n, W, U);
  return cudaGetLastError();
}

cudaError_t launch_con2prim(const Params& p, cudaStream_t s, long long n, const double* U,
                            double* W, int* iters) {
  con2prim_kernel<<<grid_for(n), 256, 0, s>>>(p, n, U, W, iters);
  return cudaGetLastError();
}

cudaError_t launch_velocity_square(const Params& p, cudaStream_t s, long long n, int Nn,
                                   const double* U, int axis, double* partial, int blocks) {
  velocity_square_kernel<<<blocks, 256, 0, s>>>(p, n, Nn, U, axis, partial);
  return cudaGetLastError();
}

cudaError_t launch_math_check(cudaStream_t s, long long n, const double* x, double* out) {
  if (n == 0) return cudaSuccess;
  math_check_kernel<<<grid_for(n), 256, 0, s>>>(n, x, out);
  return cudaGetLastError();
}

cudaError_t launch_con2prim_vjp(const Params& p, cudaStream_t s, long long n, const double* U,
                                const double* Wb, double* Ub) {
  con2prim_vjp_kernel<<<grid_for(n), 256, 0, s>>>(p, n, U, Wb, Ub);
  return cudaGetLastError();
}

}  // namespace dgsrhd
