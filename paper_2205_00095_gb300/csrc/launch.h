// Launch interface between the host API and the per-dimension kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include "params.h"

namespace dgsrhd {

enum class Op { Volume, Face, Update, Enforce, VjpFace, VjpNode, EnforceVjp, Means, Limit };

struct StageArgs {
  Op op;
  const Params* p;
  cudaStream_t stream;
  const double* U;     // Volume: state whose RHS is formed
  double* Rvol;        // volume term (also R of the VJP); the split kernels keep it as FP32
  double* Tr;          // face traces
  double* Fs;          // face fluxes (the split face/update pair: FP32 head and tail)
  double* Fref;        // split precision: per-element reference flux [dim][5][E] as FP32 head and tail
  const double* Un;    // Update: U^n
  const double* Uk;    // Update: U^(k-1)
  double* Uout;        // Update: output; Enforce: state in place
  double a_n, b_k, dt;
  // Volume / Update, FP64 kernels: when nonzero, R_vol and the lift are formed times rscale
  // (the stage's b_k dt), and the update forms a_n U^n + b_k U^(k-1) + rscale R; 0 = unscaled
  double rscale;
  int mode;            // Update: 0 = write R, 1 = RK stage
  int enforce;
  int split;           // Volume / Update: split-precision tensor-core contractions (set by the host)
  int fp64_only;       // force the FP64 kernels whatever the configured precision
  double* s_out;
  double* theta_out;   // Limit: per-element limiter factor (nullable)
  // VJP buffers
  const double* Rbar;  // VjpFace / VjpNode: adjoint of R
  double* Ubar;        // VjpNode / EnforceVjp: output adjoint of U
  double* TrBar;       // VjpFace output / VjpNode input: adjoints of the face traces
  double* Wstore;      // Volume: optional output of the nodal (rho, u, P); VjpNode: its input
  unsigned char* guard;  // Volume: optional face-guard flag per face point [E][NFP]; VjpNode: input
  double* tape;        // Face: optional face-state tape (roots and reciprocals); VjpFace: input
  double* means;       // Means: output, Limit: input; element means [5][E]
  double* Ucopy;       // Volume: optional copy of the input state
  // VjpNode with Ukb set: fused stage combination Unb += a_n Rbar, Ukb += b_k (Rbar + dt Ubar)
  double* Unb;
  double* Ukb;
  const double* s_in;  // EnforceVjp: smoothing factor per element
  const double* Tbar;  // EnforceVjp: adjoint of the smoothed state
};

template <int DIM>
cudaError_t dispatch_stage(int N, const StageArgs& a);

// point-wise kernels (dimension independent)
cudaError_t launch_prim2cons(const Params& p, cudaStream_t s, long long n, const double* W,
                             double* U);
cudaError_t launch_con2prim(const Params& p, cudaStream_t s, long long n, const double* U,
                            double* W, int* iters);
cudaError_t launch_velocity_square(const Params& p, cudaStream_t s, long long n, int Nn,
                                   const double* U, int axis, double* partial, int blocks);
cudaError_t launch_math_check(cudaStream_t s, long long n, const double* x, double* out);
cudaError_t launch_fp64_probe(cudaStream_t s, int kind, long long iters, long long threads,
                              double* sink);
cudaError_t launch_con2prim_vjp(const Params& p, cudaStream_t s, long long n, const double* U,
                                const double* Wb, double* Ub);

}  // namespace dgsrhd

struct dgsrhd_config;

namespace dgsrhd {
// Launch parameters of a configuration; false for an invalid one.  n_trace / n_face_flux
// receive the sizes (in doubles) of the trace and face-flux buffers, nodes (nullable, degree + 1
// doubles) the 1D nodes of the basis.
bool params_from_config(const ::dgsrhd_config* cfg, Params* out, long long* n_trace,
                        long long* n_face_flux, double* nodes = nullptr);
}  // namespace dgsrhd
