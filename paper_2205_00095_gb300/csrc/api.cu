// Host side of the C ABI declared in include/dgsrhd.h: configuration checks, the Gauss-Legendre
// basis tables, scratch ownership, launch sequencing of one SSP-RK step and its CUDA graph.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/dgsrhd.h"
#include "launch.h"
#include "params.h"

using dgsrhd::Op;
using dgsrhd::Params;
using dgsrhd::StageArgs;

struct dgsrhd_ctx {
  dgsrhd_config cfg;
  Params p;
  cudaStream_t stream;
  int dim, N;
  long long E, Nn, nstate;  // nstate = 5 E Nn doubles
  double x[dgsrhd::kMaxN];  // Gauss-Legendre nodes
  double dx[3];
  // scratch
  double* A;    // RK stage state
  double* Rv;   // volume term / R
  double* Tr;   // face traces
  double* Fs;   // face fluxes
  double* Fref; // split precision: reference flux per element [dim][5][E]
  double* Ud;   // device state for dgsrhd_step_host
  double* Wv;   // VJP: nodal (rho, u, P)
  double* TrB;  // VJP: trace adjoints
  double* Yb;   // stage VJP: adjoint of the stage before the operator
  double* Yb2;  // stage VJP: adjoint before the limiter (limited configurations)
  unsigned char* Gd;  // VJP: face-guard flag per face point [E][2 dim Nt]
  double* Mn;   // limiter: element means [5][E]
  long long fs_total;  // doubles of the face-flux buffer
  unsigned long long* stats;
  long long c2p_calls;
  long long launches;
  // captured step
  // captured steps, one per (state pointer, dt), least recently used evicted
  struct StepGraph {
    cudaGraphExec_t exec;
    double dt;
    double* U;
    unsigned long long used;
  };
  std::vector<StepGraph> graphs;
  unsigned long long graph_clock;
  // kernel timing
  bool profiling;
  struct TimedLaunch {
    int kind;
    cudaEvent_t start, stop;
  };
  std::vector<TimedLaunch> timed;
  std::vector<cudaEvent_t> event_pool;
};

namespace {

// ---- Gauss-Legendre nodes by Newton iteration on P_N, barycentric Lagrange tables ----------
void legendre_pair(int n, double x, double* p, double* dp) {
  double a = 1.0, b = x;
  if (n == 0) {
    *p = 1.0;
    *dp = 0.0;
    return;
  }
  for (int k = 1; k < n; ++k) {
    const double c = ((2 * k + 1) * x * b - k * a) / (k + 1);
    a = b;
    b = c;
  }
  *p = b;
  *dp = n * (a - x * b) / (1.0 - x * x);
}

void gauss_legendre(int N, double* x, double* w) {
  for (int i = 0; i < N; ++i) {
    // i-th root from the top, then stored ascending
    double t = cos(M_PI * (i + 0.75) / (N + 0.5));
    if (N == 1) t = 0.0;
    for (int k = 0; k < 60 && N > 1; ++k) {
      double p, dp;
      legendre_pair(N, t, &p, &dp);
      const double step = p / dp;
      t -= step;
      if (fabs(step) <= 1e-17) break;
    }
    double p, dp;
    legendre_pair(N, t, &p, &dp);
    x[N - 1 - i] = t;
    w[N - 1 - i] = (N == 1) ? 2.0 : 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

// N >= 2 Gauss-Lobatto-Legendre nodes (ascending) and weights: the end points and the roots of
// P'_{N-1} (Newton, with P''_n (1 - x^2) = 2 x P'_n - n (n + 1) P_n), weights
// 2 / (N (N - 1) P_{N-1}(x)^2).
void gauss_lobatto(int N, double* x, double* w) {
  const int n = N - 1;
  for (int i = 0; i < N; ++i) {
    double t = -cos(M_PI * i / n);
    if (i == 0) t = -1.0;
    if (i == n) t = 1.0;
    for (int k = 0; k < 60 && i > 0 && i < n; ++k) {
      double p, dp;
      legendre_pair(n, t, &p, &dp);
      const double step = dp * (1.0 - t * t) / (2.0 * t * dp - n * (n + 1.0) * p);
      t -= step;
      if (fabs(step) <= 1e-17) break;
    }
    double p = (i == 0) ? ((n % 2) ? -1.0 : 1.0) : 1.0, dp;
    if (i > 0 && i < n) legendre_pair(n, t, &p, &dp);
    x[i] = t;
    w[i] = 2.0 / (N * (N - 1.0) * p * p);
  }
}

// Tables of the collocated scheme: Dhat[i][a] = w_a phi_i'(x_a)/w_i, e-+_i = phi_i(-+1).
void basis_tables(int N, const double* x, const double* w, double* Dhat, double* em, double* ep) {
  double lam[dgsrhd::kMaxN];
  for (int j = 0; j < N; ++j) {
    double prod = 1.0;
    for (int k = 0; k < N; ++k)
      if (k != j) prod *= (x[j] - x[k]);
    lam[j] = 1.0 / prod;
  }
  // Dm[a][j] = phi_j'(x_a)
  double Dm[dgsrhd::kMaxN][dgsrhd::kMaxN];
  for (int a = 0; a < N; ++a) {
    double diag = 0.0;
    for (int j = 0; j < N; ++j) {
      if (j == a) continue;
      Dm[a][j] = (lam[j] / lam[a]) / (x[a] - x[j]);
      diag -= Dm[a][j];
    }
    Dm[a][a] = diag;
  }
  for (int i = 0; i < N; ++i)
    for (int a = 0; a < N; ++a) Dhat[i * N + a] = (N == 1) ? 0.0 : w[a] * Dm[a][i] / w[i];
  for (int s = 0; s < 2; ++s) {
    const double xe = s ? 1.0 : -1.0;
    double* e = s ? ep : em;
    int hit = -1;  // a node on the end point (Gauss-Lobatto): the trace is that node's value
    for (int j = 0; j < N; ++j)
      if (x[j] == xe) hit = j;
    if (hit >= 0) {
      for (int i = 0; i < N; ++i) e[i] = (i == hit) ? 1.0 : 0.0;
      continue;
    }
    double den = 0.0;
    for (int j = 0; j < N; ++j) den += lam[j] / (xe - x[j]);
    for (int i = 0; i < N; ++i) e[i] = (lam[i] / (xe - x[i])) / den;
  }
}

int32_t cuda_status(cudaError_t e) { return e == cudaSuccess ? DGSRHD_OK : DGSRHD_ECUDA; }

int kernel_kind(Op op) {
  switch (op) {
    case Op::Volume: return DGSRHD_KERNEL_VOLUME;
    case Op::Face: return DGSRHD_KERNEL_FACE;
    case Op::Update: return DGSRHD_KERNEL_UPDATE;
    case Op::Enforce:
    case Op::Means:
    case Op::Limit: return DGSRHD_KERNEL_ENFORCE;
    default: return DGSRHD_KERNEL_VJP;
  }
}

cudaEvent_t pooled_event(dgsrhd_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t ev = c->event_pool.back();
    c->event_pool.pop_back();
    return ev;
  }
  cudaEvent_t ev = nullptr;
  cudaEventCreate(&ev);
  return ev;
}

// Launch bracketed by timing events when profiling is on.
template <class F>
cudaError_t timed_launch(dgsrhd_ctx* c, int kind, F&& launch) {
  if (!c->profiling) return launch();
  dgsrhd_ctx::TimedLaunch t{kind, pooled_event(c), pooled_event(c)};
  cudaEventRecord(t.start, c->stream);
  cudaError_t e = launch();
  cudaEventRecord(t.stop, c->stream);
  c->timed.push_back(t);
  return e;
}

cudaError_t run_stage(dgsrhd_ctx* c, StageArgs& a) {
  a.p = &c->p;
  a.stream = c->stream;
  a.split = c->cfg.precision == DGSRHD_PREC_SPLIT && !a.fp64_only;
  a.Fref = c->Fref;
  cudaError_t e = timed_launch(c, kernel_kind(a.op), [&]() {
    switch (c->dim) {
      case 1: return dgsrhd::dispatch_stage<1>(c->N, a);
      case 2: return dgsrhd::dispatch_stage<2>(c->N, a);
      default: return dgsrhd::dispatch_stage<3>(c->N, a);
    }
  });
  if (e == cudaSuccess) c->launches += 1;
  return e;
}

// R_vol and face traces, then face fluxes (the first two kernels of every RHS); rscale as in
// StageArgs (nonzero only when the update that follows is a stage given the same scale)
cudaError_t volume_and_faces(dgsrhd_ctx* c, const double* U, double rscale = 0.0) {
  StageArgs a{};
  a.op = Op::Volume;
  a.U = U;
  a.Rvol = c->Rv;
  a.Tr = c->Tr;
  a.rscale = rscale;
  cudaError_t e = run_stage(c, a);
  if (e != cudaSuccess) return e;
  c->c2p_calls += c->E * c->Nn;
  StageArgs f{};
  f.op = Op::Face;
  f.Tr = c->Tr;
  f.Fs = c->Fs;
  return run_stage(c, f);
}

// The limiter after a stage: element means, then the limit kernel (which also applies the
// physicality operator when it is enabled).
cudaError_t limit_stage(dgsrhd_ctx* c, double* U, double* s_out, double* theta_out = nullptr) {
  StageArgs m{};
  m.op = Op::Means;
  m.Uout = U;
  m.means = c->Mn;
  cudaError_t e = run_stage(c, m);
  if (e != cudaSuccess) return e;
  StageArgs l{};
  l.op = Op::Limit;
  l.Uout = U;
  l.means = c->Mn;
  l.enforce = c->cfg.enforce;
  l.s_out = s_out;
  l.theta_out = theta_out;
  return run_stage(c, l);
}

// Shu-Osher coefficients U^(k) = a_n U^n + b_k (U^(k-1) + dt R(U^(k-1)))
const double kAn[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.75, 1.0 / 3.0}};
const double kBk[3][3] = {{1.0, 0.0, 0.0}, {1.0, 0.5, 0.0}, {1.0, 0.25, 2.0 / 3.0}};

cudaError_t one_step(dgsrhd_ctx* c, double* U, double dt) {
  const int ns = c->cfg.rk_stages;
  for (int k = 0; k < ns; ++k) {
    const double* Uin = (k == 0) ? U : c->A;
    double* Uout = (k == ns - 1) ? U : c->A;
    const double rscale = kBk[ns - 1][k] * dt;  // b_k dt, folded into R_vol and the lift
    cudaError_t e = volume_and_faces(c, Uin, rscale);
    if (e != cudaSuccess) return e;
    StageArgs u{};
    u.op = Op::Update;
    u.Rvol = c->Rv;
    u.Fs = c->Fs;
    u.Un = U;
    u.Uk = Uin;
    u.Uout = Uout;
    u.a_n = kAn[ns - 1][k];
    u.b_k = kBk[ns - 1][k];
    u.dt = dt;
    u.rscale = rscale;
    u.mode = 1;
    u.enforce = c->cfg.enforce && !c->cfg.limiter;
    e = run_stage(c, u);
    if (e != cudaSuccess) return e;
    if (c->cfg.limiter) {
      e = limit_stage(c, Uout, nullptr);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// One step of a state in device-addressable host memory Uh: the stage-1 volume kernel reads it
// and copies it to Ud, every later read of U^n uses Ud, and the last update writes Uh.
cudaError_t one_step_host(dgsrhd_ctx* c, double* Uh, double dt) {
  const int ns = c->cfg.rk_stages;
  for (int k = 0; k < ns; ++k) {
    const double rscale = kBk[ns - 1][k] * dt;  // b_k dt, folded into R_vol and the lift
    StageArgs a{};
    a.op = Op::Volume;
    a.U = (k == 0) ? Uh : c->A;
    a.Rvol = c->Rv;
    a.Tr = c->Tr;
    a.Ucopy = (k == 0) ? c->Ud : nullptr;
    a.rscale = rscale;
    cudaError_t e = run_stage(c, a);
    if (e != cudaSuccess) return e;
    c->c2p_calls += c->E * c->Nn;
    StageArgs f{};
    f.op = Op::Face;
    f.Tr = c->Tr;
    f.Fs = c->Fs;
    if ((e = run_stage(c, f)) != cudaSuccess) return e;
    StageArgs u{};
    u.op = Op::Update;
    u.Rvol = c->Rv;
    u.Fs = c->Fs;
    u.Un = c->Ud;
    u.Uk = (k == 0) ? c->Ud : c->A;
    u.Uout = (k == ns - 1) ? Uh : c->A;
    u.a_n = kAn[ns - 1][k];
    u.b_k = kBk[ns - 1][k];
    u.dt = dt;
    u.rscale = rscale;
    u.mode = 1;
    u.enforce = c->cfg.enforce;
    if ((e = run_stage(c, u)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

bool valid_config(const dgsrhd_config* c) {
  if (!c) return false;
  if (c->dim < 1 || c->dim > 3) return false;
  if (c->degree < 0 || c->degree + 1 > dgsrhd::kMaxN) return false;
  // fewer than 2^30 elements: element and face indices then fit the kernels' 32-bit division
  long long E = 1;
  for (int d = 0; d < c->dim; ++d) {
    if (c->n_elem[d] < 1 || c->n_elem[d] >= (1LL << 30)) return false;
    E *= c->n_elem[d];
    if (E >= (1LL << 30)) return false;
  }
  for (int d = 0; d < c->dim; ++d) {
    if (!(c->hi[d] > c->lo[d])) return false;
    for (int s = 0; s < 2; ++s)
      if (c->bc[d][s] < 0 || c->bc[d][s] > DGSRHD_BC_REFLECT) return false;
    if ((c->bc[d][0] == DGSRHD_BC_PERIODIC) != (c->bc[d][1] == DGSRHD_BC_PERIODIC)) return false;
    for (int s = 0; s < 2; ++s)
      if (c->bc[d][s] == DGSRHD_BC_DIRICHLET) {
        const double* b = c->bc_state[d][s];
        if (!(b[0] > 0.0) || !(b[4] > 0.0) || !(b[1] * b[1] + b[2] * b[2] + b[3] * b[3] < 1.0))
          return false;
      }
  }
  if (c->eos != DGSRHD_EOS_IDEAL && c->eos != DGSRHD_EOS_TAUB_MATTHEWS) return false;
  if (c->eos == DGSRHD_EOS_IDEAL && !(c->gamma_ad > 1.0)) return false;
  if (c->c2p < 0 || c->c2p > 2) return false;
  if (!(c->c2p_rtol >= 0.0 && c->c2p_rtol < 1.0)) return false;
  if (c->flux != DGSRHD_FLUX_LLF && c->flux != DGSRHD_FLUX_HLL && c->flux != DGSRHD_FLUX_HLLC)
    return false;
  if (c->rk_stages < 1 || c->rk_stages > 3) return false;
  if (c->precision != DGSRHD_PREC_FP64 && c->precision != DGSRHD_PREC_SPLIT) return false;
  if (c->nodes != DGSRHD_NODES_GL && c->nodes != DGSRHD_NODES_GLL) return false;
  if (c->nodes == DGSRHD_NODES_GLL && c->degree < 1) return false;
  if (c->limiter < DGSRHD_LIMITER_NONE || c->limiter > DGSRHD_LIMITER_MINMOD) return false;
  if (c->enforce < 0 || c->enforce > DGSRHD_ENFORCE_FACES) return false;
  if (c->limiter && !(c->limiter_alpha >= 0.0)) return false;
  return true;
}

// q = umulhi(x, m) >> s with s = floor(log2 d), m = ceil(2^(32+s)/d) (0 for a power of two)
dgsrhd::FastDiv make_fastdiv(long long d) {
  dgsrhd::FastDiv f;
  unsigned s = 0;
  while ((2LL << s) <= d) ++s;
  f.s = s;
  const unsigned long long ud = (unsigned long long)d;
  f.m = (ud & (ud - 1)) == 0 ? 0u : (unsigned)(((1ULL << (32 + s)) + ud - 1) / ud);
  return f;
}

template <class T>
cudaError_t alloc(T** p, size_t n) {
  return cudaMalloc((void**)p, n * sizeof(T));
}

}  // namespace

extern "C" {

int32_t dgsrhd_create(const dgsrhd_config* cfg, void* stream, dgsrhd_ctx** out) {
  if (!out) return DGSRHD_EINVAL;
  *out = nullptr;
  if (!valid_config(cfg)) return DGSRHD_EINVAL;
  dgsrhd_ctx* c = new (std::nothrow) dgsrhd_ctx();
  if (!c) return DGSRHD_ENOMEM;
  c->cfg = *cfg;
  c->stream = (cudaStream_t)stream;
  c->dim = cfg->dim;
  c->N = cfg->degree + 1;
  long long ntr = 0, fs_total = 0;
  if (!dgsrhd::params_from_config(cfg, &c->p, &ntr, &fs_total, c->x)) {
    delete c;
    return DGSRHD_EINVAL;
  }
  Params& p = c->p;
  for (int d = 0; d < 3; ++d) c->dx[d] = d < c->dim ? (cfg->hi[d] - cfg->lo[d]) / (double)p.n[d] : 1.0;
  const long long E = p.E;
  c->E = E;
  c->Nn = p.Nn;
  c->nstate = 5 * E * p.Nn;
  c->fs_total = fs_total;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = alloc(&c->A, c->nstate);
  if (e == cudaSuccess) e = alloc(&c->Rv, c->nstate);
  if (e == cudaSuccess) e = alloc(&c->Tr, ntr);
  if (e == cudaSuccess) e = alloc(&c->Fs, fs_total);
  if (e == cudaSuccess && cfg->precision == DGSRHD_PREC_SPLIT) e = alloc(&c->Fref, 5LL * c->dim * E);
  if (e == cudaSuccess) e = alloc(&c->Ud, c->nstate);
  if (e == cudaSuccess) e = alloc(&c->Wv, (long long)dgsrhd::kNodePrim * E * p.Nn);
  if (e == cudaSuccess) e = alloc(&c->TrB, ntr);
  if (e == cudaSuccess) e = alloc(&c->Yb, c->nstate);
  if (e == cudaSuccess && cfg->limiter) e = alloc(&c->Yb2, c->nstate);
  if (e == cudaSuccess) e = alloc(&c->Gd, 2LL * c->dim * E * p.Nt);
  if (e == cudaSuccess && cfg->limiter) e = alloc(&c->Mn, 5LL * E);
  if (e == cudaSuccess) e = alloc(&c->stats, (size_t)dgsrhd::kStatCount * 64);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->stats, 0, sizeof(unsigned long long) * dgsrhd::kStatCount * 64, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    dgsrhd_destroy(c);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? DGSRHD_ENOMEM : DGSRHD_ECUDA;
  }
  p.stats = c->stats;
  *out = c;
  return DGSRHD_OK;
}

void dgsrhd_destroy(dgsrhd_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  for (auto& t : c->timed) {
    cudaEventDestroy(t.start);
    cudaEventDestroy(t.stop);
  }
  for (auto ev : c->event_pool) cudaEventDestroy(ev);
  cudaFree(c->A);
  cudaFree(c->Rv);
  cudaFree(c->Tr);
  cudaFree(c->Fs);
  cudaFree(c->Fref);
  cudaFree(c->Ud);
  cudaFree(c->Wv);
  cudaFree(c->TrB);
  cudaFree(c->Yb);
  cudaFree(c->Yb2);
  cudaFree(c->Gd);
  cudaFree(c->Mn);
  cudaFree(c->stats);
  delete c;
}

int32_t dgsrhd_set_stream(dgsrhd_ctx* c, void* stream) {
  if (!c) return DGSRHD_EINVAL;
  if ((cudaStream_t)stream != c->stream) {
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
  }
  c->stream = (cudaStream_t)stream;
  return DGSRHD_OK;
}

int32_t dgsrhd_state_shape(const dgsrhd_ctx* c, int64_t* nvar, int64_t* n_elem, int64_t* n_node) {
  if (!c) return DGSRHD_EINVAL;
  if (nvar) *nvar = 5;
  if (n_elem) *n_elem = c->E;
  if (n_node) *n_node = c->Nn;
  return DGSRHD_OK;
}

int32_t dgsrhd_node_coords(const dgsrhd_ctx* c, double* X) {
  if (!c || !X) return DGSRHD_EINVAL;
  const int N = c->N;
  for (long long e = 0; e < c->E; ++e) {
    for (int i = 0; i < c->Nn; ++i) {
      int ijk[3] = {i % N, (i / N) % N, i / (N * N)};
      for (int d = 0; d < c->dim; ++d) {
        const long long ce = (e / c->p.stride[d]) % c->p.n[d];
        X[((long long)d * c->E + e) * c->Nn + i] =
            c->cfg.lo[d] + ((double)ce + 0.5 * (1.0 + c->x[ijk[d]])) * c->dx[d];
      }
    }
  }
  return DGSRHD_OK;
}

int32_t dgsrhd_prim2cons(dgsrhd_ctx* c, const double* W, double* U) {
  if (!c || !W || !U) return DGSRHD_EINVAL;
  cudaError_t e = timed_launch(c, DGSRHD_KERNEL_POINTWISE, [&]() {
    return dgsrhd::launch_prim2cons(c->p, c->stream, c->E * c->Nn, W, U);
  });
  if (e == cudaSuccess) c->launches += 1;
  return cuda_status(e);
}

int32_t dgsrhd_con2prim(dgsrhd_ctx* c, const double* U, double* W, int32_t* iters) {
  if (!c || !U || !W) return DGSRHD_EINVAL;
  cudaError_t e = timed_launch(c, DGSRHD_KERNEL_POINTWISE, [&]() {
    return dgsrhd::launch_con2prim(c->p, c->stream, c->E * c->Nn, U, W, iters);
  });
  if (e == cudaSuccess) {
    c->launches += 1;
    c->c2p_calls += c->E * c->Nn;
  }
  return cuda_status(e);
}

int32_t dgsrhd_rhs(dgsrhd_ctx* c, const double* U, double* R) {
  if (!c || !U || !R || U == R) return DGSRHD_EINVAL;
  cudaError_t e = volume_and_faces(c, U);
  if (e != cudaSuccess) return DGSRHD_ECUDA;
  StageArgs u{};
  u.op = Op::Update;
  u.Rvol = c->Rv;
  u.Fs = c->Fs;
  u.Uout = R;
  u.mode = 0;
  return cuda_status(run_stage(c, u));
}

int32_t dgsrhd_enforce(dgsrhd_ctx* c, double* U, double* s_out) {
  if (!c || !U) return DGSRHD_EINVAL;
  StageArgs a{};
  a.op = Op::Enforce;
  a.Uout = U;
  a.s_out = s_out;
  return cuda_status(run_stage(c, a));
}

int32_t dgsrhd_step(dgsrhd_ctx* c, double* U, double dt, int32_t nsteps) {
  if (!c || !U || nsteps < 0 || !(dt >= 0.0)) return DGSRHD_EINVAL;
  if (nsteps == 0) return DGSRHD_OK;
  const long long per_step = (c->cfg.limiter ? 5LL : 3LL) * c->cfg.rk_stages;
  if (c->stream == nullptr || c->profiling) {
    // the legacy stream cannot be captured, and timed kernels are launched one by one
    for (int s = 0; s < nsteps; ++s) {
      cudaError_t e = one_step(c, U, dt);
      if (e != cudaSuccess) return DGSRHD_ECUDA;
    }
    return DGSRHD_OK;
  }
  dgsrhd_ctx::StepGraph* hit = nullptr;
  for (auto& g : c->graphs)
    if (g.U == U && g.dt == dt) hit = &g;
  if (!hit) {
    constexpr size_t kMaxGraphs = 4;
    if (c->graphs.size() == kMaxGraphs) {
      size_t lru = 0;
      for (size_t i = 1; i < c->graphs.size(); ++i)
        if (c->graphs[i].used < c->graphs[lru].used) lru = i;
      cudaGraphExecDestroy(c->graphs[lru].exec);
      c->graphs.erase(c->graphs.begin() + lru);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return DGSRHD_ECUDA;
    const long long l0 = c->launches, k0 = c->c2p_calls;
    cudaError_t e1 = one_step(c, U, dt);
    e = cudaStreamEndCapture(c->stream, &g);
    c->launches = l0;  // captured, not launched
    c->c2p_calls = k0;
    if (e1 != cudaSuccess || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return DGSRHD_ECUDA;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return DGSRHD_ECUDA;
    c->graphs.push_back({exec, dt, U, 0});
    hit = &c->graphs.back();
  }
  hit->used = ++c->graph_clock;
  for (int s = 0; s < nsteps; ++s) {
    cudaError_t e = cudaGraphLaunch(hit->exec, c->stream);
    if (e != cudaSuccess) return DGSRHD_ECUDA;
  }
  c->launches += per_step * nsteps;
  c->c2p_calls += (long long)nsteps * c->cfg.rk_stages * c->E * c->Nn;
  return DGSRHD_OK;
}

int32_t dgsrhd_step_host(dgsrhd_ctx* c, double* U_host, double dt, int32_t nsteps) {
  if (!c || !U_host) return DGSRHD_EINVAL;
  // Pinned host memory that the GPU can address: the first kernel of every step reads the state
  // from it (over the host link, overlapped with the kernel's FP64 work) and keeps a device
  // copy; the last kernel writes the new state back to it.
  cudaPointerAttributes at;
  double* Uh_dev = nullptr;
  if (cudaPointerGetAttributes(&at, U_host) == cudaSuccess && at.type == cudaMemoryTypeHost &&
      at.devicePointer && c->cfg.precision == DGSRHD_PREC_FP64 && !c->cfg.limiter)
    Uh_dev = static_cast<double*>(at.devicePointer);
  cudaGetLastError();  // clears the error an unregistered pointer leaves
  if (Uh_dev) {
    for (int s = 0; s < nsteps; ++s)
      if (one_step_host(c, Uh_dev, dt) != cudaSuccess) return DGSRHD_ECUDA;
    return cuda_status(cudaStreamSynchronize(c->stream));
  }
  const size_t bytes = sizeof(double) * c->nstate;
  if (cudaMemcpyAsync(c->Ud, U_host, bytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
    return DGSRHD_ECUDA;
  int32_t st = dgsrhd_step(c, c->Ud, dt, nsteps);
  if (st != DGSRHD_OK) return st;
  if (cudaMemcpyAsync(U_host, c->Ud, bytes, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    return DGSRHD_ECUDA;
  return cuda_status(cudaStreamSynchronize(c->stream));
}

int32_t dgsrhd_cfl_dt(const dgsrhd_ctx* c, double cfl, double* dt) {
  if (!c || !dt || !(cfl > 0.0)) return DGSRHD_EINVAL;
  double s = 0.0;
  for (int d = 0; d < c->dim; ++d) s += 1.0 / c->dx[d];
  *dt = cfl / ((2.0 * c->cfg.degree + 1.0) * s);
  return DGSRHD_OK;
}

int32_t dgsrhd_get_stats(dgsrhd_ctx* c, dgsrhd_stats* out, int32_t reset) {
  if (!c || !out) return DGSRHD_EINVAL;
  unsigned long long h[dgsrhd::kStatCount * 64];
  const size_t bytes = sizeof h;
  if (cudaMemcpyAsync(h, c->stats, bytes, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    return DGSRHD_ECUDA;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return DGSRHD_ECUDA;
  unsigned long long v[dgsrhd::kStatCount] = {0};
  for (int k = 0; k < dgsrhd::kStatCount; ++k)
    for (int s = 0; s < 64; ++s) {
      const unsigned long long x = h[k * 64 + s];
      if (k == dgsrhd::kStatItersMax)
        v[k] = x > v[k] ? x : v[k];
      else
        v[k] += x;
    }
  out->c2p_calls = c->c2p_calls;
  out->c2p_iters_total = (int64_t)v[dgsrhd::kStatItersTotal];
  out->c2p_iters_max = (int64_t)v[dgsrhd::kStatItersMax];
  out->c2p_nonconverged = (int64_t)v[dgsrhd::kStatNonConv];
  out->c2p_invalid_input = (int64_t)v[dgsrhd::kStatInvalid];
  out->face_guard_hits = (int64_t)v[dgsrhd::kStatFaceGuard];
  out->enforced_cells = (int64_t)v[dgsrhd::kStatEnforced];
  out->mean_inadmissible_cells = (int64_t)v[dgsrhd::kStatMeanBad];
  out->limited_cells = (int64_t)v[dgsrhd::kStatLimited];
  if (reset) {
    if (cudaMemsetAsync(c->stats, 0, bytes, c->stream) != cudaSuccess) return DGSRHD_ECUDA;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return DGSRHD_ECUDA;
    c->c2p_calls = 0;
  }
  if (out->c2p_invalid_input) return DGSRHD_EBADSTATE;
  if (out->c2p_nonconverged) return DGSRHD_EC2P_NOCONV;
  if (out->mean_inadmissible_cells) return DGSRHD_EUNPHYS_MEAN;
  return DGSRHD_OK;
}

int64_t dgsrhd_kernel_launches(const dgsrhd_ctx* c) { return c ? c->launches : 0; }

int32_t dgsrhd_set_profiling(dgsrhd_ctx* c, int32_t enable) {
  if (!c) return DGSRHD_EINVAL;
  c->profiling = enable != 0;
  return DGSRHD_OK;
}

int32_t dgsrhd_kernel_times(dgsrhd_ctx* c, double* ms, int64_t* counts, int32_t reset) {
  if (!c || !ms || !counts) return DGSRHD_EINVAL;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return DGSRHD_ECUDA;
  for (int k = 0; k < DGSRHD_KERNEL_KINDS; ++k) {
    ms[k] = 0.0;
    counts[k] = 0;
  }
  for (auto& t : c->timed) {
    float v = 0.0f;
    if (cudaEventElapsedTime(&v, t.start, t.stop) != cudaSuccess) return DGSRHD_ECUDA;
    ms[t.kind] += v;
    counts[t.kind] += 1;
  }
  if (reset) {
    for (auto& t : c->timed) {
      c->event_pool.push_back(t.start);
      c->event_pool.push_back(t.stop);
    }
    c->timed.clear();
  }
  return DGSRHD_OK;
}

}  // extern "C"

namespace {

// Reverse sweep of the RHS.  `saved` (nullable) holds the nodal (rho, u, P) and the face traces
// of the forward evaluation at U (written by dgsrhd_step_stage); without it the forward volume
// kernel is re-run to provide them.
long long trace_doubles(const dgsrhd_ctx* c) { return 2LL * c->dim * 5 * c->E * c->p.Nt; }
// face-state tape: 2 kFaceTape doubles per face point, face points = fs_total / 5
long long tape_doubles(const dgsrhd_ctx* c) { return (c->fs_total / 5) * 2 * dgsrhd::kFaceTape; }
// face-guard flags: one byte per face point of every element, rounded up to whole doubles
long long guard_doubles(const dgsrhd_ctx* c) { return (2LL * c->dim * c->E * c->p.Nt + 7) / 8; }

// Sections of a stage's saved forward quantities: nodal (rho, u, P), face traces, face-state
// tape, face-guard flags.
struct Saved {
  double* W;
  double* Tr;
  double* tape;
  unsigned char* guard;
  double* theta;  // the limiter's factor per element (limited configurations)
};
Saved saved_sections(const dgsrhd_ctx* c, double* save) {
  Saved v{};
  if (!save) return v;
  v.W = save;
  v.Tr = save + (long long)dgsrhd::kNodePrim * c->E * c->Nn;
  v.tape = v.Tr + trace_doubles(c);
  v.guard = reinterpret_cast<unsigned char*>(v.tape + tape_doubles(c));
  v.theta = c->cfg.limiter ? v.tape + tape_doubles(c) + guard_doubles(c) : nullptr;
  return v;
}

// (dR/dU)^T R_bar -> U_bar; with Ukb set, the stage combination Unb += a_n R_bar,
// Ukb += b_k (R_bar + dt U_bar) replaces the write of U_bar.
int32_t rhs_vjp_core(dgsrhd_ctx* c, const double* U, const double* R_bar, double* U_bar,
                     const double* saved, double* Unb = nullptr, double* Ukb = nullptr,
                     double a_n = 0.0, double b_k = 0.0, double dt = 0.0) {
  Saved sv = saved_sections(c, const_cast<double*>(saved));
  if (!saved) {
    StageArgs v{};
    v.op = Op::Volume;
    v.fp64_only = 1;
    v.U = U;
    v.Rvol = c->Rv;
    v.Tr = c->Tr;
    v.Wstore = c->Wv;
    v.guard = c->Gd;
    if (run_stage(c, v) != cudaSuccess) return DGSRHD_ECUDA;
    c->c2p_calls += c->E * c->Nn;
    sv.W = c->Wv;
    sv.Tr = c->Tr;
    sv.tape = nullptr;  // the face reverse sweep evaluates its roots and reciprocals itself
    sv.guard = c->Gd;
  }
  StageArgs f{};
  f.op = Op::VjpFace;
  f.Tr = sv.Tr;
  f.tape = sv.tape;
  f.Rbar = R_bar;
  f.TrBar = c->TrB;
  if (run_stage(c, f) != cudaSuccess) return DGSRHD_ECUDA;
  StageArgs n{};
  n.op = Op::VjpNode;
  n.U = U;
  n.Wstore = sv.W;
  n.guard = sv.guard;
  n.Rbar = R_bar;
  n.TrBar = c->TrB;
  n.Ubar = U_bar;
  n.Unb = Unb;
  n.Ukb = Ukb;
  n.a_n = a_n;
  n.b_k = b_k;
  n.dt = dt;
  return cuda_status(run_stage(c, n));
}


}  // namespace

extern "C" {

int32_t dgsrhd_rhs_vjp(dgsrhd_ctx* c, const double* U, const double* R_bar, double* U_bar) {
  if (!c || !U || !R_bar || !U_bar || U_bar == U || U_bar == R_bar) return DGSRHD_EINVAL;
  return rhs_vjp_core(c, U, R_bar, U_bar, nullptr);
}

int32_t dgsrhd_stage_save_size(const dgsrhd_ctx* c, int64_t* n) {
  if (!c || !n) return DGSRHD_EINVAL;
  *n = (long long)dgsrhd::kNodePrim * c->E * c->Nn + trace_doubles(c) + tape_doubles(c) +
       guard_doubles(c) + (c->cfg.limiter ? c->E : 0);
  return DGSRHD_OK;
}

int32_t dgsrhd_enforce_vjp(dgsrhd_ctx* c, const double* s, const double* Ut_bar, double* U_bar) {
  if (!c || !s || !Ut_bar || !U_bar) return DGSRHD_EINVAL;
  StageArgs a{};
  a.op = Op::EnforceVjp;
  a.s_in = s;
  a.Tbar = Ut_bar;
  a.Ubar = U_bar;
  return cuda_status(run_stage(c, a));
}

int32_t dgsrhd_step_stage(dgsrhd_ctx* c, const double* Un, const double* Uk, double* Uout,
                          int32_t stage, double dt, double* s_out, double* save) {
  if (!c || !Un || !Uk || !Uout || stage < 0 || stage >= c->cfg.rk_stages || !(dt >= 0.0))
    return DGSRHD_EINVAL;
  const int ns = c->cfg.rk_stages;
  const Saved sv = saved_sections(c, save);
  StageArgs v{};
  v.op = Op::Volume;
  v.U = Uk;
  v.Rvol = c->Rv;
  v.Tr = save ? sv.Tr : c->Tr;
  v.Wstore = sv.W;
  v.guard = sv.guard;
  v.rscale = kBk[ns - 1][stage] * dt;  // b_k dt, as in a step
  if (save) v.fp64_only = 1;  // the saved quantities feed the FP64 reverse sweep
  if (run_stage(c, v) != cudaSuccess) return DGSRHD_ECUDA;
  c->c2p_calls += c->E * c->Nn;
  StageArgs f{};
  f.op = Op::Face;
  f.fp64_only = v.fp64_only;  // the update below reads the fluxes in the same precision
  f.Tr = v.Tr;
  f.Fs = c->Fs;
  f.tape = sv.tape;
  if (run_stage(c, f) != cudaSuccess) return DGSRHD_ECUDA;
  StageArgs u{};
  u.op = Op::Update;
  u.fp64_only = v.fp64_only;
  u.Rvol = c->Rv;
  u.Fs = c->Fs;
  u.Un = Un;
  u.Uk = Uk;
  u.Uout = Uout;
  u.a_n = kAn[ns - 1][stage];
  u.b_k = kBk[ns - 1][stage];
  u.dt = dt;
  u.rscale = v.rscale;
  u.mode = 1;
  u.enforce = c->cfg.enforce && !c->cfg.limiter;
  u.s_out = s_out;
  if (run_stage(c, u) != cudaSuccess) return DGSRHD_ECUDA;
  if (c->cfg.limiter) return cuda_status(limit_stage(c, Uout, s_out, sv.theta));
  return DGSRHD_OK;
}

int32_t dgsrhd_stage_vjp(dgsrhd_ctx* c, const double* Uk, const double* s, const double* saved,
                         const double* Z_bar, double* Un_bar, double* Uk_bar, int32_t stage,
                         double dt) {
  if (!c || !Uk || !Z_bar || !Un_bar || !Uk_bar || stage < 0 || stage >= c->cfg.rk_stages)
    return DGSRHD_EINVAL;
  if (Z_bar == Un_bar || Z_bar == Uk_bar) return DGSRHD_EINVAL;
  // the limiter's factors exist only in the saved forward quantities (recomputing them would
  // need U^n)
  if (c->cfg.limiter && !saved) return DGSRHD_EINVAL;
  const int ns = c->cfg.rk_stages;
  const double* Yb = Z_bar;
  if (c->cfg.enforce && s) {
    int32_t st = dgsrhd_enforce_vjp(c, s, Z_bar, c->Yb);
    if (st != DGSRHD_OK) return st;
    Yb = c->Yb;
  }
  if (c->cfg.limiter) {
    // U_i <- mean + theta (U_i - mean) with theta frozen: the same linear map as the operator's
    Saved sv = saved_sections(c, const_cast<double*>(saved));
    double* out = (Yb == c->Yb) ? c->Yb2 : c->Yb;
    int32_t st = dgsrhd_enforce_vjp(c, sv.theta, Yb, out);
    if (st != DGSRHD_OK) return st;
    Yb = out;
  }
  // the node reverse sweep adds a_n Yb to Un_bar and b_k (Yb + dt (dR/dU)^T Yb) to Uk_bar
  const double a_n = kAn[ns - 1][stage], b_k = kBk[ns - 1][stage];
  return rhs_vjp_core(c, Uk, Yb, nullptr, saved, Un_bar, Uk_bar, a_n, b_k, dt);
}

int32_t dgsrhd_con2prim_vjp(dgsrhd_ctx* c, const double* U, const double* W_bar, double* U_bar) {
  if (!c || !U || !W_bar || !U_bar) return DGSRHD_EINVAL;
  cudaError_t e = timed_launch(c, DGSRHD_KERNEL_VJP, [&]() {
    return dgsrhd::launch_con2prim_vjp(c->p, c->stream, c->E * c->Nn, U, W_bar, U_bar);
  });
  if (e == cudaSuccess) c->launches += 1;
  return cuda_status(e);
}

int32_t dgsrhd_mean_square_velocity(dgsrhd_ctx* c, const double* U, int32_t axis, double* out) {
  if (!c || !U || !out || axis < 0 || axis > 2) return DGSRHD_EINVAL;
  const long long n = c->E * c->Nn;
  const int blocks = (int)std::min<long long>(1024, (n + 255) / 256);
  cudaError_t e = timed_launch(c, DGSRHD_KERNEL_POINTWISE, [&]() {
    return dgsrhd::launch_velocity_square(c->p, c->stream, n, (int)c->Nn, U, axis, c->Rv, blocks);
  });
  if (e != cudaSuccess) return DGSRHD_ECUDA;
  c->launches += 1;
  std::vector<double> part((size_t)blocks);
  e = cudaMemcpyAsync(part.data(), c->Rv, sizeof(double) * blocks, cudaMemcpyDeviceToHost,
                      c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return DGSRHD_ECUDA;
  double sum = 0.0, jac = 1.0, vol = 1.0;
  for (int b = 0; b < blocks; ++b) sum += part[(size_t)b];
  for (int d = 0; d < c->dim; ++d) {
    jac *= 0.5 * c->dx[d];
    vol *= c->cfg.hi[d] - c->cfg.lo[d];
  }
  *out = sum * jac / vol;
  return DGSRHD_OK;
}

int32_t dgsrhd_math_check(const double* x, int64_t n, double* out, void* stream) {
  if (!x || !out || n < 0) return DGSRHD_EINVAL;
  return cuda_status(dgsrhd::launch_math_check((cudaStream_t)stream, n, x, out));
}

int32_t dgsrhd_arith_probe(int32_t kind, int64_t iters, double* sink, int64_t threads,
                           void* stream, int64_t* ops) {
  if (kind < 0 || kind >= DGSRHD_PROBE_KINDS || iters < 1 || !sink || threads < 256 ||
      threads % 256 != 0 || threads > (int64_t)256 * 65535)
    return DGSRHD_EINVAL;
  if (ops) *ops = 4 * threads * iters;
  return cuda_status(dgsrhd::launch_fp64_probe((cudaStream_t)stream, kind, iters, threads, sink));
}

const char* dgsrhd_status_string(int32_t s) {
  switch (s) {
    case DGSRHD_OK: return "ok";
    case DGSRHD_EINVAL: return "invalid argument";
    case DGSRHD_ECUDA: return "CUDA error";
    case DGSRHD_ENOMEM: return "out of device memory";
    case DGSRHD_EC2P_NOCONV: return "con2prim did not converge";
    case DGSRHD_EUNPHYS_MEAN: return "inadmissible element mean";
    case DGSRHD_EBADSTATE: return "invalid conserved state";
    default: return "unknown status";
  }
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Launch parameters of a configuration: mesh, face-flux layout, method choices and the basis
// tables.  dgsrhd_create and the static-scratch right-hand side both take them from here.
// ---------------------------------------------------------------------------------------
namespace dgsrhd {

bool params_from_config(const dgsrhd_config* cfg, Params* out, long long* n_trace,
                        long long* n_face_flux, double* nodes) {
  if (!valid_config(cfg) || !out) return false;
  Params p;
  memset(&p, 0, sizeof p);
  const int dim = cfg->dim, N = cfg->degree + 1;
  p.dim = dim;
  p.N = N;
  p.Nn = 1;
  p.Nt = 1;
  for (int d = 0; d < dim; ++d) p.Nn *= N;
  for (int d = 0; d < dim - 1; ++d) p.Nt *= N;
  long long E = 1;
  for (int d = 0; d < 3; ++d) {
    p.n[d] = d < dim ? cfg->n_elem[d] : 1;
    p.stride[d] = E;
    E *= p.n[d];
    const double dx = d < dim ? (cfg->hi[d] - cfg->lo[d]) / (double)p.n[d] : 1.0;
    p.inv_half_dx[d] = 2.0 / dx;
  }
  p.E = E;
  for (int d = 0; d < 3; ++d) {
    p.ndiv[d] = make_fastdiv(p.n[d]);
    p.sdiv[d] = make_fastdiv(p.stride[d]);
  }
  long long off = 0;
  for (int d = 0; d < 3; ++d) {
    if (d < dim) {
      p.nface[d] = E + (cfg->bc[d][0] == DGSRHD_BC_PERIODIC ? 0 : E / p.n[d]);
      p.fs_off[d] = off;
      off += 5 * p.nface[d] * p.Nt;
    }
    for (int s = 0; s < 2; ++s) {
      p.bc[d][s] = d < dim ? cfg->bc[d][s] : 0;
      const double* b = cfg->bc_state[d][s];
      const double v2 = b[1] * b[1] + b[2] * b[2] + b[3] * b[3];
      const double lor = (v2 < 1.0) ? 1.0 / sqrt(1.0 - v2) : 1.0;
      p.ghost[d][s][0] = b[0];
      for (int k = 1; k < 4; ++k) p.ghost[d][s][k] = lor * b[k];
      p.ghost[d][s][4] = b[4];
    }
  }
  p.eos = cfg->eos;
  p.gamma_ad = cfg->gamma_ad;
  p.alpha = cfg->eos == DGSRHD_EOS_IDEAL ? cfg->gamma_ad / (cfg->gamma_ad - 1.0) : 0.0;
  {
    const double G = cfg->gamma_ad;
    p.gm1 = G - 1.0;
    p.gm1sq = p.gm1 * p.gm1;
    p.m2G = -2.0 * G;
    p.m2Ggm1 = -2.0 * G * p.gm1;
    p.G2 = G * G;
    p.tgm1 = 2.0 * p.gm1;
    p.amG = p.alpha - G;
  }
  p.c2p = cfg->c2p == DGSRHD_C2P_DEFAULT ? (cfg->eos == DGSRHD_EOS_IDEAL ? 0 : 1) : cfg->c2p;
  p.max_iter = cfg->c2p_max_iter > 0 ? cfg->c2p_max_iter : (cfg->eos == DGSRHD_EOS_IDEAL ? 30 : 100);
  p.c2p_rtol = cfg->c2p_rtol;
  p.flux = cfg->flux;
  p.enforce_faces = cfg->enforce == DGSRHD_ENFORCE_FACES;
  {
    double h = 1e300;
    for (int d = 0; d < cfg->dim; ++d) h = fmin(h, (cfg->hi[d] - cfg->lo[d]) / (double)cfg->n_elem[d]);
    p.limiter = cfg->limiter;
    // scaling limiter: bound relaxation alpha h^(3/2); minmod: TVB threshold M h^2
    p.lim_alpha = cfg->limiter == DGSRHD_LIMITER_SCALING  ? cfg->limiter_alpha * pow(h, 1.5)
                  : cfg->limiter == DGSRHD_LIMITER_MINMOD ? cfg->limiter_alpha * h * h
                                                          : 0.0;
  }
  double x[kMaxN];
  if (cfg->nodes == DGSRHD_NODES_GLL)
    gauss_lobatto(N, x, p.w);
  else
    gauss_legendre(N, x, p.w);
  basis_tables(N, x, p.w, p.Dhat, p.em, p.ep);
  for (int i = 0; i < N; ++i) {
    p.lm[i] = p.em[i] / p.w[i];
    p.lp[i] = p.ep[i] / p.w[i];
    for (int d = 0; d < dim; ++d) {
      p.slm[d][i] = p.inv_half_dx[d] * p.lm[i];
      p.slp[d][i] = p.inv_half_dx[d] * p.lp[i];
    }
  }
  p.wsum = (double)(1 << dim);
  *out = p;
  if (nodes)
    for (int i = 0; i < N; ++i) nodes[i] = x[i];
  if (n_trace) *n_trace = 2LL * dim * 5 * E * p.Nt;
  if (n_face_flux) *n_face_flux = off;
  return true;
}

}  // namespace dgsrhd
