/*
 * dgsrhd: discontinuous-Galerkin special-relativistic hydrodynamics on one GPU (sm_103a).
 *
 * C ABI of the hot path of arXiv 2205.00095 (Glines et al., "A Robust, Performance-Portable
 * Discontinuous Galerkin Method for Relativistic Hydrodynamics"): conserved-to-primitive
 * recovery at the nodes, the nodal DG right-hand side with LLF/HLL/HLLC face fluxes, the
 * limiters and the physicality-enforcing operator, SSP Runge-Kutta steps, a split-precision
 * form, and the vector-Jacobian products of the right-hand side and of whole stages.
 * Units c = 1.
 *
 * Data layout (every state array):
 *   contiguous FP64, structure of arrays [var][elem][node];
 *   elem = ex + nx * (ey + ny * ez)              (x fastest)
 *   node = a + N * (b + N * c), N = degree + 1   (tensor nodes, Gauss-Legendre by default or
 *                                                 Gauss-Lobatto-Legendre, x fastest)
 *   conserved U: var = (D, S_x, S_y, S_z, tau), tau = E - D   (Eq. primitive_to_conserved)
 *   primitive W: var = (rho, v_x, v_y, v_z, P)                 (Sec. 2.1)
 * Five variables are carried in every dimension.
 *
 * Memory: arrays passed to the calls are caller-owned DEVICE pointers (except where a
 * name ends in _host).  The library owns only the scratch buffers it allocates in
 * dgsrhd_create and frees in dgsrhd_destroy; no other call allocates.
 *
 * Streams and errors: every call is ordered on the context's stream and returns before the
 * GPU work ends.  Argument errors return DGSRHD_EINVAL synchronously; launch failures return
 * DGSRHD_ECUDA.  Problems found on the device (non-converged or invalid con2prim,
 * inadmissible element means) are counted in device counters and reported by
 * dgsrhd_get_stats, which synchronises the stream.  No kernel traps.
 *
 * Threads: a context is used by one host thread at a time (its scratch, counters and cached
 * CUDA graphs are not guarded); distinct contexts are independent.
 */
#ifndef DGSRHD_H
#define DGSRHD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define DGSRHD_OK 0
#define DGSRHD_EINVAL 1          /* bad argument or configuration */
#define DGSRHD_ECUDA 2           /* a CUDA call failed */
#define DGSRHD_ENOMEM 3          /* scratch allocation failed in dgsrhd_create */
#define DGSRHD_EC2P_NOCONV 4     /* get_stats: some con2prim did not converge */
#define DGSRHD_EUNPHYS_MEAN 5    /* get_stats: some element mean was inadmissible */
#define DGSRHD_EBADSTATE 6       /* get_stats: some node held an invalid conserved state */

/* equation of state (Sec. 2.2) */
#define DGSRHD_EOS_IDEAL 0
#define DGSRHD_EOS_TAUB_MATTHEWS 1

/* conserved-to-primitive solver (Sec. 3) */
#define DGSRHD_C2P_ANALYTIC 0    /* ideal: quartic closed form; TM: cubic closed form */
#define DGSRHD_C2P_ITERATIVE 1   /* ideal: Newton on the Riccardi quartic; TM: Brent */
#define DGSRHD_C2P_DEFAULT 2     /* ideal -> analytic, Taub-Matthews -> iterative */

/* numerical flux (Sec. 2.4) */
#define DGSRHD_FLUX_LLF 0
#define DGSRHD_FLUX_HLL 1
#define DGSRHD_FLUX_HLLC 2       /* HLL with the contact restored (the relativistic HLLC of the
                                    literature the paper cites) */

/* boundary condition per side */
#define DGSRHD_BC_PERIODIC 0     /* both sides of an axis must be periodic together */
#define DGSRHD_BC_DIRICHLET 1    /* ghost state = bc_state (rho, vx, vy, vz, P) */
#define DGSRHD_BC_OUTFLOW 2      /* ghost state = the interior face trace */
#define DGSRHD_BC_REFLECT 3      /* reflecting wall: the interior trace with its normal velocity
                                    reversed */

/* node family of the collocated nodal basis (the paper's node set is unnamed: Gauss-Legendre
 * is the default; Gauss-Lobatto-Legendre puts nodes on the faces, so the face traces are nodal
 * values that the physicality operator covers, at the price of an inexact (degree 2N - 3)
 * collocated quadrature) */
#define DGSRHD_NODES_GL 0
#define DGSRHD_NODES_GLL 1

/* limiter after every RK stage, before the physicality operator (Sec. 2.3 names the limiters of
 * Moe et al. and the minmod limiter, printing neither); both scale each element toward its mean
 * by one factor theta, so admissible nodes stay admissible and the mean is kept */
#define DGSRHD_LIMITER_NONE 0
#define DGSRHD_LIMITER_SCALING 1 /* theta keeps nodal and face values within the face
                                    neighbours' means widened by limiter_alpha h^(3/2) */
#define DGSRHD_LIMITER_MINMOD 2  /* theta keeps every face-mean deviation within the minmod bound
                                    of the neighbour-mean differences; deviations below
                                    limiter_alpha h^2 (the TVB constant M) are left alone */

/* physicality operator (Sec. 2.5) after every RK stage */
#define DGSRHD_ENFORCE_OFF 0
#define DGSRHD_ENFORCE_NODES 1   /* the paper's operator: s = min over the element's nodes */
#define DGSRHD_ENFORCE_FACES 2   /* the minimum also over the face points of the element's conserved
                                    polynomial (sum_a phi_a(-+1) U_a along each normal line), which
                                    the same s smooths toward the mean, so the polynomial is left
                                    admissible at the faces too (with Gauss-Legendre nodes the
                                    faces hold no node) */

/* arithmetic of the basis contractions */
#define DGSRHD_PREC_FP64 0
#define DGSRHD_PREC_SPLIT 1      /* split precision: the volume term and face traces as 3xTF32
                                    tensor-core products and the lift as FP32 FMAs, all on
                                    deviations from a per-element reference; FP64 elsewhere */
#define DGSRHD_PREC_3XTF32 DGSRHD_PREC_SPLIT /* the same */
/* No BF16x3 precision is offered, deliberately: its two-part split of each operand keeps 16
 * significant bits against 3xTF32's 22, and the tensor-core contractions are not what bounds the
 * split kernels (the FP64 con2prim and fluxes are), so it would lose accuracy for no speed.  The
 * code 2 is rejected with DGSRHD_EINVAL like any other unknown precision. */

typedef struct dgsrhd_config {
  int32_t dim;                 /* 1, 2 or 3 */
  int32_t degree;              /* p in 0..4 (1..4 for Gauss-Lobatto); N = p + 1 nodes per axis */
  int64_t n_elem[3];           /* elements per axis (unused axes: 1); fewer than 2^30 in total */
  double lo[3], hi[3];         /* domain box */
  int32_t eos;                 /* DGSRHD_EOS_* */
  double gamma_ad;             /* adiabatic index of the ideal EOS (ignored for TM) */
  int32_t c2p;                 /* DGSRHD_C2P_* */
  int32_t c2p_max_iter;        /* <= 0: 30 Newton / 100 Brent iterations */
  double c2p_rtol;             /* 0: the iterative solvers stop at their rounding-level rules;
                                  in (0, 1): they also stop once Newton's step, or Brent's
                                  bracket, is within c2p_rtol of the iterate */
  int32_t flux;                /* DGSRHD_FLUX_* */
  int32_t rk_stages;           /* 1 (forward Euler), 2 (SSPRK2), 3 (SSPRK3) */
  int32_t bc[3][2];            /* DGSRHD_BC_* for the low and high side of each axis */
  double bc_state[3][2][5];    /* Dirichlet primitive (rho, vx, vy, vz, P) per side */
  int32_t enforce;             /* DGSRHD_ENFORCE_*: physicality operator after every RK stage */
  int32_t precision;           /* DGSRHD_PREC_* */
  int32_t nodes;               /* DGSRHD_NODES_*: node family of the collocated basis */
  int32_t limiter;             /* DGSRHD_LIMITER_* */
  double limiter_alpha;        /* scaling: bound relaxation limiter_alpha h^(3/2); minmod: TVB
                                  constant M, threshold M h^2 (h the smallest element width) */
} dgsrhd_config;

typedef struct dgsrhd_stats {
  int64_t c2p_calls;               /* node recoveries since the last reset */
  int64_t c2p_iters_total;         /* iterations of the iterative solvers */
  int64_t c2p_iters_max;
  int64_t c2p_nonconverged;        /* iteration cap hit / closed form broke down */
  int64_t c2p_invalid_input;       /* D <= 0, q <= 0 or non-finite conserved state */
  int64_t face_guard_hits;         /* face traces with rho <= 0 or P <= 0 replaced */
  int64_t enforced_cells;          /* elements smoothed by the physicality operator */
  int64_t mean_inadmissible_cells; /* flagged elements whose mean was inadmissible */
  int64_t limited_cells;           /* elements scaled towards their mean by the limiter */
} dgsrhd_stats;

typedef struct dgsrhd_ctx dgsrhd_ctx;

/* Create a solver for one mesh and method choice on the current CUDA device.  `stream` is a
 * cudaStream_t (NULL: the legacy default stream).  Allocates all scratch (about 8x the state
 * size).  Returns DGSRHD_EINVAL for an invalid configuration, DGSRHD_ENOMEM if scratch cannot
 * be allocated. */
int32_t dgsrhd_create(const dgsrhd_config* cfg, void* stream, dgsrhd_ctx** out);

/* Free the scratch and the context (synchronises its stream). NULL is ignored. */
void dgsrhd_destroy(dgsrhd_ctx* ctx);

/* Change the stream later calls are ordered on. */
int32_t dgsrhd_set_stream(dgsrhd_ctx* ctx, void* stream);

/* Shape of a state array: nvar = 5, n_elem = elements, n_node = (degree + 1)^dim. */
int32_t dgsrhd_state_shape(const dgsrhd_ctx* ctx, int64_t* nvar, int64_t* n_elem,
                           int64_t* n_node);

/* Node coordinates into a HOST array X_host[dim][n_elem][n_node]. */
int32_t dgsrhd_node_coords(const dgsrhd_ctx* ctx, double* X_host);

/* prim -> cons at every node (Eq. primitive_to_conserved): W (rho, v, P) -> U. */
int32_t dgsrhd_prim2cons(dgsrhd_ctx* ctx, const double* W, double* U);

/* cons -> prim at every node (Sec. 3, the configured solver): U -> W (rho, v, P).
 * iters (nullable, int32 per node) receives the iteration count of the iterative solvers.
 * Invalid states give NaN and are counted. */
int32_t dgsrhd_con2prim(dgsrhd_ctx* ctx, const double* U, double* W, int32_t* iters);

/* R = dU/dt of the nodal DG semi-discretisation (Eq. discrete_hyperbolic_conservation_law
 * with node-collocated quadrature, Eqs. quad-vol-flux and quad-surface-flux): primitives
 * recovered at the nodes, (rho, u, P) extrapolated to the faces, LLF/HLL face flux (Sec.
 * 2.4) lifted into the element.  No physicality operator.  U and R must not alias. */
int32_t dgsrhd_rhs(dgsrhd_ctx* ctx, const double* U, double* R);

/* Physicality-enforcing operator on every element, in place (Sec. 2.5, Eq. smoothed_states).
 * s_out (nullable, [n_elem]) receives each element's smoothing factor (1 = untouched). */
int32_t dgsrhd_enforce(dgsrhd_ctx* ctx, double* U, double* s_out);

/* nsteps SSP-RK steps of size dt in place, the operator after every stage when enabled
 * (Sec. 2.3, Shu-Osher form).  The first call with a given dt captures the step into a CUDA
 * graph; later calls replay it. */
int32_t dgsrhd_step(dgsrhd_ctx* ctx, double* U, double dt, int32_t nsteps);

/* The same with a HOST state, synchronising the stream at the end.  Pinned host memory that the
 * GPU can address (an FP64 context without the limiter): the first kernel of every step reads
 * the state from it over the host link, overlapped with its FP64 work, and keeps a device copy,
 * and the last kernel writes the new state back; the results are those of dgsrhd_step.  Other
 * host memory: copied to the device, stepped, copied back. */
int32_t dgsrhd_step_host(dgsrhd_ctx* ctx, double* U_host, double dt, int32_t nsteps);

/* U_bar = (dR/dU)^T R_bar for R = dgsrhd_rhs(U) (vector-Jacobian product), in FP64 whatever
 * the configured precision: transposed lift, reverse of the LLF/HLL flux, transposed trace
 * extrapolation and volume term, transposed flux Jacobians and the con2prim adjoint
 * (dU/dW)^{-T}.  Non-smooth choices (the min/max wavespeed selection, the clamps of HLL, |lambda|
 * of LLF, the face guard) are frozen at their forward branch.  U_bar must not alias U or R_bar.
 * A reflecting wall contributes the mirrored adjoint of its ghost trace; HLLC keeps the side of
 * its contact and its supersonic cases at their forward choice. */
int32_t dgsrhd_rhs_vjp(dgsrhd_ctx* ctx, const double* U, const double* R_bar, double* U_bar);

/* VJP of the physicality operator with each element's factor s frozen at its forward value
 * (s from dgsrhd_enforce): U_bar_i = s Ut_bar_i + (1 - s) w_i / sum(w) sum_j Ut_bar_j. */
int32_t dgsrhd_enforce_vjp(dgsrhd_ctx* ctx, const double* s, const double* Ut_bar,
                           double* U_bar);

/* One Shu-Osher stage `stage` (0-based) of the configured scheme:
 * Uout = a_k Un + b_k (Uk + dt R(Uk)), followed (if configured) by the limiter and (if enabled)
 * by the physicality operator, whose per-element factors go to s_out (nullable, [n_elem]).  Uout may alias Un or Uk.  Composing
 * the stages reproduces dgsrhd_step.  save (nullable, device, dgsrhd_stage_save_size doubles)
 * receives what dgsrhd_stage_vjp needs from the forward stage: the nodal (rho, u, P, gamma,
 * 1/gamma), the face traces, the face-state tape (per face state its roots and reciprocals, A,
 * B, K, rho (h - 1), U, r, the wavespeeds and the normal flux), the face-guard flags and, with
 * a limiter, its factor theta per element; a stage with save runs the FP64 kernels whatever the
 * configured precision. */
int32_t dgsrhd_step_stage(dgsrhd_ctx* ctx, const double* Un, const double* Uk, double* Uout,
                          int32_t stage, double dt, double* s_out, double* save);

/* Doubles of the `save` buffer of dgsrhd_step_stage: 7 E Nn (nodal primitives) + 10 dim E Nt
 * (traces) + 52 (face points) (tape) + one byte per face point of every element (guard flags),
 * rounded up to whole doubles, + E (the limiter's factors, with a limiter). */
int32_t dgsrhd_stage_save_size(const dgsrhd_ctx* ctx, int64_t* n);

/* Reverse sweep of one stage (the transpose of dgsrhd_step_stage at its input Uk, with the
 * operator's factors s and the limiter's factors theta frozen; s NULL or enforcement off: no
 * operator):
 *   Y_bar = enforce_vjp(theta, enforce_vjp(s, Z_bar)),  Un_bar += a_k Y_bar,
 *   Uk_bar += b_k (Y_bar + dt (dR/dU)^T Y_bar)  at U = Uk
 * (the limiter U_i <- mean + theta (U_i - mean) is the operator's linear map with theta for s).
 * saved (nullable): the `save` buffer of the forward stage; without it the forward quantities
 * are recomputed, which a limited configuration cannot do (theta needs U^n): it returns
 * DGSRHD_EINVAL.  Both outputs ACCUMULATE (zero them first); they may alias each other but
 * not Z_bar. */
int32_t dgsrhd_stage_vjp(dgsrhd_ctx* ctx, const double* Uk, const double* s, const double* saved,
                         const double* Z_bar, double* Un_bar, double* Uk_bar, int32_t stage,
                         double dt);

/* Adjoint of con2prim by the implicit-function theorem (Sec. 3): W = (rho, v, P) solves
 * U = prim2cons(W) (Eq. primitive_to_conserved), so U_bar = (dU/dW)^{-T} W_bar, one 5 x 5 solve
 * per node at the recovered root.  W_bar is in the layout of W. */
int32_t dgsrhd_con2prim_vjp(dgsrhd_ctx* ctx, const double* U, const double* W_bar, double* U_bar);

/* Time step of the CFL rule dt = cfl / ((2p + 1) sum_d 1/dx_d) (all speeds <= c = 1). */
int32_t dgsrhd_cfl_dt(const dgsrhd_ctx* ctx, double cfl, double* dt);

/* Read (and if reset != 0, zero) the device counters; synchronises the stream.  Returns
 * DGSRHD_EBADSTATE, DGSRHD_EC2P_NOCONV or DGSRHD_EUNPHYS_MEAN (in that order of priority)
 * when the counters show such events, DGSRHD_OK otherwise. */
int32_t dgsrhd_get_stats(dgsrhd_ctx* ctx, dgsrhd_stats* out, int32_t reset);

/* Number of kernels the library launched through this context (graph replays count every
 * kernel node). */
int64_t dgsrhd_kernel_launches(const dgsrhd_ctx* ctx);

/* Kernel timing.  While enabled, every kernel launch is bracketed by a pair of CUDA events on
 * the context's stream and dgsrhd_step launches its kernels directly instead of replaying a
 * graph.  dgsrhd_kernel_times synchronises the stream and returns, per kernel kind
 * (DGSRHD_KERNEL_*), the summed duration in milliseconds and the launch count since the last
 * reset.  ms and counts are HOST arrays of DGSRHD_KERNEL_KINDS entries. */
#define DGSRHD_KERNEL_VOLUME 0    /* con2prim + nodal flux + volume term + face traces */
#define DGSRHD_KERNEL_FACE 1      /* numerical flux at every face point */
#define DGSRHD_KERNEL_UPDATE 2    /* lift + RK stage + physicality operator */
#define DGSRHD_KERNEL_ENFORCE 3   /* stand-alone physicality operator */
#define DGSRHD_KERNEL_POINTWISE 4 /* prim2cons / con2prim */
#define DGSRHD_KERNEL_VJP 5       /* the kernels of dgsrhd_rhs_vjp / dgsrhd_enforce_vjp */
#define DGSRHD_KERNEL_KINDS 6
int32_t dgsrhd_set_profiling(dgsrhd_ctx* ctx, int32_t enable);
int32_t dgsrhd_kernel_times(dgsrhd_ctx* ctx, double* ms, int64_t* counts, int32_t reset);

/* dgsrhd_rhs without any device allocation, for callers that cannot allocate GPU memory
 * themselves and cannot let a library do it either: code running under a host framework that
 * owns all device memory, code that must not trigger the implicit synchronisation or failure of
 * cudaMalloc (inside another library's callback, or with device memory fully reserved), or
 * deployments that must fix their device footprint at load time.  The paper has no
 * counterpart; this is a deployment variant of the right-hand side.
 *
 * Computes R = dU/dt exactly as dgsrhd_rhs does for the configuration `cfg` (the split-precision
 * kernels for precision = DGSRHD_PREC_SPLIT, the FP64 ones otherwise), on `stream` (a
 * cudaStream_t, NULL = legacy default stream), with no context.  U (input) and R (output) are
 * caller-owned device arrays in the state layout above; they must not alias.  The scratch is a
 * fixed 64 MiB array in device global memory (8,388,608 doubles) that every GPU loading the
 * library holds until the process exits.  A configuration needs
 *   5 E Nn + 10 dim E Nt + 5 Nt sum_d nface_d + 576 doubles (+ 5 dim E with split precision),
 * with Nn = (p+1)^dim, Nt = (p+1)^(dim-1), nface_d = E (periodic axis) or E + E/n_d, and 576 =
 * 64 slots for each of the 9 device counters; a larger mesh, an invalid configuration or a
 * NULL/aliased array returns DGSRHD_EINVAL before any GPU work.  No call allocates: no
 * cudaMalloc, no cudaFree, no allocating library routine.
 *
 * Every call made outside stream capture looks up the array's device address on the current
 * device (a device reset or another context loads the library's module at a new address); a
 * call made while `stream` is being captured reuses the address of the last call made outside
 * capture on that device, and returns DGSRHD_ECUDA if there was none, so make one call before
 * capturing, and again after a device reset.  All calls share the one array and leave their
 * intermediate results in it, so calls whose GPU work can overlap (different streams, or
 * several host threads) race and must be serialised by the caller.
 *
 * stats_out (nullable, HOST): when given, the call synchronises `stream`, fills the con2prim and
 * face-guard counters of this call and returns DGSRHD_EBADSTATE / DGSRHD_EC2P_NOCONV as
 * dgsrhd_get_stats would; when NULL the call returns as soon as the kernels are queued. */
int32_t dgsrhd_rhs_noalloc(const dgsrhd_config* cfg, void* stream, const double* U, double* R,
                           dgsrhd_stats* stats_out);

/* Spatial mean of a squared velocity component, <v_a^2> = (1/|Omega|) int v_a^2 dV, the
 * diagnostic of the Kelvin-Helmholtz study (Sec. 4.5, the mean of v_y^2 whose growth rate the
 * paper fits), by the nodal quadrature of the basis with con2prim at every node.
 * U: DEVICE state [5][E][Nn]; axis: 0, 1 or 2 (v_x, v_y, v_z); out: HOST double.
 * Synchronises the context's stream (the per-block partial sums are added on the host in a
 * fixed order, so the result is reproducible).  Uses the context's R scratch buffer: do not
 * overlap with another call on the same context.  DGSRHD_EINVAL for null pointers or a bad
 * axis, DGSRHD_ECUDA on a CUDA error; a state con2prim cannot invert gives NaN. */
int32_t dgsrhd_mean_square_velocity(dgsrhd_ctx* ctx, const double* U, int32_t axis, double* out);

/* Diagnostic (no paper counterpart): the library's FP64 reciprocal and root primitives next to
 * CUDA's own, for checking the former against the latter.
 * x:   DEVICE, n doubles.  out: DEVICE, 8 n doubles, written as eight blocks of n:
 *      [ reciprocal 1/x by a third-order correction of an FP32 seed | 1.0 / x (division) |
 *        the library's sqrt(x) | sqrt(x) | the library's x^(-1/3) | rcbrt(x) |
 *        the library's 1/sqrt(x) | rsqrt(x) ]
 *      (the two cube-root blocks are 0 at x = 0).
 * stream: cudaStream_t or NULL for the default stream; the call only queues the kernel.
 * Returns DGSRHD_EINVAL for null pointers or n < 0, DGSRHD_ECUDA on a launch failure. */
int32_t dgsrhd_math_check(const double* x, int64_t n, double* out, void* stream);

/* Diagnostic (no paper counterpart): arithmetic throughput probe, the denominator of the FP64
 * roofline and the cost of the library's FP64 primitives.  Launches one kernel of `threads`
 * threads (a positive multiple of 256, at most 256 x 65535) on `stream` (cudaStream_t, NULL =
 * default); each thread runs four independent chains of `iters` applications of one
 * operation, x <- op(x):
 *   DGSRHD_PROBE_DFMA    x <- fma(x, a, b) in FP64 (2 flops each: the FP64 peak)
 *   DGSRHD_PROBE_DDIV    x <- b / x (CUDA's FP64 division)
 *   DGSRHD_PROBE_DSQRT, DGSRHD_PROBE_DRSQRT, DGSRHD_PROBE_DRCBRT   CUDA's sqrt, rsqrt, rcbrt
 *   DGSRHD_PROBE_RECIP, DGSRHD_PROBE_SQRT, DGSRHD_PROBE_RCBRT, DGSRHD_PROBE_RSQRT
 *                        the library's reciprocal, square root, reciprocal cube root and
 *                        reciprocal square root (FP32 seed, FP64 correction)
 *   DGSRHD_PROBE_FFMA    x <- fmaf(x, a, b) in FP32.
 * sink: DEVICE, `threads` doubles (each thread stores its chains' sum).  *ops (nullable, HOST)
 * receives the number of operations, 4 threads iters; the caller times the kernel (CUDA events
 * on `stream`) and divides.  Returns DGSRHD_EINVAL for a bad kind, iters < 1, a NULL sink or a
 * bad thread count, DGSRHD_ECUDA on a launch failure; only queues the kernel. */
#define DGSRHD_PROBE_DFMA 0
#define DGSRHD_PROBE_DDIV 1
#define DGSRHD_PROBE_DSQRT 2
#define DGSRHD_PROBE_DRSQRT 3
#define DGSRHD_PROBE_DRCBRT 4
#define DGSRHD_PROBE_RECIP 5
#define DGSRHD_PROBE_SQRT 6
#define DGSRHD_PROBE_RCBRT 7
#define DGSRHD_PROBE_FFMA 8
#define DGSRHD_PROBE_RSQRT 9
#define DGSRHD_PROBE_KINDS 10
int32_t dgsrhd_arith_probe(int32_t kind, int64_t iters, double* sink, int64_t threads,
                           void* stream, int64_t* ops);

/* Human-readable name of a status code. */
const char* dgsrhd_status_string(int32_t status);

#ifdef __cplusplus
}
#endif

#endif /* DGSRHD_H */
