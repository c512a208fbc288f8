/*
 * expdg.h - C-ABI of libexpdg, the GB300 (sm_103a) exponential-DG hot path.
 *
 * Method: Kang & Bui-Thanh, "A scalable exponential-DG approach for
 * nonlinear conservation laws" (arXiv 2011.01316).
 *
 *   dq/dt = R(q) = L q + N(q)                                  (Sec. 2.3, Eq. splitDG)
 *   R: nodal DG right-hand side with Lax-Friedrichs fluxes      (Sec. 2.2, 3.1, 3.2)
 *   L = L(q^n): the DG operator of the linear flux A(q^n) q,
 *       stabilisation frozen at q^n                              (Sec. 2.2, Eq. linearflux)
 *   phi-sums  sum_i phi_i(dt L) c_i  by Krylov on an augmented
 *       matrix                                                   (Sec. 2.3)
 *   EPI2 / EXPRB32 / EXPRB42 steps                               (Sec. 5 footnotes)
 *
 * Conventions for every call:
 *   - State arrays are FP64 in the canonical layout q[f][e][n]: field f
 *     (Burgers: u; Euler: rho, rho u_1..rho u_dim, rho E), element
 *     e = ex + ne[0]*(ey + ne[1]*ez), LGL node n = i + (p+1)*(j + (p+1)*k)
 *     with i along x.  Length expdg_num_unknowns().
 *   - Pointers may be host or device memory (detected per call).  Host
 *     buffers are copied through library-owned device memory; the copies
 *     are part of the call.  Device memory must belong to the context's
 *     device (or be managed memory); another device's memory is rejected
 *     with EXPDG_EINVAL.  The caller owns every buffer it passes; the
 *     library owns all device memory it allocates (released by
 *     expdg_destroy).
 *   - Calls are synchronous with respect to the host: they return after the
 *     work on the context's stream has finished.
 *   - A non-zero status leaves outputs unspecified and records a message
 *     for expdg_last_error().  A context is not thread-safe; distinct
 *     contexts are independent.
 */
#ifndef EXPDG_H
#define EXPDG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EXPDG_OK = 0,
  EXPDG_EINVAL = 1,        /* bad argument or configuration */
  EXPDG_ENOMEM = 2,        /* device allocation failed */
  EXPDG_EKRYLOV = 3,       /* no Krylov convergence within max_substeps halvings */
  EXPDG_ENONPHYSICAL = 4,  /* Euler state with rho <= 0 or p <= 0 (never clipped) */
  EXPDG_ETIMEOUT = 5,      /* a bounded device wait gave up */
  EXPDG_ECUDA = 6          /* CUDA runtime error; see expdg_last_error() */
} expdg_status;

typedef enum { EXPDG_BURGERS = 1, EXPDG_EULER = 2 } expdg_equation;
typedef enum { EXPDG_EPI2 = 2, EXPDG_EXPRB32 = 3, EXPDG_EXPRB42 = 4 } expdg_scheme;
/* Boundary conditions: periodic box, or zero Dirichlet data at both ends
 * (1D Burgers only; the paper's footnote to Sec. 4: u+ = u_D = 0 in the
 * convective numerical fluxes, u** = u_D = 0, q** = q-). */
typedef enum { EXPDG_BC_PERIODIC = 0, EXPDG_BC_DIRICHLET = 1 } expdg_bc;
/* Numerical flux of the Euler equations: Lax-Friedrichs (Sec. 5.1, the
 * paper's Euler experiments) or Roe (Sec. 3.2: {F} + 1/2 |A(q*_Roe)| [q] for
 * both the nonlinear and the linear flux, q*_Roe the Roe average). */
typedef enum { EXPDG_FLUX_LF = 0, EXPDG_FLUX_ROE = 1 } expdg_flux;

/* Arithmetic of the operator applies (R, Jv) and of the Arnoldi process.
 *   EXPDG_FP64:     everything in FP64 (reference form).
 *   EXPDG_MIXED:    the linear operator L v (every Jv) in FP32 arithmetic with
 *                   FP32 accumulation, on the FP32 rounding of its input (kept
 *                   beside each FP64 basis vector; conversions on the integer
 *                   pipes); the Krylov basis, the Arnoldi inner products and
 *                   orthogonalisation, phi(H) and the solution update in FP64.
 *                   The residual R in float-float arithmetic (pairs of FP32
 *                   numbers, 48-bit significand, below), delivered in FP64:
 *                   an FP32 residual's rounding (relative 3e-6 on smooth
 *                   data, where R is a small difference of large fluxes) cost
 *                   extra Arnoldi steps and errors above 1e-6 after tens of
 *                   steps; an FP64 one runs 3.7x slower on this GPU.
 *   EXPDG_MIXED_FF: a variant: Jv in FP32; the residual in float-float
 *                   arithmetic (pairs of FP32 numbers, 48-bit significand,
 *                   error-free transformations on the FP32 pipes); Krylov
 *                   basis, inner products, orthogonalisation and phi(H) in
 *                   float-float; the solution update in FP64.  On this GPU the
 *                   FP64 pipe runs about 1/70 of the FP32 rate, so this form's
 *                   streaming Krylov kernels stay off it; its results are
 *                   within 48-bit rounding of FP64 arithmetic, not FP64. */
typedef enum { EXPDG_FP64 = 0, EXPDG_MIXED = 1, EXPDG_MIXED_FF = 2 } expdg_precision;

typedef struct {
  int dim;              /* 1, 2 or 3 (Burgers: 1) */
  int p;                /* polynomial order, 1..EXPDG_MAX_ORDER */
  int ne[3];            /* elements per direction (unused entries ignored) */
  double lo[3], hi[3];  /* periodic box [lo_d, hi_d] */
  int eq;               /* expdg_equation */
  double gamma;         /* ratio of specific heats (Euler) */
  int scheme;           /* expdg_scheme */
  int prec;             /* expdg_precision */
  double krylov_tol;    /* accept when err <= tol * beta (see expdg_phi) */
  int m_max;            /* Krylov dimension limit, <= EXPDG_MAX_KRYLOV */
  int m_step;           /* error checks at m = m_step, 2 m_step, ... */
  int max_substeps;     /* limit on rejected (halved) Krylov attempts per solve */
  int iop;              /* Krylov orthogonalisation: 0 = full (Arnoldi by two-pass classical
                           Gram-Schmidt with delayed re-orthogonalisation); k = 1..EXPDG_MAX_IOP =
                           incomplete orthogonalisation against the last k basis vectors, the
                           procedure KIOPS uses in place of Arnoldi (Sec. 1, Sec. 2.3) */
  double kappa;         /* viscosity of the Burgers equation (Sec. 3.1, Eq. pde-burgers-eq), >= 0;
                           > 0 adds kappa d/dx(q) with q = du/dx, central fluxes u** = {u},
                           q** = {q} (Eq. gov-burgers1d); Burgers only */
  int bc;               /* expdg_bc */
  int flux;             /* expdg_flux (Euler; Burgers uses Lax-Friedrichs) */
  int tile;             /* expdg_tile: CTA size of the FP32 operator apply (EXPDG_MIXED, EXPDG_MIXED_FF) */
} expdg_config;

/* CTA size (elements per CTA, one thread per node) of the FP32 operator
 * apply L(qt) v (EXPDG_MIXED, EXPDG_MIXED_FF).  EXPDG_TILE_AUTO times the
 * three sizes on the context's own mesh when it is created (about 20 operator
 * applies on zero data) and keeps the fastest; the choice is cached per mesh
 * shape and form for the process, so later contexts of the same shape do not
 * time again.  The EXPDG_FP64 form and the other kernels always use
 * EXPDG_TILE_256. */
typedef enum {
  EXPDG_TILE_AUTO = 0,
  EXPDG_TILE_256 = 1,  /* about 256 threads per CTA */
  EXPDG_TILE_128 = 2,
  EXPDG_TILE_512 = 3,
  /* Tensor-core trial (2D / 3D Euler, LF flux, EXPDG_MIXED; elsewhere these
   * act as EXPDG_TILE_256): the operator's derivative contractions
   * sum_j D_ij F_j as warp-level m16n8k8 TF32 matrix products (lines of 16
   * along each direction against D^T), FP32 accumulation.  Never chosen by
   * EXPDG_TILE_AUTO: measured slower than the FP32 FMA form at p = 4..8. */
  EXPDG_TILE_TC3 = 4,  /* operands split hi + lo, three products: about FP32 accuracy */
  EXPDG_TILE_TC1 = 5   /* one TF32 product (10-bit significands): far above the 1e-6 bar */
} expdg_tile;

#define EXPDG_MAX_ORDER 8
#define EXPDG_MAX_KRYLOV 64
#define EXPDG_MAX_PHI 3      /* phi_0 .. phi_3 */
#define EXPDG_MAX_IOP 8      /* largest incomplete-orthogonalisation window */

typedef struct {
  int krylov_iters;       /* Arnoldi iterations (operator applies), incl. rejected attempts */
  int substeps;           /* accepted Krylov sub-steps */
  int rejected;           /* attempts that reached m_max without acceptance */
  int jv_applies;         /* L(q~) v applies */
  int residual_applies;   /* R(q) applies */
  double err_est;         /* largest error estimate of an accepted sub-step */
} expdg_stats;

/* Krylov decision trace: one record per accepted sub-step, in order, for all
 * Krylov solves of a step (solve = 0 for the first phi-sum of the step, 1 for
 * the second stage of EXPRB32/EXPRB42). */
typedef struct {
  int solve;
  int m;          /* Krylov dimension used */
  double sigma;   /* sub-step length (fraction of the solve's interval) */
  double eta;     /* tail scale of the augmented matrix */
} expdg_trace_entry;

typedef struct expdg_ctx expdg_ctx;

/* Default configuration: 2D Euler, p = 4, 64 x 64 on [0,10]^2, EPI2, FP64,
 * tol 1e-10, m_max 64, m_step 5, max_substeps 32, iop 0 (full orthogonalisation). */
void expdg_default_config(expdg_config* cfg);

/* Create a context (validates cfg, builds LGL tables, allocates the device
 * state, Krylov basis and scratch on the current CUDA device).
 * Returns EXPDG_EINVAL for a bad configuration, EXPDG_ENOMEM / EXPDG_ECUDA on
 * device failures; *out is NULL then. */
expdg_status expdg_create(const expdg_config* cfg, expdg_ctx** out);
void expdg_destroy(expdg_ctx* ctx);

/* Run the context's work on this cudaStream_t (NULL = the legacy default
 * stream).  The stream must belong to the context's device. */
expdg_status expdg_set_stream(expdg_ctx* ctx, void* cuda_stream);

/* Sizes: fields m, elements, nodes per element (p+1)^dim, unknowns m*Ne*Np. */
size_t expdg_num_unknowns(const expdg_ctx* ctx);
int expdg_num_fields(const expdg_ctx* ctx);
size_t expdg_num_elements(const expdg_ctx* ctx);
int expdg_nodes_per_element(const expdg_ctx* ctx);

/* Physical LGL node coordinates, host buffer xyz[dim][Ne][Np] (FP64):
 * x_d = lo_d + h_d (e_d + (r_i + 1)/2), LGL nodes r of order p. */
expdg_status expdg_node_coords(const expdg_ctx* ctx, double* xyz);
/* The same without a context (host computation only). */
expdg_status expdg_config_node_coords(const expdg_config* cfg, double* xyz);

/* Time-independent forcing s added to R (N values in the canonical layout,
 * host or device memory; NULL removes it), e.g. the source of a manufactured
 * solution (Sec. 5.1).  The first call allocates N doubles on the device
 * (not counted by expdg_context_bytes).  Used by expdg_residual and the
 * exponential steps (R = L q + N(q) + s); not by expdg_jv. */
expdg_status expdg_set_source(expdg_ctx* ctx, const double* s);

/* R(q): the DG right-hand side (Sec. 2.2, Eq. EXPO-SemiDiscretizedForm_ode;
 * strong collocated LGL form; LF flux with lambda = max(|u|) for Burgers,
 * Sec. 3.1, and max(|u.n| + a) for Euler, Sec. 5.1).  q, r: canonical layout.
 * In EXPDG_MIXED_FF the arithmetic is float-float (inputs and outputs stay
 * FP64), FP64 in the other forms. */
expdg_status expdg_residual(expdg_ctx* ctx, const double* q, double* r);

/* L(qt) v: the frozen-flux linear DG operator (Sec. 2.2, Eq. linearflux, with
 * (u~u)* of Sec. 3.1 / (A~q)* of Sec. 3.2; LF coefficient from qt).  In
 * EXPDG_MIXED and EXPDG_MIXED_FF the arithmetic is FP32. */
expdg_status expdg_jv(expdg_ctx* ctx, const double* qt, const double* v, double* out);

/* out = sum_{i=0}^{P} phi_i(tau L(qt)) c_i with c = [c_0, ..., c_P] (P <= 3;
 * c[i] may be NULL for a zero vector), Sec. 2.3 Eq.
 * linear_combination_of_phifunctions with the dt^i folded into c_i.
 * Method: Arnoldi (classical Gram-Schmidt, twice) on the augmented matrix
 *   A_hat = [[sigma tau L, eta W], [0, J]],  W = [b_P .. b_1],  J = upper shift,
 * started from [b_0; e_P / eta], beta = its norm; the top block of
 * beta V_m exp(H_m) e_1 approximates the sum.  With cfg.iop = k > 0 the
 * Arnoldi process is replaced by incomplete orthogonalisation: step j
 * orthogonalises A_hat v_j against v_{j-k+1}, ..., v_j only (H_m banded);
 * the approximation and the error estimate are unchanged.  The error estimate
 * err = beta h_{m+1,m} |e_m^T exp(H_m) e_1| is checked at m = m_step,
 * 2 m_step, ..., m_max; accepted when err <= krylov_tol * beta (or on a happy
 * breakdown).  In the FP32-operator forms (EXPDG_MIXED, EXPDG_MIXED_FF) a
 * check at m is also accepted when the
 * approximation changed by at most krylov_tol * beta since m - 1
 * (beta |y_m - [y_{m-1}; 0]|, y_{m-1} = exp(H_{m-1}) e_1 evaluated in the same
 * launch, on problems of at least 131072 unknowns), else when it
 * changed by at most that since the previous check: the FP32 operator's
 * rounding noise inflates Saad's estimate there without slowing the
 * convergence of the approximation.  Reaching m_max halves the sub-step sigma; after an accepted
 * sub-step with m <= m_max/2 sigma doubles (never past the end).  Sub-step
 * vectors: b_0 = w(s), b_i = sigma^i sum_j s^j/j! c_{i+j}.  The tail scale
 * eta = 2^-round(log2(max_i ||b_i||)) (formed on the device when deciding
 * adaptively; an accepted sub-step then costs one device-to-host read, the
 * check's).  If replay != NULL, the nreplay
 * records (all with solve == 0) are followed instead of deciding; otherwise,
 * if trace != NULL, up to trace_cap accepted sub-steps are written there and
 * *ntrace is set.  EXPDG_EINVAL for a tau that is not finite. */
expdg_status expdg_phi(expdg_ctx* ctx, const double* qt, double tau, const double* const* c, int P,
                       double* out, expdg_stats* stats,
                       const expdg_trace_entry* replay, int nreplay,
                       expdg_trace_entry* trace, int trace_cap, int* ntrace);

/* One exponential step of the configured scheme from time-independent state
 * q (in place): EPI2 q += dt phi_1(dt L) R(q) (Sec. 5.1 footnote), EXPRB32 /
 * EXPRB42 (Sec. 5.1 / 5.2 footnotes).  replay / trace as in expdg_phi, with
 * the solve index distinguishing the two stages.  Without replay, the error
 * checks of each stage's first sub-step start at m_prev, the m that stage
 * accepted in this context's previous step, and every eighth step (and after
 * a probe that was accepted) one check lower (m_prev - 1 with paired checks,
 * else max(m_step, m_prev - m_step)) so that a falling m is found
 * (steps in a row need similar m; starting later can only give a more
 * accurate result).  Then m_prev itself, with paired checks (above) m_prev + 2
 * and m_prev + 4, and the multiples of m_step.  EXPDG_EINVAL (q untouched)
 * unless dt is finite and > 0. */
expdg_status expdg_step(expdg_ctx* ctx, double* q, double dt, expdg_stats* stats,
                        const expdg_trace_entry* replay, int nreplay,
                        expdg_trace_entry* trace, int trace_cap, int* ntrace);

/* nsteps steps of size dt (in place); stats accumulate over the steps.  The
 * check-start memory of expdg_step is cleared first, so the result depends only
 * on the arguments (not on earlier calls on the context).  EXPDG_EINVAL (q
 * untouched) unless dt is finite and > 0 and nsteps >= 0. */
expdg_status expdg_advance(expdg_ctx* ctx, double* q, double dt, int nsteps, expdg_stats* stats);

/* Kernel classes of the hot path, for profiling. */
typedef enum {
  EXPDG_K_RESIDUAL = 0,  /* R(q) */
  EXPDG_K_JV = 1,        /* L(qt) v, incl. the augmented-matrix tail */
  EXPDG_K_DOTS = 2,      /* Gram-Schmidt inner products */
  EXPDG_K_UPDATE = 3,    /* Gram-Schmidt updates (+ norm) */
  EXPDG_K_PHI = 4,       /* exp(H_m) e_1 of the projected matrix */
  EXPDG_K_COMBINE = 5,   /* w = beta V_m y (+ state update) */
  EXPDG_K_VECTOR = 6,    /* linear combinations, norms, conversions, start vector */
  EXPDG_K_COUNT = 7
} expdg_kernel_class;

typedef struct {
  long long launches;    /* kernel launches of this class */
  double ms;             /* summed device time (CUDA events around each launch; 0 unless profiling) */
  double bytes;          /* algorithmic bytes moved: the minimum global-memory reads + writes the
                            launch's operation needs (neighbour traces and re-reads counted 0) */
} expdg_kernel_prof;

/* Turn per-launch CUDA-event timing on or off and clear the counters.  Launch
 * counts and algorithmic bytes are always accumulated; durations only while
 * profiling is on (each launch is then bracketed by two events on the
 * context's stream). */
expdg_status expdg_profile_enable(expdg_ctx* ctx, int on);

/* Copy the per-class counters accumulated since the last enable/reset into
 * out[EXPDG_K_COUNT] (synchronises the stream).  If reset != 0 the counters
 * restart from zero. */
expdg_status expdg_profile_get(expdg_ctx* ctx, expdg_kernel_prof* out, int reset);

/* Device memory one context of this configuration holds (state, scratch,
 * Krylov basis of m_max + 1 vectors, reduction buffers), each allocation
 * rounded up to 2 MiB; 0 if cfg is invalid. */
size_t expdg_context_bytes(const expdg_config* cfg);

/* ---- Solve server: continuous batching of independent solves --------------
 * Serving pattern (not in the paper, which runs one solve per MPI job):
 * requests are queued and taken in arrival order by worker threads, each with
 * its own CUDA stream, as soon as the device-memory budget admits the
 * request's context (expdg_context_bytes); solves arriving while others run
 * start as soon as a worker and memory free up, and their kernels overlap on
 * the GPU.  Each solve's state and Krylov basis stay resident on the device
 * for the whole solve.  Finished contexts are cached and reused by requests of
 * the same configuration (no device allocation per request); idle cached
 * contexts are released when a request needs their memory.  Results are
 * deterministic: a solve gives the same result alone or among others. */
typedef struct expdg_server expdg_server;
typedef struct {
  size_t hbm_budget;  /* bytes of device memory the server's contexts may hold (0: 90% of free memory) */
  int workers;        /* solves in flight at once, 1..64 (one host thread and CUDA stream each) */
} expdg_server_config;

expdg_status expdg_server_create(const expdg_server_config* cfg, expdg_server** out);
/* Waits for running solves, releases all contexts. */
void expdg_server_destroy(expdg_server* s);
/* Queue nsteps steps of size dt of configuration cfg from host state q0 (copied
 * before returning).  Non-blocking.  EXPDG_ENOMEM if the context can never fit
 * the budget, EXPDG_EINVAL for a bad configuration or a dt that is not finite
 * and > 0. */
expdg_status expdg_server_submit(expdg_server* s, const expdg_config* cfg, const double* q0, double dt, int nsteps,
                                 int64_t* id);
/* Non-blocking: ids (up to cap) of solves finished since the last poll. */
expdg_status expdg_server_poll(expdg_server* s, int64_t* ids, int cap, int* n);
/* Result of a finished solve (host q_out, stats, times[3] = queueing, service and
 * total latency in seconds; any may be NULL); releases the request.  Returns the
 * solve's own status (EXPDG_EINVAL if id is unknown or not finished). */
expdg_status expdg_server_fetch(expdg_server* s, int64_t id, double* q_out, expdg_stats* stats, double* times);
/* Bytes held by contexts, queued and running solve counts. */
expdg_status expdg_server_info(expdg_server* s, size_t* used_bytes, int* pending, int* running);

/* ---- Resident batch: many small solves, one launch per class ---------------
 * Batching pattern (not in the paper): n independent EPI2 solves (Sec. 5.1
 * footnote; the phi_1 sum by the augmented Krylov method of Sec. 2.3, with the
 * decisions of expdg_phi: checks at multiples of m_step and at m_max, Saad's
 * estimate <= krylov_tol beta, happy breakdown, sub-steps halving at m_max and
 * doubling after an accepted sub-step with m <= m_max / 2) run as ONE kernel
 * launch per class of equal (eq, dim, p, prec), one CTA per instance; every
 * step of every instance runs inside that launch (Krylov basis in device
 * memory, H and exp(H_m) in shared memory, decisions on the device), and the
 * classes' launches run side by side.  For instances too small to fill the
 * GPU, where a solve through a context is a chain of short launches.
 *   - Each configuration: scheme EXPDG_EPI2; 1D Burgers (periodic or
 *     Dirichlet, kappa >= 0) or 2D Euler; p = 1..5; LF flux; prec EXPDG_FP64
 *     or EXPDG_MIXED (FP32 operator applies on the FP32 rounding of each basis
 *     vector, float-float residual, FP64 Krylov basis, inner products,
 *     orthogonalisation (modified Gram-Schmidt), exp(H_m) and update); m_max
 *     <= EXPDG_BATCH_MAX_KRYLOV; iop = 0 (full orthogonalisation) or the
 *     window.  Other configurations: EXPDG_EINVAL.
 *   - expdg_batch_create allocates every instance's scratch (basis of
 *     m_max + 1 vectors, the operator's state, four vectors).
 *   - expdg_batch_advance: nsteps steps of size dt[i] of instance i from its
 *     state q[i] (a DEVICE array of the current device, canonical layout),
 *     in place, on `stream` (NULL: legacy default stream); returns after the
 *     stream has finished.  Returns EXPDG_OK, or the status of the first
 *     instance (in the given order) that failed (EXPDG_ENONPHYSICAL,
 *     EXPDG_EKRYLOV); that instance stopped at the start of the failing
 *     step, the others ran all steps.  EXPDG_EINVAL for a bad pointer or dt.
 *   - expdg_batch_result: instance i's status, its statistics over the last
 *     advance, and the steps it completed.
 *   - Results do not depend on the other instances of the batch. */
#define EXPDG_BATCH_MAX_KRYLOV 40
typedef struct expdg_batch expdg_batch;
expdg_status expdg_batch_create(const expdg_config* cfgs, int n, expdg_batch** out);
expdg_status expdg_batch_advance(expdg_batch* b, double* const* q, const double* dt, int nsteps, void* stream);
expdg_status expdg_batch_result(const expdg_batch* b, int i, expdg_stats* stats, int* steps_done);
/* Kernel launches one advance makes (the number of classes). */
int expdg_batch_launches(const expdg_batch* b);
void expdg_batch_destroy(expdg_batch* b);


/* ---- Allocation-free residual ---------------------------------------------
 * The paper has no counterpart to this call; it is a deployment convenience.
 *
 * Some callers cannot let a library allocate device memory: an application
 * whose GPU memory is entirely owned by its own pool allocator (cudaMalloc
 * would fail or fragment that pool), code on a latency-critical path where
 * cudaMalloc / cudaFree and their implicit device synchronisation are not
 * acceptable, or a plug-in that may not create allocations its host cannot
 * account for.  expdg_residual_noalloc computes exactly what expdg_residual
 * computes for the configuration cfg, with no context and without allocating:
 *
 *   - q (input) and r (output) are caller-owned DEVICE arrays of the current
 *     device (or managed memory), m * Ne * (p+1)^dim doubles in the canonical
 *     layout; host pointers and other devices' memory are rejected with
 *     EXPDG_EINVAL.  cuda_stream: the stream to run on (NULL = legacy default
 *     stream); the call returns after that stream has finished.
 *   - Scratch (the float-float state copy of EXPDG_MIXED and
 *     EXPDG_MIXED_FF, the float-float output of EXPDG_MIXED_FF, and the
 *     non-physical-state flag of every form) is a fixed static device array
 *     of about 8 MiB that every GPU which loads the library keeps until the
 *     process exits.  EXPDG_MIXED and EXPDG_MIXED_FF are limited to
 *     EXPDG_NOALLOC_MAX_UNKNOWNS unknowns (larger sizes return EXPDG_EINVAL);
 *     EXPDG_FP64 works in place on q and r and has no size limit.
 *   - The first call on a device looks up the array's device address (once
 *     per device, safe from several host threads).  Every call copies the
 *     status word to the host and synchronises the stream, so the call cannot
 *     be used inside a stream capture.
 *   - All calls share the array: calls that overlap on the GPU (other streams,
 *     other host threads) race and must be serialised by the caller.
 *   - Returns EXPDG_ENONPHYSICAL for an Euler state with rho <= 0 or p <= 0,
 *     EXPDG_EINVAL for a bad configuration, size or pointer, EXPDG_ECUDA on a
 *     CUDA error.  Other fields of cfg (scheme, Krylov settings) are ignored. */
#define EXPDG_NOALLOC_MAX_UNKNOWNS (1u << 19)
expdg_status expdg_residual_noalloc(const expdg_config* cfg, const double* q, double* r, void* cuda_stream);

/* Message of the last failing call on this context ("" if none). */
const char* expdg_last_error(const expdg_ctx* ctx);

/* The expdg_tile the context's operator apply uses (never EXPDG_TILE_AUTO);
 * 0 for a null context. */
int expdg_tile_in_use(const expdg_ctx* ctx);

/* Library version string. */
const char* expdg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* EXPDG_H */
