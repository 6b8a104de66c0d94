/*
 * rsfde.h -- C ABI of the GB300 (sm_103a) solver for one implicit time step of
 * the volume-penalized 2D Riesz space-fractional diffusion scheme, solved by
 * flexible GMRES with the sine-transform (tau) preconditioner of Huang & Sun,
 * arXiv 2102.11576.
 *
 * Notation (Section 2):  the box (ax,bx) x (ay,by) holds the convex domain
 * Omega; its interior grid is n1 x n2 with h_x = (bx-ax)/(n1+1),
 * h_y = (by-ay)/(n2+1).  Each step solves Eq. 2.17,
 *     M u^k = u^{k-1} + dt f^{k-1},   M = I - A + D,
 *     A = I (x) A_x + A_y (x) I,  A_x = c_x G_{n1}^{(alpha1)}, A_y = c_y G_{n2}^{(alpha2)},
 * with c_x = dt k_x c_{alpha1} / h_x^{alpha1}, G the symmetric Toeplitz matrix of
 * Eq. 2.16 built from the weights of Eq. 2.6, and D = (dt/eta) Phi the penalty
 * (Phi = 1 outside Omega).  The preconditioner is Eq. 4.6:
 *     P^-1 = (I - Phi)(I - tau_1(A))^-1 + Phi((1 + dt/eta) I - tau_1(A))^-1.
 *
 * Layout: every grid array holds N = n1*n2 values, x fastest
 * (u[j*n1 + i], i the x-index, j the y-index), as u^k is ordered in Section 2.
 *
 * Ownership and streams: unless an argument says "host", array arguments are
 * caller-owned DEVICE pointers (16-byte aligned, e.g. from torch or
 * cudaMalloc) on the context's device.  The context owns its workspace.  Every
 * call is enqueued on the context's stream (rsfde_opts.stream, or
 * rsfde_set_stream); calls that report statistics synchronise that stream
 * before returning.  A context must not be used from two host threads at once.
 *
 * Errors: every int-returning call returns RSFDE_OK (0) or a negative code;
 * nothing aborts the process.  rsfde_strerror() names a code.  After
 * RSFDE_ECUDA the context should be destroyed.
 */
#ifndef RSFDE_H
#define RSFDE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RSFDE_OK 0
#define RSFDE_EINVAL (-1)      /* bad argument: alpha outside (1,2), k/dt/eta <= 0, n < 1, NULL, ... */
#define RSFDE_ENOMEM (-2)      /* device or host allocation failed */
#define RSFDE_ECUDA (-3)       /* a CUDA runtime call failed */
#define RSFDE_ENOTCONV (-4)    /* max_iter reached; x holds the last iterate, stats its residual */
#define RSFDE_ENONFINITE (-5)  /* NaN or Inf met in the right side or in the Arnoldi process */
#define RSFDE_ETIMEOUT (-6)    /* a bounded device-side wait gave up */

/* Precisions.  Four choices are independent:
 *  - precond_prec: the preconditioner apply (Eq. 4.6) in RSFDE_FP64,
 *    RSFDE_FP32, RSFDE_BF16X3 or RSFDE_BF16;
 *  - matvec_prec: the arithmetic of the operator M applied to the Arnoldi
 *    vectors (Eq. 2.14-2.17), RSFDE_FP64, RSFDE_DF32 or RSFDE_FP32;
 *  - basis_prec: the storage of the Krylov basis and the arithmetic of the
 *    Gram-Schmidt orthogonalisation, RSFDE_FP64 (any operator), RSFDE_DF32
 *    (with the double-FP32 operator) or RSFDE_FP32 (with the FP32 operator);
 *  - resid_prec: the arithmetic of M x in the true residual b - M x that
 *    decides convergence, RSFDE_FP64, RSFDE_EXACT or RSFDE_DF32.
 * The Hessenberg matrix, the Givens least squares, the solution x and the
 * subtraction b - M x and its norm are FP64 in every mode.  Flexible GMRES
 * tolerates the inexact preconditioner.  With every choice FP64 except the
 * preconditioner (FP32 or BF16X3) and, optionally, the operator's FFT
 * arithmetic, the orthogonalisation, the least squares and the true residual
 * are FP64 arithmetic throughout. */
#define RSFDE_FP64 0
#define RSFDE_FP32 1
/* Preconditioner sine transforms as tensor-core GEMMs in split BF16
 * (X = X_hi + X_lo; X_hi S_hi + X_hi S_lo + X_lo S_hi with FP32 accumulation). */
#define RSFDE_BF16X3 3
/* Preconditioner sine transforms as tensor-core GEMMs in plain BF16 (one
 * product X_hi S_hi with FP32 accumulation; about 3 significant digits). */
#define RSFDE_BF16 4
/* Double-FP32 arithmetic (pairs of FP32 numbers, ~48-bit significand,
 * error-free transforms of Dekker and Knuth) for the operator, the Krylov
 * basis or the M x of the true residual. */
#define RSFDE_DF32 2
/* True residual only: the Toeplitz products of M x (Eq. 2.14-2.16) computed
 * exactly in integer arithmetic -- each row or column of x scaled by a power
 * of two to integers below 2^55, the Toeplitz column to integers whose row
 * sums stay below 2^63, the convolution (an integer below 2^118) by
 * number-theoretic transforms modulo four 30-bit primes and the Chinese
 * remainder theorem -- then rounded to FP64 (53 bits, truncated).  Its only
 * errors are the two scalings (2^-54 of each vector's largest entry; 2^-63
 * of the Toeplitz row sum per coefficient) and that final rounding: below
 * the rounding error bounds of FP64 evaluation.  The rest of b - M x and its
 * norm are FP64 arithmetic.  It runs on the integer pipes, which GB300 has
 * in far greater number than FP64 units. */
#define RSFDE_EXACT 5

/* Krylov variant.  RSFDE_FGMRES_RIGHT (default): right-preconditioned flexible
 * GMRES, stop when the true ||b - M x||_2 <= tol ||b||_2.  RSFDE_GMRES_LEFT:
 * the left-preconditioned GMRES(m) of the paper's experiments (Section 5),
 * applied to P^-1 M x = P^-1 b and stopped when
 * ||P^-1 (b - M x)||_2 <= tol ||P^-1 b||_2 (rel_res then reports that ratio);
 * with use_precond = 0 it is plain GMRES. */
#define RSFDE_FGMRES_RIGHT 0
#define RSFDE_GMRES_LEFT 1

/* Arnoldi orthogonalisation: classical Gram-Schmidt, or with one re-orthogonalisation pass. */
#define RSFDE_CGS 0
#define RSFDE_CGS2 1

typedef struct rsfde_ctx rsfde_ctx;
typedef struct rsfde_batch rsfde_batch;

/* Section 2: the box Omega-bar = (ax,bx) x (ay,by) and its interior grid n1 x n2. */
typedef struct {
  int32_t n1, n2;
  double ax, bx, ay, by;
} rsfde_grid;

typedef struct {
  int32_t restart;      /* m of FGMRES(m); Section 5 uses 20.  1..64 */
  int32_t max_iter;     /* cap on inner iterations per solve */
  double tol;           /* stop when ||b - M x||_2 <= tol ||b||_2 */
  int32_t precond_prec; /* RSFDE_FP64 | RSFDE_FP32 | RSFDE_BF16X3 | RSFDE_BF16 */
  int32_t arnoldi;      /* RSFDE_CGS | RSFDE_CGS2 */
  int32_t use_precond;  /* 1: P-hat of Eq. 4.6; 0: unpreconditioned GMRES */
  int32_t matvec_prec;  /* RSFDE_FP64 | RSFDE_DF32 | RSFDE_FP32: arithmetic of M applied to the
                           Arnoldi vectors (its output is stored in basis_prec) */
  int32_t variant;      /* RSFDE_FGMRES_RIGHT | RSFDE_GMRES_LEFT */
  int32_t use_graph;    /* 1: the cycles of a solve replay as one CUDA graph with a device-side
                           loop (one host synchronisation per solve); 0: direct launches with
                           one host check per cycle.  Profiling always uses direct launches. */
  void* stream;         /* cudaStream_t; NULL = the legacy default stream */
  int32_t resid_prec;   /* RSFDE_FP64 (default) | RSFDE_EXACT | RSFDE_DF32: arithmetic of M x in
                           the true residual b - M x that decides convergence (paper mode: FP64
                           or exact; double-FP32 is taken as FP64 there).  b - M x and its norm
                           are FP64 in every case.  RSFDE_EXACT needs an FP64 or FP32 basis.
                           Double-FP32 carries ~48 significant bits: its rounding error is a few
                           units of 1e-14 times |M||x|, far below a 1e-10 tolerance, but it is
                           not FP64 arithmetic. */
  int32_t basis_prec;   /* RSFDE_FP64 (default) | RSFDE_DF32 | RSFDE_FP32: Krylov basis storage and
                           Gram-Schmidt arithmetic (right-preconditioned FGMRES; paper mode always
                           FP64).  RSFDE_DF32 needs matvec_prec RSFDE_DF32, RSFDE_FP32 needs
                           matvec_prec RSFDE_FP32 (else RSFDE_EINVAL). */
} rsfde_opts;

typedef struct {
  int32_t iters;     /* inner (Arnoldi) iterations of the last solve */
  int32_t restarts;  /* restarts of the last solve */
  int32_t converged; /* 1 if ||b - M x|| <= tol ||b|| was met */
  int32_t status;    /* RSFDE_OK, RSFDE_ENOTCONV or RSFDE_ENONFINITE */
  double rel_res;    /* final true ||b - M x||_2 / ||b||_2 */
  double bnorm;      /* ||b||_2 */
  double t_ms[6];    /* device time of the last call per hot-path phase, measured only while the
                        profiler is on (rsfde_profile_enable), else 0:
                        [0] right side, norms and loop control, [1] operator M on the Arnoldi
                        vectors, [2] preconditioner, [3] Gram-Schmidt with the Givens step,
                        [4] least-squares back substitution, [5] solution update and true
                        residual */
  double bytes;      /* algorithmic HBM bytes of the last call: every grid vector the method must
                        read or write once per use (the operands of each preconditioner apply,
                        operator apply, Gram-Schmidt pass, solution update and true residual, the
                        mask bits), in the precisions configured; excludes the transforms'
                        intermediates and any re-read */
} rsfde_stats;

/* Defaults: restart 20, max_iter 10000, tol 1e-10, FP64 preconditioner, CGS,
 * preconditioned, FP64 operator, basis and residual, right-preconditioned
 * FGMRES, CUDA graph, default stream. */
void rsfde_opts_default(rsfde_opts* o);

/* Section 2 / Eq. 2.16 / Section 4.1 (setup of one linear system).
 * mask: DEVICE pointer to N uint8, 1 where the grid point lies in Omega,
 * 0 in the extension region (copied; the caller keeps ownership).
 * n1, n2 in 1..4096; alpha1, alpha2 in (1,2); kx, ky, dt, eta > 0.  opts may
 * be NULL (defaults).
 * Builds the Toeplitz and tau tables on the host in FP64 and uploads them.
 * Returns RSFDE_EINVAL, RSFDE_ENOMEM or RSFDE_ECUDA on failure (*out = NULL). */
int rsfde_setup(rsfde_ctx** out, const rsfde_grid* grid, const uint8_t* mask, double alpha1,
                double alpha2, double kx, double ky, double dt, double eta, const rsfde_opts* opts);

/* Re-runs the parameter-dependent setup (c_x, c_y, dt/eta, spectra) for new
 * k_x, k_y, dt; grid, mask, alpha and eta are kept. */
int rsfde_set_params(rsfde_ctx* ctx, double kx, double ky, double dt);

/* Replaces the options (restart must not exceed the one given at setup). */
int rsfde_set_opts(rsfde_ctx* ctx, const rsfde_opts* opts);
int rsfde_set_stream(rsfde_ctx* ctx, void* stream);

/* Eq. 2.17 solved for x: M x = b by right-preconditioned flexible GMRES(m).
 * b: device, N doubles.  x: device, N doubles, in: initial guess, out: the
 * solution (or the last iterate with RSFDE_ENOTCONV).  stats may be NULL.
 * Synchronises the stream. */
int rsfde_solve(rsfde_ctx* ctx, const double* b, double* x, rsfde_stats* stats);

/* One implicit step of Eq. 2.17 with the built-in source f(u) = u - u^3 (+ src),
 * zero outside Omega (Section 2):  b = u^{k-1} + dt (1-Phi)(u^{k-1} - (u^{k-1})^3 + src),
 * initial guess u^{k-1} if u_prevprev is NULL, else 2u^{k-1} - u^{k-2} (Section 5).
 * u_prev: device N doubles; u_prevprev, src: device N doubles or NULL;
 * u_next: device N doubles (may alias neither input).  Synchronises the stream.
 * The built-in f does not depend on t, so the step takes no time argument; a
 * time-dependent source is passed as this step's src (its values at t_{k-1}),
 * and any other f(u, x, y, t) goes through rsfde_solve with a right side the
 * caller builds. */
int rsfde_step(rsfde_ctx* ctx, const double* u_prev, const double* u_prevprev, const double* src,
               double* u_next, rsfde_stats* stats);

/* rsfde_step with HOST arrays: copies the inputs to the device, runs the
 * step, copies u^k back (all on the context's stream).  Host arrays may be
 * pageable or pinned. */
int rsfde_step_host(rsfde_ctx* ctx, const double* u_prev_host, const double* u_prevprev_host,
                    const double* src_host, double* u_next_host, rsfde_stats* stats);

/* Adjoint solve for the backward time march: M^T mu = lam.  M is symmetric
 * (Lemma 2.3), so this is the forward solver applied to lam; mu: in initial
 * guess, out solution.  Synchronises the stream. */
int rsfde_adjoint(rsfde_ctx* ctx, const double* lam, double* mu, rsfde_stats* stats);

/* One backward step of the discrete adjoint of the time march (gradient of a
 * loss of u^m; the paper itself states no gradient -- this is the exact
 * derivative of the scheme of Eq. 2.17 with f(u) = u - u^3 + s).  Given
 * u^{k-1}, u^k and lam = dL/du^k:
 *   solves M mu = lam (M symmetric, Lemma 2.3), mu holding the initial guess;
 *   lam_prev = mu + dt (1 - Phi)(1 - 3 (u^{k-1})^2) mu          (= dL/du^{k-1});
 *   grad_src += dt (1 - Phi) mu                                  (if not NULL);
 *   grad_k[0] += <mu, (I (x) A_x) u^k> / k_x,  grad_k[1] += <mu, (A_y (x) I) u^k> / k_y
 *   (A_x, A_y are linear in k_x, k_y).
 * u_prev, u_k, lam, mu, lam_prev, grad_src: device N doubles (lam_prev may
 * alias lam); grad_k: DEVICE array of 2 doubles.  Synchronises the stream. */
int rsfde_adjoint_step(rsfde_ctx* ctx, const double* u_prev, const double* u_k, const double* lam, double* mu,
                       double* lam_prev, double* grad_src, double* grad_k, rsfde_stats* stats);

/* ---- batched instances ------------------------------------------------------ */
/* Many independent problems (each its own grid, mask, alphas, k, dt, eta)
 * advanced together; one CUDA graph launch advances the whole batch by one
 * step.  With right-preconditioned FGMRES, the FP32 operator and either the
 * FP32 preconditioner (FP64 basis with the FP64 or exact true residual, or FP32
 * basis with the FP64 one) or the split-BF16 one (FP64 basis, FP64 or exact
 * residual), the instances run in lock step: every kernel
 * of the FGMRES cycle is one launch over all instances still iterating (the
 * split-BF16 GEMMs of all instances in one grouped launch per pass), with
 * each instance's results bit-identical to its single-instance solve (up to
 * 1024 instances, grid sides up to 2048).  Other options run every
 * instance's step as one branch of the graph.  The paper solves one
 * instance; this is the batched deployment of the same step.  Arguments
 * are arrays of `count` entries (grids, masks: device pointers as in
 * rsfde_setup); opts (may be NULL) apply to all. */
int rsfde_batch_create(rsfde_batch** out, int32_t count, const rsfde_grid* grids, const uint8_t* const* masks,
                       const double* alpha1, const double* alpha2, const double* kx, const double* ky,
                       const double* dt, const double* eta, const rsfde_opts* opts);
/* Sets instance i's u^0 (device, N_i doubles) and source (device or NULL); restarts its march. */
int rsfde_batch_set(rsfde_batch* b, int32_t i, const double* u0, const double* src);
/* Advances every instance by `steps` implicit steps (f = u - u^3 + src, Eq. 2.17).
 * stats: HOST array of `count` (statistics of each instance's last step) or
 * NULL.  Returns RSFDE_ETIMEOUT if a grouped split-BF16 GEMM's pipeline wait
 * gave up (its output was incomplete; the batch stays usable), else the first
 * non-OK instance status, else RSFDE_OK.  Synchronises. */
int rsfde_batch_run(rsfde_batch* b, int32_t steps, rsfde_stats* stats);
/* Copies instance i's current u^k to the device array u_out (N_i doubles). */
int rsfde_batch_get(rsfde_batch* b, int32_t i, double* u_out);
int64_t rsfde_batch_kernel_launches(rsfde_batch* b);
void rsfde_batch_destroy(rsfde_batch* b);

/* ---- operator-level entry points (each one step of the hot path) --------- */
/* Eq. 2.14-2.17: w = M z in the context's operator precision (matvec_prec).
 * z, w device N doubles (distinct). */
int rsfde_apply_M(rsfde_ctx* ctx, const double* z, double* w);
/* The true residual r = b - M x (Eq. 2.17's system) with M x in the context's
 * resid_prec, RSFDE_FP64 or RSFDE_EXACT (RSFDE_DF32: RSFDE_EINVAL).  x, b, r
 * device N doubles (r distinct from x and b). */
int rsfde_residual(rsfde_ctx* ctx, const double* x, const double* b, double* r);
/* Eq. 4.6: z = P-hat^-1 v in the context's preconditioner precision (result in FP64). */
int rsfde_apply_precond(rsfde_ctx* ctx, const double* v, double* z);
/* Section 4.1: out = (S_{n2} (x) S_{n1}) v, the orthonormal 2D sine transform, FP64. */
int rsfde_dst2(rsfde_ctx* ctx, const double* v, double* out);
/* Right side and initial guess of rsfde_step: b and x0 device N doubles. */
int rsfde_rhs(rsfde_ctx* ctx, const double* u_prev, const double* u_prevprev, const double* src,
              double* b, double* x0);
/* Setup tables copied to HOST arrays: eigenvalues of tau(A_x) (n1) and tau(A_y) (n2),
 * and the scaled Toeplitz first columns t_x (n1), t_y (n2).  Any pointer may be NULL. */
int rsfde_get_tables(rsfde_ctx* ctx, double* lam_x, double* lam_y, double* t_x, double* t_y);
/* c_x, c_y, dt/eta, h_x, h_y to a HOST array of 5 doubles. */
int rsfde_get_params(rsfde_ctx* ctx, double* out5);

/* ---- allocation-free variant ------------------------------------------------ */
/* The paper has no counterpart to this entry point: it exists for callers
 * that cannot call cudaMalloc, such as an application or framework that owns
 * every device allocation through its own memory pool (a stray cudaMalloc
 * would bypass its accounting or fragment the memory it manages).  They
 * cannot make an rsfde_ctx (rsfde_setup allocates), so this call computes
 * out = (S_{n2} (x) S_{n1}) v -- the same transform and kernels as
 * rsfde_dst2 -- with no context.
 *
 * v, out: caller-owned DEVICE arrays of n1*n2 doubles, x fastest, distinct.
 * stream: cudaStream_t or NULL.  The intermediate between the row and column
 * passes and the transform tables live in static device arrays of the
 * library (about 2.1 MB, held by every GPU that loads the library until the
 * process exits), so sizes are limited: n1, n2 in 1..RSFDE_NOALLOC_MAX_N,
 * else RSFDE_EINVAL.  Calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * The first call on each device looks up the static arrays' device
 * addresses (cudaGetSymbolAddress) with that device current.  A call whose (n1, n2) or stream
 * differs from the previous call's on that device copies the tables from
 * host memory, which makes the host wait for the stream's earlier work; a
 * repeat with the same sizes and stream reuses them.  Every call uses the
 * same static arrays and overwrites all of them that its kernels read, so
 * nothing carries over from one call to the next; calls whose work overlaps
 * on the GPU (two streams, or two devices' work racing on one device's
 * arrays from several host threads) race on the arrays and must be
 * serialised by the caller.  The host side of the call is serialised
 * internally. */
#define RSFDE_NOALLOC_MAX_N 512
int rsfde_dst2_noalloc(int32_t n1, int32_t n2, const double* v, double* out, void* stream);

/* ---- measurement ------------------------------------------------------------ */
/* Kernel classes timed by the profiler. */
#define RSFDE_K_TOEPLITZ_ROWS 0 /* (I (x) A_x) z, Eq. 2.15 */
#define RSFDE_K_TOEPLITZ_COLS 1 /* (A_y (x) I) z fused with the rest of M (or the residual) */
#define RSFDE_K_DST_ROWS 2      /* first row sine transform of Eq. 4.6 */
#define RSFDE_K_PRECOND_COLS 3  /* column sine transforms and tau divides of Eq. 4.6 */
#define RSFDE_K_PRECOND_ROWS 4  /* last row sine transforms and the masked combine of Eq. 4.6 */
#define RSFDE_K_MULTIDOT 5      /* Arnoldi inner products */
#define RSFDE_K_UPDATE 6        /* Arnoldi update, norm and Givens step */
#define RSFDE_K_XUPDATE 7       /* solution update x += Z y */
#define RSFDE_K_OTHER 8         /* right side, norms, scalar kernels */
#define RSFDE_K_DST_GEMM 9      /* preconditioner as tensor-core GEMMs (split-BF16 or BF16): the four
                                   GEMMs and, when the previous Gram-Schmidt update did not write the
                                   first operand, the split */
#define RSFDE_K_RESID_ROWS 10   /* row pass of M x in the true residual (Eq. 2.15) */
#define RSFDE_K_RESID_COLS 11   /* column pass of the true residual b - M x and its norm */
#define RSFDE_K_SOLVE_Y 12      /* back substitution of the Givens-rotated least squares */
#define RSFDE_K_COUNT 13

/* While on, every kernel launch of the context is bracketed by a pair of CUDA
 * events on the context's stream (adds one event record per launch). */
int rsfde_profile_enable(rsfde_ctx* ctx, int on);
/* Synchronises the stream and writes, per kernel class, the summed device
 * time in ms (HOST array of RSFDE_K_COUNT doubles) and the number of launches
 * (HOST array of RSFDE_K_COUNT int64), then clears the accumulators. */
int rsfde_profile_read(rsfde_ctx* ctx, double* ms, int64_t* launches);
const char* rsfde_kernel_class_name(int k);

/* Tile-shape autotuner.  The transform kernels process F vectors (rows or
 * columns) per block; for the context's transform lengths and precisions
 * this times every feasible F of each kernel family (reps calls each, CUDA
 * events on the context's stream, on its own buffers) and records the
 * fastest in a process-wide table that every later launch with the same
 * length and precision uses (captured graphs are rebuilt).  With a
 * tensor-core preconditioner it also times each of its four GEMMs with 64-
 * and 128-wide tiles and records the faster width in the context.  chosen: HOST
 * array of RSFDE_TUNE_COUNT int32 (the chosen F per family, 0 = not tuned)
 * or NULL.  With a double-FP32 true residual and an operator in another
 * precision, the 8-byte shapes are timed on the residual's own two passes.
 * Overwrites the context's Krylov workspace, its internal right-hand side and
 * iterate, and its solver state (every solve and step re-initialises them). */
#define RSFDE_TUNE_COUNT 10 /* F of: Toeplitz rows, Toeplitz columns, sine rows, sine columns,
                               preconditioner columns, preconditioner rows; then the tile width
                               (64 or 128) of each of the tensor-core preconditioner's four GEMMs */
int rsfde_autotune(rsfde_ctx* ctx, int32_t reps, int32_t* chosen);
int rsfde_batch_autotune(rsfde_batch* b, int32_t reps);

/* Failure detection.  Every wait of the tensor-core preconditioner's
 * pipeline (a TMA copy landing in a ring slot, a slot freed by the MMAs) is
 * bounded; a wait that runs out makes that launch give up and the call
 * return RSFDE_ETIMEOUT, after every copy and MMA the launch had issued has
 * completed, so the context stays usable.  cycles: the bound of each such
 * wait in SM clock cycles; 0 restores the default (4e9, about 2 s at
 * 2.07 GHz).  A small bound makes the waits give up on purpose, which is how
 * the timeout path is tested.  The waits that let issued work complete
 * before a block frees its memory keep the default bound. */
int rsfde_set_wait_cycles(rsfde_ctx* ctx, int64_t cycles);

/* Number of this library's kernel launches since the context was made (host counter). */
int64_t rsfde_kernel_launches(const rsfde_ctx* ctx);

void rsfde_destroy(rsfde_ctx* ctx);
const char* rsfde_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* RSFDE_H */
