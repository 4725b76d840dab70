/*
 * tfde.h -- C ABI of the GB300 (sm_103a) solver library for the Crank-Nicolson
 * finite-volume discretisation of the 3-D conservative two-sided
 * Riemann-Liouville space-fractional diffusion equation, with the DST-I
 * (tau) preconditioned PCG / PGMRES solvers of Qu, Lei, Hon and Huang,
 * "Optimal preconditioning techniques for finite volume approximation of
 * three-dimensional conservative space-fractional diffusion equations".
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - A grid function is n1*n2*n3 doubles in the paper's lexicographic order
 *   (Sec. 2, definition of u^m): x fastest, then y, then z, i.e. element
 *   (i, j, k) (0-based) sits at i + n1*(j + n2*k).
 * - Vector arguments are DEVICE pointers (cudaMalloc / torch CUDA storage on the
 *   current device), owned by the caller, 8-byte aligned; they must not alias
 *   unless an argument says so.  Host pointers are rejected only when the CUDA
 *   runtime reports them as host memory (TFDE_EINVAL).
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   All work is enqueued on it.  Solver entry points synchronise the stream
 *   for their convergence tests; matvec / precond / source do not.
 * - A tfde_problem owns every device buffer it needs (operators, eigenvalue
 *   arrays, Krylov workspace).  It is created by tfde_assemble and released by
 *   tfde_destroy.  One problem must not be used from two host threads or two
 *   streams at once (its workspace is shared by all its calls).
 * - Every function returns a tfde_status; nothing aborts or throws across the
 *   ABI.  tfde_last_error() returns a thread-local message for the last
 *   failure on the calling thread.  Asynchronous kernel faults surface as
 *   TFDE_ECUDA at the next synchronising call.
 */
#ifndef TFDE_H
#define TFDE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TFDE_OK = 0,
    TFDE_EINVAL = 1,        /* invalid argument (sizes, orders, pointers)        */
    TFDE_ENOMEM = 2,        /* device or host allocation failed                  */
    TFDE_ECUDA = 3,         /* CUDA runtime / driver error                       */
    TFDE_ENOCONV = 4,       /* maxit reached before the tolerance                */
    TFDE_EBREAKDOWN = 5,    /* Krylov breakdown (p.Ap <= 0, zero Arnoldi norm)   */
    TFDE_ENAN = 6,          /* NaN or Inf in a residual or inner product         */
    TFDE_ETIMEOUT = 7,      /* a bounded device-side wait ran out                */
    TFDE_EUNSUPPORTED = 8   /* valid request this build does not implement       */
} tfde_status;

typedef enum {
    /* every operator, transform and Krylov vector in native FP64 */
    TFDE_FP64 = 0,
    /* inner Krylov solves on FP32 vectors with split-BF16 tcgen05 contractions
       (Toeplitz matvec: 3 BF16 products; DST: 2), wrapped in FP64 iterative
       refinement whose residual uses the exact-integer slice (Ozaki) tcgen05
       contraction; the stopping test is always the true FP64 residual.
       Grids the contraction does not take (an n_a that is not a multiple of
       8 or above 448, and the 2-D problem) run the same FP64 refinement
       around FP32 inner solves on the FFT passes (FFT-embedded Toeplitz
       products, DST-I by FFT), the residual on the FP64 FFT passes; these
       need every n_a <= 2048 */
    TFDE_MIXED = 1
} tfde_precision;

/* One problem (Sec. 1 and Sec. 2).  Axis a = 0, 1, 2 is x, y, z.
 * n[2] = 0 selects the two-dimensional problem of Sec. 4, Example 1 on
 * (lo_0, hi_0) x (lo_1, hi_1): the system of Eq. (linear_sys) without the
 * third axis (A = A_2 (x) A_1 + eta_a A_2 (x) B_1 + eta_b B_2 (x) A_1); the
 * third entries of delta, kp, km, lo, hi are then ignored, grid functions hold
 * n1*n2 values; TFDE_MIXED runs on the FFT passes. */
typedef struct {
    int n[3];          /* interior grid points per axis, n_a >= 1 (n[2] = 0: 2-D); h_a = (hi_a - lo_a)/(n_a + 1) */
    double lo[3];      /* Omega = prod_a (lo_a, hi_a), lo_a < hi_a                  */
    double hi[3];
    double delta[3];   /* alpha, beta, gamma in (0, 1); the derivative order is 2 - delta */
    double kp[3];      /* k_{a,+} > 0                                               */
    double km[3];      /* k_{a,-} > 0                                               */
    double dt;         /* Crank-Nicolson step Delta t > 0                           */
} tfde_params;

/* Filled by the solver entry points (may be NULL). */
typedef struct {
    int iters;          /* PCG iterations / GMRES inner (Arnoldi) steps, all sweeps  */
    int restarts;       /* GMRES cycles started                                      */
    int refine_sweeps;  /* FP64 refinement sweeps (TFDE_MIXED), else 0               */
    int fallback;       /* 1 if a mixed solve fell back to FP64 inner solves         */
    double relres;      /* final true relative residual ||b - A x||_2 / ||b||_2     */
    double relres0;     /* initial true relative residual                            */
    float ms;           /* wall time of the call, milliseconds                       */
} tfde_info;

typedef struct tfde_problem tfde_problem;

/* Operator selectors for tfde_matvec. */
#define TFDE_OP_A    0   /* y = A x, A the CN-FV matrix of Eq. (linear_sys)          */
#define TFDE_OP_RHS  1   /* y = (A_N - eta-terms) x = (2 A_N - A) x, the RHS operator */
#define TFDE_OP_FAST 2   /* OR-able: for TFDE_MIXED problems use the inner (split-BF16,
                            FP32-accumulated, or FP32 FFT) arithmetic instead of the accurate one */
#define TFDE_OP_STIFF 4  /* y = (A - A_N) x = eta_a A3(x)A2(x)B1 x + eta_b A3(x)B2(x)A1 x +
                            eta_c B3(x)A2(x)A1 x, the three stiffness terms alone (not with FAST) */

/*
 * tfde_assemble -- build a problem (Sec. 2, Eq. (coef_expression) to Eq. (linear_sys);
 * Sec. 3, Eq. (pre_definition) and Eq. (diag_tau_pre)).
 *   Computes h_a, eta_a = dt / (2 Gamma(delta_a + 1) h_a^{2 - delta_a}), the
 *   generators q_k (k = 0..n_a) without cancellation, the dense per-axis
 *   operators eta_a B_a and the DST-I matrices S_{n_a}, the tau eigenvalues
 *   lambda_k = q_1 + (q_0+q_2) cos t_k + sum_{j=2}^{n-1} q_{j+1} cos(j t_k)
 *   and the mass eigenvalues (6 + 2 cos t_k)/8, and allocates the workspace.
 *   Errors: TFDE_EINVAL for n_a < 1, delta outside (0,1), k <= 0, dt <= 0,
 *   lo >= hi, NULL pointers; TFDE_EUNSUPPORTED when TFDE_MIXED is requested
 *   on a grid the tensor-core contraction does not take (an n_a that is not
 *   a multiple of 8 -- tensor-map row alignment -- or above 448, where the
 *   exact-integer residual's FP32 accumulators would pass 2^24, or 2-D) and
 *   the FFT passes do not either (an n_a above 2048);
 *   TFDE_ENOMEM / TFDE_ECUDA.  *out is NULL on failure.  Synchronises `stream`.
 */
int tfde_assemble(const tfde_params* params, int precision, void* stream, tfde_problem** out);

/* Release every resource of a problem (NULL is a no-op).  Synchronises the device. */
int tfde_destroy(tfde_problem* prob);

/*
 * tfde_matvec -- y = A x (op TFDE_OP_A) or y = (2 A_N - A) x (op TFDE_OP_RHS),
 * Eq. (linear_sys):  A = A_N + eta_a A3(x)A2(x)B1 + eta_b A3(x)B2(x)A1 + eta_c B3(x)A2(x)A1.
 *   x, y: device, n1*n2*n3 doubles, must not alias.  Asynchronous.
 */
int tfde_matvec(const tfde_problem* prob, int op, const double* x, double* y, void* stream);

/*
 * tfde_precond -- z = P^{-1} r = S_N Lambda^{-1} S_N r, Eq. (diag_tau_pre).
 *   r, z: device, n1*n2*n3 doubles; z may alias r.  Asynchronous.
 */
int tfde_precond(const tfde_problem* prob, const double* r, double* z, void* stream);

/*
 * tfde_pcg -- solve A x = b by tau-preconditioned CG (Sec. 3.1; requires
 * k_{a,+} = k_{a,-} on every axis, else TFDE_EINVAL).
 *   b: device input; x: device, initial guess on entry, solution on exit.
 *   Stops when ||b - A x||_2 <= tol ||b||_2 for the TRUE residual (the
 *   recursive residual only triggers the check).  maxit bounds the iterations
 *   (all refinement sweeps together).  Returns TFDE_ENOCONV if maxit is hit,
 *   TFDE_EBREAKDOWN if p.Ap <= 0, TFDE_ENAN on a non-finite residual.
 */
int tfde_pcg(const tfde_problem* prob, const double* b, double* x, double tol, int maxit,
             tfde_info* info, void* stream);

/*
 * tfde_pgmres -- solve A x = b by restarted GMRES(restart) on the left
 * preconditioned system P^{-1} A x = P^{-1} b (Sec. 3.2, Eq. (one_side_system)).
 *   Arnoldi with classical Gram-Schmidt and one re-orthogonalisation; Givens
 *   rotations in FP64 on the host.  Converged when the TRUE relative residual
 *   ||b - A x|| / ||b|| <= tol.  1 <= restart <= 64.  Errors as tfde_pcg.
 */
int tfde_pgmres(const tfde_problem* prob, const double* b, double* x, int restart, double tol,
                int maxit, tfde_info* info, void* stream);

/*
 * tfde_cn_step -- one Crank-Nicolson step u^{m-1} -> u^m (Sec. 2, Eq. (CN) and
 * Eq. (linear_sys)):  b = (2 A_N - A) u^{m-1} + dt F^{m-1/2};  solve A u^m = b
 * by PCG when k_+ = k_- on every axis, else by PGMRES(20).
 *   u_prev: device input.  F_half: device cell averages of f at t_{m-1/2}, or
 *   NULL for f = 0.  x0: device initial guess, or NULL for u_prev.  u_next:
 *   device output; may alias x0 but not u_prev or F_half.  maxit = 10000.
 */
int tfde_cn_step(const tfde_problem* prob, const double* u_prev, const double* F_half,
                 const double* x0, double* u_next, double tol, tfde_info* info, void* stream);

/*
 * tfde_cn_advance -- one Crank-Nicolson step u^{m-1} -> u^m IN PLACE, for
 * marching many steps on one problem (Sec. 2, Eq. (CN) and Eq. (linear_sys)).
 *   Same result and stopping rule as tfde_cn_step with x0 = u^{m-1}, but the
 *   problem keeps the right-hand side b^{m-1} and final true residual r^{m-1}
 *   of the previous call, and uses A u^{m-1} = b^{m-1} - r^{m-1}: the new
 *   right-hand side needs only the mass operator A_N, and the initial residual
 *   no operator application at all.  The first call (restart != 0) instead
 *   evaluates the stiffness terms K u once and uses b = A_N u - K u + dt F,
 *   r_0 = dt F - 2 K u.
 *   u: device, in/out.  The chain is valid only while u is the same pointer as
 *   in the previous call and nothing else wrote it in between; pass restart = 1
 *   on the first call and whenever that does not hold (also after any other
 *   solver call on the same problem, which reuses the same workspace).
 *   F_half: device cell averages at t_{m-1/2}, or NULL for f = 0.
 *   Errors as tfde_cn_step; after an error the next call must restart.
 */
int tfde_cn_advance(const tfde_problem* prob, double* u, const double* F_half, int restart, double tol,
                    tfde_info* info, void* stream);

/*
 * tfde_cn_advance_host -- tfde_cn_advance (Sec. 2, Eq. (CN)) for a state kept
 * in HOST memory: u^{m-1} is copied from u_host_in into the device state u,
 * the step runs as tfde_cn_advance(prob, u, F_half, restart, tol), and u^m is
 * copied to u_host_out (and stays in u, so that the next call chains on it).
 *   The copies overlap the step's own work: the input copy runs on a stream
 *   of the problem's own, beside the work that reads no u (the minimal-
 *   residual sums of the order-3 guess), and the output copy leaves as soon
 *   as an iterate that may be final exists, while the exact residual that
 *   decides it is formed (a later write of u waits for that copy and is
 *   copied again).  Page-locked host buffers are needed for the copies to
 *   overlap; u_host_out may alias u_host_in.
 *   u_host_in, u_host_out: host, N doubles each.  u: device, N doubles.
 *   Chain, F_half and errors as tfde_cn_advance (TFDE_EINVAL also for a NULL
 *   or device host buffer).  Synchronises `stream`.
 */
int tfde_cn_advance_host(const tfde_problem* prob, const double* u_host_in, double* u_host_out, double* u,
                         const double* F_half, int restart, double tol, tfde_info* info, void* stream);

/*
 * tfde_cn_advance_guess -- tfde_cn_advance with a candidate initial guess x0
 * (e.g. from the warm-start network): the solve starts from the point
 * u^{m-1} + c (x0 - u^{m-1}) of least FP64 residual ||b^m - A x||, c >= 0
 * (c = 1: x0 itself), when that residual is smaller than the one of u^{m-1},
 * else from u^{m-1} (the previous-step guess stays the fallback; the
 * stopping rule is the same).  The residual of x0 costs one accurate
 * operator application on x0 - u^{m-1} (A u^{m-1} is known from the chain);
 * c costs three inner products.  *used_guess (may be NULL) is set to 1 when
 * x0 contributed (c > 0).  x0: device, not aliasing u.  The
 *   polynomial extrapolation of tfde_set_guess_order is not applied on such a
 *   step, and its history restarts.  Errors as tfde_cn_advance.
 */
int tfde_cn_advance_guess(const tfde_problem* prob, double* u, const double* F_half, const double* x0, int restart,
                          double tol, tfde_info* info, int* used_guess, void* stream);

/*
 * tfde_set_guess_order -- initial guess of the chained tfde_cn_advance steps:
 *   order 0 (default): x0 = u^{m-1}, as the paper's solves from the previous
 *   time level; order 1: x0 = 2u^{m-1} - u^{m-2}; order 2:
 *   x0 = 3u^{m-1} - 3u^{m-2} + u^{m-3} (polynomial extrapolation in time).
 *   The problem then keeps (u, A u) of the two previous levels (4 vectors of
 *   n_1 n_2 n_3 doubles, allocated on first use); A x0, and with it the
 *   initial residual, is the same combination of the stored A u, so the guess
 *   costs one fused vector pass.  Order 3: the order-2 guess plus
 *   c1 (u^{m-1} - u^{m-2}) + c2 (u^{m-1} - 2u^{m-2} + u^{m-3}), with (c1, c2)
 *   minimising the 2-norm of the initial residual over that plane, from five
 *   sums over the stored A u (one more read-only vector pass; the 2 x 2
 *   system is solved on the device, no host read; the polynomial
 *   coefficients do not follow
 *   the CN transient of the stiff modes, and at the n = 256 workload the
 *   correction lowers the initial residual ~40-fold).  The order in force is
 *   limited by the history the chain has built since its last restart (the
 *   restart step stores the first level from the products it forms anyway,
 *   so the next step extrapolates at order 1 and the one after at up to
 *   order 3).
 *   The guess changes only the iterations, not the stopping rule.
 *   Errors: TFDE_EINVAL for order outside 0..3 or a NULL problem.
 */
int tfde_set_guess_order(tfde_problem* prob, int order);

/*
 * tfde_set_device_loop -- how the inner PCG of a TFDE_MIXED problem runs its
 * iterations (Sec. 3.1; no effect on TFDE_FP64 problems or on PGMRES).
 *   enable != 0 (default): each refinement sweep's inner iterations run as one
 *   CUDA graph launch, a device-side while loop whose stop test (the inner
 *   residual norm against the sweep's target) is taken on the device; the host
 *   reads the iteration count and residual once per sweep.  enable = 0: the
 *   host takes the stop test after every iteration (one blocking read each).
 *   Both give the same iterates.  While tfde_stats_reset(1) times every
 *   tensor-core launch, the host-driven loop is used.  The graph is built on
 *   the problem's first sweep and captures its workspace pointers; it is
 *   released with the problem.  Errors: TFDE_EINVAL for a NULL problem.
 */
int tfde_set_device_loop(tfde_problem* prob, int enable);

/*
 * tfde_device_loop_launches -- how many inner solves of a TFDE_MIXED problem
 * on the tensor-core path (PCG sweeps and GMRES cycles, Sec. 3.1-3.2) so far
 * ran as one CUDA-graph launch with the stop test on the device (see
 * tfde_set_device_loop); 0 for other problems and a NULL problem.  The
 * graphs are captured on a stream of the library's own, so they serve
 * callers on any stream, the legacy default stream included.
 */
long long tfde_device_loop_launches(const tfde_problem* prob);

/*
 * tfde_set_spectral_inner -- the basis in which the inner Krylov solves of a
 * TFDE_MIXED problem on the tensor-core path iterate: PCG (Sec. 3.1) and
 * left-preconditioned GMRES (Sec. 3.2, Eq. (one_side_system)) with the tau
 * preconditioner P = S_N Lambda S_N of Eq. (diag_tau_pre).
 *   enable != 0 (default): in the sine-transform eigenbasis.  S_N is
 *   symmetric and orthogonal and diagonalises P and the mass operator A_N, so
 *   the preconditioned system becomes S_N A S_N with the diagonal Lambda: the
 *   residual is transformed once per refinement sweep (three split-BF16
 *   passes with S_n split into hi + lo), each iteration applies S_N A S_N as
 *   three split passes (one per axis: S_n eta_a B_a S_n along the axis, the
 *   other axes' mass eigenvalues as per-line factors; for GMRES Lambda^{-1}
 *   fused into the last) and the preconditioner pointwise, and the
 *   correction goes back through S_N once per sweep.  The same iterates as
 *   enable = 0 in exact arithmetic; 3 instead of 9 tensor-core passes per
 *   iteration.
 *   enable = 0: the grid basis (operator in 3 and preconditioner in 6 split
 *   passes per iteration).
 * The refinement's FP64 residual, and so the result's accuracy, are the same
 * either way.  The batched solver always iterates in the grid basis.
 * Errors: TFDE_EINVAL for a NULL problem; TFDE_EUNSUPPORTED when enable != 0
 * for a TFDE_FP64 problem or a TFDE_MIXED problem on the FFT passes (enable =
 * 0 is accepted and has no effect there).
 */
int tfde_set_spectral_inner(tfde_problem* prob, int enable);

/*
 * tfde_spectrum -- spectral estimates of the preconditioned system of one
 * problem (Sec. 3) at sizes far beyond a dense eigensolve, in FP64 on the FFT
 * passes.  With H(A) = (A + A^T)/2 and S(A) = (A - A^T)/2 (Sec. 2 notation):
 *   sym_min, sym_max  extreme Ritz values of P^{-1/2} H(A) P^{-1/2} after
 *                     `steps` Lanczos steps from v0 (Theorem
 *                     CG_bounded_sprctrum, Lemma prop:eigen_S: the spectrum
 *                     lies in (1/2, 3/2));
 *   skew_rho          largest Ritz value of the spectral radius of
 *                     P^{-1/2} S(A) P^{-1/2} (Lanczos on its negated square;
 *                     0 when k_+ = k_- on every axis), against
 *   varsigma          the bound of Lemma eigen_Skew,
 *                     3/2 max_a tan(delta_a pi / 2) |k_{a,+} - k_{a,-}| / (k_{a,+} + k_{a,-});
 *   omega             the GMRES rate sqrt((2 + 4 varsigma^2) / (3 + 4 varsigma^2))
 *                     of Theorem theorem_main, and
 *   omega_est         the same bound from the estimates:
 *                     sqrt(1 - sym_min^2 / (sym_min sym_max + skew_rho^2)).
 *   Ritz values lie inside the spectrum: sym_min / sym_max approach the
 *   extremes from inside, skew_rho the radius from below.
 *   params: as tfde_assemble (every n_a <= 2048).  steps: 2..500.  v0: device
 *   grid function, the start vector (not zero).  out: host.  Errors:
 *   TFDE_EINVAL, TFDE_EUNSUPPORTED, TFDE_ENOMEM, TFDE_ENAN, TFDE_ECUDA.
 *   Allocates two FP64 problems for the call.  Synchronises `stream`.
 */
typedef struct {
    int steps;
    double sym_min, sym_max, skew_rho, varsigma, omega, omega_est;
} tfde_spectrum_info;
int tfde_spectrum(const tfde_params* params, int steps, const double* v0, tfde_spectrum_info* out, void* stream);

/* ------------------------------------------------------------------ batches */
typedef struct tfde_batch tfde_batch;

/*
 * tfde_batch_create -- `count` independent problems of possibly different
 * sizes and coefficients (params[0..count-1], each as for tfde_assemble with
 * TFDE_MIXED: every n_a a multiple of 8 and at most 448), solved together.
 *   Each problem takes the CN step of Eq. (CN) / Eq. (linear_sys) inside FP64
 *   iterative refinement, with PCG (Sec. 3.1) when it is symmetric (k+ = k-
 *   on every axis; see tfde_batch_set_symmetric_pcg) and left-preconditioned
 *   restarted GMRES(restart) (Sec. 3.2, Eq. (one_side_system)) otherwise.
 *   The problems advance in lock step through the Krylov iterations: every
 *   split-BF16 operator or preconditioner pass is one persistent tensor-core
 *   launch over a work list of the tiles of all problems (largest problems
 *   first), every vector step one launch over all problems, and a problem
 *   whose inner cycle has met its target drops out of the work lists.  The
 *   FP64 residual of each refinement sweep is evaluated per problem (exact
 *   slice contraction) on a pool of streams.
 *   1 <= count <= 1024, 1 <= restart <= 63.  Errors: as tfde_assemble for any
 *   problem; TFDE_EINVAL for count/restart out of range.  *out is NULL on
 *   failure.  Synchronises `stream`.  Device memory: the workspace of each
 *   problem plus (restart + 1) FP32 basis vectors per problem.
 */
int tfde_batch_create(const tfde_params* params, int count, int restart, void* stream, tfde_batch** out);

/* Release a batch and all its problems (NULL is a no-op).  Synchronises the device. */
int tfde_batch_destroy(tfde_batch* batch);

/* Number of problems of a batch (0 for NULL). */
int tfde_batch_count(const tfde_batch* batch);

/*
 * tfde_batch_set_guess_order -- the initial guess of tfde_batch_cn_advance's
 *   chained steps for every problem of the batch, as tfde_set_guess_order
 *   (orders 0..3, 0 by default; each problem keeps its own history).
 *   Errors: TFDE_EINVAL for a NULL batch or an order outside 0..3.
 */
int tfde_batch_set_guess_order(tfde_batch* batch, int order);

/*
 * tfde_batch_set_spectral_inner -- the basis of the batched GMRES cycles
 * (Sec. 3.2), as tfde_set_spectral_inner for one problem: enable != 0
 * (default) runs every Arnoldi step as three grouped split passes of
 * Lambda^{-1} S_N A S_N over all problems' tiles, with one forward (Lambda^{-1}
 * fused) and one backward sine transform per cycle; enable = 0 the grid basis
 * (five operator and six preconditioner passes per step).  Errors:
 * TFDE_EINVAL for a NULL batch.
 */
int tfde_batch_set_spectral_inner(tfde_batch* batch, int enable);

/*
 * tfde_batch_set_symmetric_pcg -- the inner solver of the batch's symmetric
 * problems (k+ = k- on every axis): enable != 0 (default) solves them by PCG
 * (Sec. 3.1) in lock step, in the sine-transform eigenbasis where the tau
 * preconditioner is the diagonal Lambda (Eq. (diag_tau_pre)): per iteration
 * three grouped split passes of S_N A S_N over every symmetric problem's
 * tiles, <p, A p> per problem fused into the last, then one update, one
 * stop-test and one direction launch over all of them; per refinement sweep
 * one forward and one backward sine transform.  A problem leaves when its
 * inner residual has dropped by the sweep's target or after 100 iterations.
 * The iterations of a sweep run as one CUDA-graph launch (a while node; the
 * iteration index, the stop tests and the loop condition on the device)
 * unless tfde_stats_reset(1) times every tensor-core launch (the host then
 * drives them, learning the count of problems left one iteration late).
 * The non-symmetric problems keep GMRES.  enable = 0, or the grid basis
 * (tfde_batch_set_spectral_inner(batch, 0)), sends every problem through
 * GMRES.  Errors: TFDE_EINVAL for a NULL batch.
 */
int tfde_batch_set_symmetric_pcg(tfde_batch* batch, int enable);

/* tfde_batch_pcg_solves -- inner solves (one per problem and refinement
 * sweep) run so far by the batched PCG; 0 for a NULL batch. */
long long tfde_batch_pcg_solves(const tfde_batch* batch);

/* tfde_batch_pcg_graph_launches -- refinement sweeps whose batched PCG
 * iterations ran as one graph launch; 0 for a NULL batch. */
long long tfde_batch_pcg_graph_launches(const tfde_batch* batch);

/* tfde_batch_grouped_prepares -- batched CN steps whose right-hand sides,
 * corrected order-3 guesses and initial residuals (Eq. (linear_sys) on the
 * chain) ran as grouped launches over all problems: the steady state of a
 * chain in which every problem has its mass term from the previous step's
 * exact residual and two history levels (else each problem prepares its own
 * step).  0 for a NULL batch. */
long long tfde_batch_grouped_prepares(const tfde_batch* batch);

/*
 * tfde_batch_graph_cycles -- how many batched GMRES cycles (Sec. 3.2) so far
 * ran their Arnoldi steps as one CUDA-graph launch (a while node: the step
 * index, each problem's Hessenberg column, Givens rotation and stop test,
 * and the loop condition on the device; no host read inside a cycle).  The
 * eigenbasis cycles take that path unless tfde_stats_reset(1) times every
 * tensor-core launch (the host then drives the steps) or the graph could not
 * be built.  Returns 0 for a NULL batch.
 */
long long tfde_batch_graph_cycles(const tfde_batch* batch);

/*
 * tfde_batch_cn_advance -- one CN step u_i^{m-1} -> u_i^m IN PLACE for every
 * problem i of the batch, with the chained right-hand side and initial
 * residual of tfde_cn_advance (x0 = u_i^{m-1}).
 *   u: host array of `count` device pointers (in/out, distinct), in the order
 *   of the params given to tfde_batch_create.  F_half: host array of `count`
 *   device pointers to the source cell averages (entries may be NULL for
 *   f = 0), or NULL for f = 0 everywhere.  restart: as tfde_cn_advance (1 on
 *   the first call and whenever any u_i was written in between).  Stopping
 *   rule per problem: ||b_i - A_i u_i|| <= tol ||b_i|| in FP64.  infos: host
 *   array of `count` results (may be NULL); ms is the wall time of the whole
 *   batched step.  Returns TFDE_OK when every problem converged, else the
 *   first failing status (TFDE_ENOCONV, TFDE_ENAN, ...).  Synchronises `stream`.
 */
int tfde_batch_cn_advance(tfde_batch* batch, double* const* u, const double* const* F_half, int restart, double tol,
                          tfde_info* infos, void* stream);

/* ---------------------------------------------------------------- autotuner */
/*
 * Autotuner of the tensor-core contraction's launch parameters (no
 * counterpart in the paper): the number of persistent CTAs (the SM count,
 * the count that deals the tiles evenly over the same number of waves, 7/8
 * and 3/4 of the SMs) and the depth of the operand ring (2 .. 4 stages of
 * 48 KB, or 2 of 96 KB), per launch class.  A class is the kernel instance
 * (grouped, operand layout, output mode), the stage size, the rows n of the
 * contraction (0 for grouped launches) and the number of 128 x 256 tiles.
 *
 * tfde_tune records the launches of one operator and one preconditioner
 * application of a TFDE_MIXED problem on the tensor-core path, times each
 * class's candidates (one warm-up launch, then `reps` launches between CUDA
 * events on `stream`) and keeps the fastest in a process-wide table that
 * every later launch of that class uses (device-side loop graphs captured
 * before are recaptured).  tfde_batch_tune does the same for a batch's
 * grouped launches.  Call between solves: the trials overwrite the inner
 * solvers' scratch vectors and the batch's activity mask.  Errors:
 * TFDE_EUNSUPPORTED for a problem off the tensor-core path, TFDE_EINVAL for
 * NULL or reps outside [1, 1000], TFDE_ECUDA.  Synchronises `stream`.
 *
 * tfde_tune_get copies up to `cap` entries of the table into out (host
 * memory) and sets *count to the number copied; tfde_tune_set adds or
 * replaces `count` entries (a caller caches the table, e.g. as JSON keyed by
 * the GPU name, and applies it in a fresh process before assembling);
 * tfde_tune_clear empties it.  Not thread-safe.
 */
typedef struct {
    int grouped;      /* 1: one launch over the tiles of several contractions   */
    int kmajor;       /* operand layout: 1 for x-axis contractions              */
    int out_mode;     /* 0 FP32, 1 split planes, 2 direction update, 3 hi plane */
    int stage_bytes;  /* ring stage size of the class                            */
    int n;            /* rows of the contraction (0 for grouped launches)        */
    long long tiles;  /* 128 x 256 tiles of the launch                           */
    int grid;         /* chosen persistent CTAs                                  */
    int stages;       /* chosen ring stages                                      */
    float us;         /* measured microseconds per launch with the choice        */
    float us_default; /* measured microseconds per launch with the defaults      */
} tfde_tune_entry;
int tfde_tune(tfde_problem* prob, int reps, void* stream);
int tfde_batch_tune(tfde_batch* batch, int reps, void* stream);
int tfde_tune_get(tfde_tune_entry* out, int cap, int* count);
int tfde_tune_set(const tfde_tune_entry* in, int count);
int tfde_tune_clear(void);

/* ------------------------------------------------------ warm-start network */
/*
 * The learned initial guess of the CN solves (no counterpart in the paper,
 * whose solves start from the previous time level).  Four 3x3x3 convolutions
 * with zero padding, ReLU between them, 16 channels, BF16 weights and
 * activations, FP32 accumulation on the tensor cores.  Per grid point the 11
 * inputs are (u / s, dt F / s, c_1..c_9), s = max |u|, c the nine constants
 * the caller passes (the package's driver uses delta_1..3 and the logarithms of
 * the stiffness scales eta_a k+_a, eta_a k-_a, which fix the discrete operator at any
 * resolution), and the output is the predicted (u^{m+1} - u^m) / s.
 *
 * Parameters (host FP32, TFDE_CNN_PARAMS floats): for layers l = 0..3 in
 * order, W_l[co][ci][tap] (16 x 16 x 27; tap = (dz+1) 9 + (dy+1) 3 + (dx+1),
 * the weight of input point p + (dz, dy, dx) for output point p) followed by
 * b_l[co] (16).  Layer 0 reads input channels 0..10, layer 3 writes output
 * channel 0; weights of the unused channels must be zero.
 */
#define TFDE_CNN_PARAMS (4 * (16 * 16 * 27 + 16))
typedef struct tfde_cnn tfde_cnn;

/* Network with workspace for grids of n[0] x n[1] x n[2] points (any n_a >= 1);
 * parameters start at zero.  Errors: TFDE_EINVAL, TFDE_ENOMEM, TFDE_ECUDA. */
int tfde_cnn_create(const int n[3], tfde_cnn** out);
int tfde_cnn_destroy(tfde_cnn* net);
/* Upload / download parameters (layout above); set also clears the gradient
 * accumulator and the Adam moments.  Synchronous. */
int tfde_cnn_set_params(tfde_cnn* net, const float* params);
int tfde_cnn_get_params(const tfde_cnn* net, float* params);
/* Download the accumulated gradients (sum over tfde_cnn_accumulate calls since
 * the last Adam step), same layout as the parameters.  Synchronous. */
int tfde_cnn_get_grads(const tfde_cnn* net, float* grads);
/*
 * tfde_cnn_predict -- x0 = u + s * net(u / s, dtF / s, coef), the initial guess
 * of the step from u.  u, dtF (NULL for f = 0), x0: device FP64 grids of the
 * network's size (x fastest); coef: host, the 9 constants (delta_1..3,
 * k+_1..3, k-_1..3).  Synchronises `stream`.
 */
int tfde_cnn_predict(tfde_cnn* net, const double* u, const double* dtF, const double* coef, double* x0, void* stream);
/*
 * tfde_cnn_accumulate -- one training sample (u^m, dt F, coef) -> u^{m+1}:
 * forward pass, loss = mean over points of (out - (u^{m+1} - u^m) / s)^2 into
 * *loss (may be NULL), and the gradients of the loss added to the
 * accumulator.  Synchronises `stream`.
 */
int tfde_cnn_accumulate(tfde_cnn* net, const double* u, const double* dtF, const double* coef, const double* u_next,
                        double* loss, void* stream);
/*
 * tfde_cnn_predict_hist / tfde_cnn_accumulate_hist -- the same with the time
 * history u1 = u^{m-1} and u2 = u^{m-2} (device; u2 may be NULL, both NULL
 * gives the calls above): input channels 11 and 12 carry the first and
 * second differences d1 = u - u1, d2 = u - 2 u1 + u2 (divided by s), and the
 * network predicts the correction to the polynomial extrapolation in time,
 * base = 3u - 3u1 + u2 (2u - u1 with one level): x0 = base + s * net(...),
 * training target (u^{m+1} - base) / s.  Weights of channels 11, 12 are
 * ordinary layer-0 parameters.  Errors: TFDE_EINVAL for u2 without u1.
 */
int tfde_cnn_predict_hist(tfde_cnn* net, const double* u, const double* u1, const double* u2, const double* dtF,
                          const double* coef, double* x0, void* stream);
int tfde_cnn_accumulate_hist(tfde_cnn* net, const double* u, const double* u1, const double* u2, const double* dtF,
                             const double* coef, const double* u_next, double* loss, void* stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) with the accumulated gradients
 * averaged over the samples, then clears the accumulator.  lr > 0. */
int tfde_cnn_adam_step(tfde_cnn* net, float lr, void* stream);

/*
 * tfde_source_example2 -- cell averages F_{ijk} (Sec. 2, definition of F^{m-1/2})
 * of the manufactured source of Sec. 4, Example 2, on Omega = (0,1)^3:
 *   f = cP P(x)P(y)P(z) + cS [S_a(x)P(y)P(z) + P(x)S_b(y)P(z) + P(x)P(y)S_c(z)],
 *   P(x) = x^2 (1-x)^2,
 *   S_d(x) = sum_{k=0}^2 (-1)^{2-k} C(2,k) Gamma(5-k)/Gamma(3-k+d) [k_+ x^{2-k+d} + k_- (1-x)^{2-k+d}].
 *   For u = phi(t) P P P:  cP = phi'(t), cS = -phi(t).  Integrals are exact.
 *   2-D problems (Example 1): the same without the third factor,
 *   f = cP P(x)P(y) + cS [S_a(x)P(y) + P(x)S_b(y)] (u = 4 e^t P P: cP = 4e^t, cS = -4e^t).
 *   Requires lo = 0, hi = 1 on every axis (else TFDE_EINVAL).  F: device output.
 */
int tfde_source_example2(const tfde_problem* prob, double cP, double cS, double* F, void* stream);

/*
 * tfde_coefficients -- host copies of the assembled 1-D data of one axis:
 *   q (n_a + 1 doubles, Eq. (coef_expression)), tau eigenvalues (n_a doubles,
 *   Lemma 1D_tau_SPD) and eta_a.  Any output may be NULL.  Synchronous, no GPU work.
 */
int tfde_coefficients(const tfde_problem* prob, int axis, double* q, double* lam_tau, double* eta);

/*
 * tfde_host_coefficients -- the same 1-D data as tfde_coefficients computed on
 * the host from parameters alone (no problem, no GPU): q (n_a + 1), tau
 * eigenvalues (n_a), mass eigenvalues (6 + 2 cos(k pi/(n_a+1)))/8 (n_a) and
 * eta_a.  Outputs may be NULL.  TFDE_EINVAL for invalid parameters.
 */
int tfde_host_coefficients(const tfde_params* params, int axis, double* q, double* lam_tau, double* lam_mass,
                           double* eta);

/* Counters of the library's own GPU work (process-wide), per kind of
 * per-axis kernel: TFDE_KIND_SPLIT = the split-BF16 tensor-core contraction
 * (fast operator and preconditioner), TFDE_KIND_EXACT = the exact-integer
 * slice contraction (FP64-accurate operator), TFDE_KIND_CONV = the
 * warm-start network's convolution, TFDE_KIND_FFT = the FFT-embedded Toeplitz
 * and DST-I passes (bytes: the grid functions read and written once; flops:
 * 5 L log2 L per complex transform of length L plus the spectral products). */
enum { TFDE_KIND_SPLIT = 0, TFDE_KIND_EXACT = 1, TFDE_KIND_CONV = 2, TFDE_KIND_FFT = 3, TFDE_NKINDS = 4 };
typedef struct {
    unsigned long long launches;  /* launches of this kind                               */
    unsigned long long timed;     /* launches covered by ms                               */
    double ms;                    /* summed CUDA-event duration (timing enabled)          */
    double bytes;                 /* algorithmic bytes: operands read once, output written */
    double flops;                 /* tensor-core flops (2 x m x k x n per BF16 product)    */
} tfde_kernel_stats;
typedef struct {
    unsigned long long kernel_launches;  /* every kernel this library launched */
    tfde_kernel_stats kind[TFDE_NKINDS];
} tfde_stats;

/*
 * tfde_stats_reset -- zero the counters; `time_tc` != 0 additionally brackets
 * every tensor-core kernel launch with a CUDA event pair on its stream so that
 * kind[k].ms is the sum of their device durations (the inner PCG then runs its
 * host-driven loop, see tfde_set_device_loop).  Not thread-safe.
 */
int tfde_stats_reset(int time_tc);

/* tfde_stats_get -- synchronise the device and copy the counters to *out. */
int tfde_stats_get(tfde_stats* out);

/*
 * tfde_mass_apply_noalloc -- y = A_N x = (A_{n3} (x) A_{n2} (x) A_{n1}) x, the
 * tridiagonal mass operator of the CN-FV system, WITHOUT allocating memory.
 * The paper has no counterpart to this entry point: it exists for callers that
 * cannot allocate device memory when they need the operator (a solver step
 * inside a memory budget fixed at start-up, a latency-critical loop where the
 * allocator's implicit device synchronisation is not allowed, a plug-in that
 * only receives ready-made device buffers from its host).
 *   n: host array of the three grid extents, each >= 1, with
 *      n[0]*n[1]*n[2] <= 262144 (2^18, e.g. 64^3); larger grids return
 *      TFDE_EINVAL with a message naming the limit.
 *   x, y: device grid functions (x fastest), caller-owned; y may alias x.
 *   The two intermediate grid functions live in a fixed 4 MiB device array
 *   compiled into the library, which every GPU that loads the library keeps
 *   until the process exits.  All calls share that array and it keeps the
 *   previous call's contents (each call overwrites what it reads), so calls
 *   that overlap on the GPU -- on different streams or devices' contexts
 *   sharing a device -- race and give wrong results.  The first call on each
 *   device looks up the array's device address (cudaGetSymbolAddress); make
 *   that first call before any stream capture.  No cudaMalloc, cudaFree or
 *   allocating library routine is called.  Asynchronous on `stream`.
 */
int tfde_mass_apply_noalloc(const int n[3], const double* x, double* y, void* stream);

/*
 * tfde_selftest_wait -- diagnostic of the bounded device-side waits (no
 * counterpart in the paper).  Every mbarrier wait of the library's
 * tensor-core kernels gives up after a wall-clock limit (2 s), raises the
 * kernel's error flag, releases the kernel's tensor memory and returns, so
 * that a lost arrival surfaces as TFDE_ETIMEOUT instead of a hung GPU.  This
 * entry point runs that path on purpose: one CTA allocates tensor memory,
 * waits with the shared bounded-wait routine and limit_ns (1000 ..
 * 2000000000) on an mbarrier that nothing ever arrives on, releases the
 * tensor memory and exits; no copy or MMA is in flight.
 *   Returns TFDE_ETIMEOUT when the wait ran out as designed (the expected
 *   result) with *tmem_freed (may be NULL) = 1 once the kernel released its
 *   tensor memory; TFDE_EINVAL for a limit out of range; TFDE_ECUDA otherwise.
 *   The device stays usable afterwards.  Synchronises `stream`.
 */
int tfde_selftest_wait(long long limit_ns, int* tmem_freed, void* stream);

/* Thread-local description of the last failure on this thread ("" if none). */
const char* tfde_last_error(void);

/* Library version string. */
const char* tfde_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TFDE_H */
