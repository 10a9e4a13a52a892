/*
 * aao.h -- C ABI of the GB300 (sm_103a) all-at-once Crank-Nicolson solver with the
 * generalized block alpha-circulant preconditioner of arXiv 2401.16113.
 *
 * Conventions shared by every entry point
 *  - Space-time vectors are FP64, time-block-major: u[t * nx + i] holds u^{t+1} at the
 *    interior spatial node i (the ordering of the all-at-once unknown in Sec. 2.2),
 *    t = 0..nt-1, i = 0..nx-1. Their length is nx * nt (nx * nv * nt for AAO_OP_HESTON, whose
 *    time level holds nx * nv unknowns).
 *  - Pointers named *_dev are device pointers owned by the caller; the library never
 *    frees caller memory. Pointers named *_host are ordinary (pageable or pinned) host
 *    pointers.
 *  - Work is issued on the stream given in aao_problem.stream (0 = legacy default stream)
 *    and is stream-ordered; calls that report statistics synchronise that stream.
 *  - Every call returns AAO_OK (0) or a negative status; aao_last_error() returns a
 *    human-readable message for the calling thread's most recent failure.
 *  - A handle is not thread-safe: serialise calls on one handle.
 */
#ifndef AAO_H
#define AAO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define AAO_OK 0
#define AAO_EINVAL (-1)        /* invalid argument or unsupported size            */
#define AAO_ECUDA (-2)         /* a CUDA runtime call failed                      */
#define AAO_ENOMEM (-3)        /* device allocation failed                        */
#define AAO_NOT_CONVERGED (-4) /* FGMRES hit maxit before reaching tol            */
#define AAO_BREAKDOWN (-5)     /* non-finite value or Arnoldi breakdown w/o convergence */
#define AAO_TIMEOUT (-6)       /* a bounded device-side wait gave up              */
#define AAO_EUNSUPPORTED (-7)  /* operator / size combination not built           */

/* spatial operator A (Eq. 1.2, discretised by finite differences) */
#define AAO_OP_BS 0       /* Black-Scholes in S, constant sigma, 3-point central FD      */
#define AAO_OP_LOCALVOL 1 /* Black-Scholes with sigma(S,t) = sigma + lv_bump *
                             exp(-ln(S/K)^2) * (1 + lv_tslope * t); row k of the AaO system
                             uses A(t_{k+1/2}) (the time-dependent form of Eq. 5.8), the
                             preconditioner the time mean of those matrices (Sec. 5.3)      */
#define AAO_OP_RIESZ 2    /* Riesz fractional operator (beta, Eq. 1.2 second case) in
                             log-price x in [-s_max, s_max] with drift (r - sigma^2/2) u_x;
                             step (b) by the explicit inverses of the shifted matrices (made at
                             create from their LU factors; one dense product per bin and
                             apply, nt/2+1 x nx^2 complex64 resident), or, when the drift vanishes
                             (r = sigma^2/2, a symmetric operator), by the eigendecomposition
                             tau Abar = Q diag(lambda) Q^T: two products with Q per apply   */

#define AAO_OP_HESTON 3   /* the two-dimensional Heston operator of Sec. 5.1 (Eq. 5.1) in (s, v) on a
                             uniform grid: s_i = i s_max / nx, i = 1..nx (s = s_max carries the
                             Neumann condition u_s = 1 through a ghost node), v_j = j v_max / nv,
                             j = 0..nv-1 (v = 0 carries the boundary equation u_t = kappa eta u_v +
                             r s u_s - r u with a one-sided second-order u_v; v = v_max the Dirichlet
                             value u = s), u(0, v) = 0; central differences, the mixed derivative by
                             the four-point cross stencil; call payoff only. Unknown (i, j) of a
                             time level at j nx + i - 1. Step (b) by block elimination over the v
                             levels with dense inverses of the diagonal blocks made at create
                             (precision AAO_MIXED only) */
#define AAO_OP_SABR 4     /* the two-dimensional SABR operator of Sec. 5.2 (Eq. 5.7):
                             u_t = 1/2 v^2 s^(2 beta) D^(2(1-beta)) u_ss + rho sigma s^beta D^(1-beta)
                             v^2 u_sv + 1/2 sigma^2 v^2 u_vv + r s u_s - r u, D(t) = e^{-rt}, on the
                             grid, boundary conditions, unknown order and step (b) of AAO_OP_HESTON;
                             at v = 0 the boundary equation u_t = r s u_s - r u (u_t = 0 for r = 0;
                             kappa and eta unused). For r != 0 row k of the AaO system uses A at
                             t_{k+1/2} (Eq. 5.8) and step (b) the time mean of those matrices */

#define AAO_PUT 0
#define AAO_CALL 1

#define AAO_FP64 0  /* preconditioner apply in FP64 complex                           */
#define AAO_MIXED 1 /* preconditioner apply in FP32 complex inside FP64 FGMRES        */

/*
 * Problem descriptor (plain old data; copied by aao_create).
 *  nx, nt      interior spatial nodes (2..8192) and CN steps (1..8192; prime factors 2, 3, 5,
 *              7 only: a power of two takes the register FFT, any other nt the mixed-radix
 *              shared-memory FFT, up to 4096 in FP64)
 *  op, payoff  AAO_OP_*, AAO_PUT / AAO_CALL
 *  precision   AAO_FP64 or AAO_MIXED
 *  T, r, K, sigma   maturity, rate, strike, volatility
 *  s_max       S-domain [0, s_max]; the grid is S_i = i h, h = s_max / (nx + 1), i = 1..nx,
 *              with Dirichlet values V(0,t) = K e^{-rt} (put) or 0, V(s_max,t) = 0 (put)
 *              or s_max - K e^{-rt} (call), t = time to maturity
 *  alpha       the free parameter of P_alpha (Eq. 3.1), 0 < alpha < 1 (alpha = 1 allowed:
 *              the classical block-circulant preconditioner P_1)
 *  flags       0, or one AAO_FLAG_STEPB_* to fix how the tridiagonal step (b) is solved (by
 *              default, AAO_MIXED with nt a power of two: the recomputing method where one bin
 *              fits in shared memory; otherwise the factored method where one bin's staged tables
 *              fit; each falls back to the other; both give P_alpha^{-1} v up to rounding)
 *  stream      cudaStream_t on which all work is issued
 *  nv, kappa, eta, rho, v_max
 *              AAO_OP_HESTON and AAO_OP_SABR: nodes in v (3..512; nx 3..512 nodes in s), mean
 *              reversion and long-run variance (Heston only), correlation of the two Brownian
 *              motions, v-domain [0, v_max]; sigma is then the volatility of the variance
 *              (Heston) or of the volatility (SABR), and beta the SABR exponent of s (0..1).
 *              A time level holds nx * nv unknowns.
 */
#define AAO_FLAG_STEPB_FACTORED 1  /* partition method with per-bin pivot tables made at create */
#define AAO_FLAG_STEPB_RECOMPUTE 2 /* partition method, pivots recomputed in every apply      */
typedef struct aao_problem {
  int32_t nx, nt, op, payoff, precision, flags;
  double T, r, K, sigma, s_max, lv_bump, lv_tslope, beta, alpha;
  void* stream;
  int32_t nv, reserved;
  double kappa, eta, rho, v_max;
} aao_problem;

/* FGMRES outcome. iterations counts inner Arnoldi steps (= preconditioned matrix-vector
   products, the "Its" of Sec. 5); rel_residual is the true ||b - M x||_2 / ||b||_2 at exit,
   computed in FP64; ms is wall time of the call including setup of the first cycle. */
typedef struct aao_stats {
  int32_t status, iterations, restarts, launches;
  double rel_residual, est_residual, ms;
} aao_stats;

typedef struct aao_handle aao_handle;

/* Validate *p, build the operator coefficients, the eigenvalues lambda_{1,k}, lambda_{2,k}
   (Sec. 3.1, Eq. eigCx), Lambda_alpha, the FFT twiddles and the preconditioner workspace
   on the device. Ownership: *h owns all of it until aao_destroy. Errors: AAO_EINVAL for
   bad sizes or parameters, AAO_EUNSUPPORTED for nt with a prime factor above 7 or a size
   the operator's step (b) does not support, AAO_ENOMEM / AAO_ECUDA from the device, AAO_BREAKDOWN if the
   eigendecomposition of a symmetric Riesz operator does not converge. On error *h is set to
   NULL. */
int aao_create(const aao_problem* p, aao_handle** h);

/* Free every device buffer of h (NULL is accepted). */
int aao_destroy(aao_handle* h);

/* b_dev <- b = xi + tau f of Eq. 2.2: xi = [(I + A~_0/2) u^0; 0; ...], u^0 = payoff, f the
   Dirichlet data averaged over t_k and t_{k+1}. b_dev: nx*nt doubles, device. */
int aao_rhs(aao_handle* h, double* b_dev);

/* y_dev <- M x_dev with M = B1 (x) I - B2 (x) A~ (Eq. 2.2; the Eq. 5.8 form, A at t_{k+1/2} in block
   row k, for AAO_OP_LOCALVOL and for AAO_OP_SABR with r != 0).
   x_dev, y_dev: nx*nt doubles (nx*nv*nt for the two-dimensional operators), device, must not
   alias. */
int aao_matvec(aao_handle* h, const double* x_dev, double* y_dev);

/* z_dev <- P_alpha^{-1} v_dev by the three steps of Eq. 3.2 with the conjugate-pair saving
   of Remark 1: Lambda_alpha scaling and a real-to-complex FFT along t (mixed radix when nt is
   not a power of two), floor(nt/2)+1 complex-shifted spatial solves
   (lambda_{1,k} I - lambda_{2,k} A~) z_k = z1_k (tridiagonal; dense for AAO_OP_RIESZ), then
   the inverse FFT and Lambda_alpha^{-1}. FP32 complex inside when precision = AAO_MIXED (z is
   still returned in FP64). v_dev, z_dev: nx*nt doubles, device; may alias. Returns AAO_OK, or
   AAO_TIMEOUT when a tensor-core product of the symmetric Riesz operator's step (b) gave up a
   bounded wait (z is then not valid; for that operator this call synchronises the stream to
   read the error word), or an error. */
int precond_apply(aao_handle* h, const double* v_dev, double* z_dev);

/* Solve M x = b (Eq. 2.2) by right-preconditioned flexible GMRES(m) with P_alpha
   (Sec. 5: right preconditioning, relative-residual stop). x_dev holds the initial guess on
   entry (zero it for the paper's protocol) and the solution on exit. Orthogonalisation is
   classical Gram-Schmidt with a second pass when the first cancels more than 1 - 1e-5 of
   the vector's norm, the least-squares update uses Givens rotations, all in FP64; the true
   residual is recomputed at every restart. 1 <= m <= 64,
   maxit >= 1 bounds the total inner iterations. st may be NULL. Returns AAO_OK,
   AAO_NOT_CONVERGED, AAO_BREAKDOWN, AAO_TIMEOUT (a tensor-core product of the symmetric Riesz
   operator's step (b) gave up a bounded wait and skipped its output) or an error. */
int fgmres_solve(aao_handle* h, const double* b_dev, double* x_dev, double tol, int m, int maxit,
                 aao_stats* st);

/* As fgmres_solve from the zero initial guess of the paper's protocol: x_dev is output only (its
   contents on entry are ignored), and the first residual r_0 = b is formed by one copy of b
   (with the FP32 copy that a mixed-precision preconditioner reads and ||b||) instead of the
   matrix-vector product b - M x_0. Same arguments, results and errors as fgmres_solve. */
int fgmres_solve_zero(aao_handle* h, const double* b_dev, double* x_dev, double tol, int m, int maxit,
                      aao_stats* st);

/* As fgmres_solve_zero with host buffers: copies b_host to the device, solves from a zero
   initial guess, copies the solution to x_host. Both are nx*nt doubles, owned by the caller
   (pinned host memory gives the fastest copies). The handle keeps its two device copies of them
   from the first call until aao_destroy (16 * nx*nt bytes). */
int fgmres_solve_host(aao_handle* h, const double* b_host, double* x_host, double tol, int m,
                      int maxit, aao_stats* st);

/* z_dev <- P_alpha^{-1} v_dev, the same computation as precond_apply, for callers that cannot
   allocate device memory (the paper has no counterpart: this is a deployment variant).
   Processes that run under a fixed device-memory budget handed out up front, or latency-critical
   paths that cannot afford an allocation's implicit synchronisation or its failure, cannot call
   aao_create, which allocates its tables and workspace. This entry point takes the problem
   descriptor directly and keeps every table and the half spectrum in one static device array of
   32 MiB (reserved on each GPU that loads the library until the process exits); it calls no
   cudaMalloc or cudaFree.
    - Operators: AAO_OP_BS and AAO_OP_LOCALVOL. AAO_OP_RIESZ, AAO_OP_HESTON and AAO_OP_SABR return
      AAO_EUNSUPPORTED: their step (b) needs the dense inverses, the eigendecomposition or the
      block factors that aao_create builds.
    - Size limit: the half spectrum plus tables must fit in 32 MiB, roughly
      (nt/2+1) * 64*ceil(nx/64) * 8 bytes (mixed) or * 16 bytes (FP64) plus O(nt + nx);
      e.g. nx 2047, nt 2048 fits in mixed precision. Larger problems return AAO_EINVAL
      with a message; use precond_apply for them.
    - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
      with that device current and keeps it for the life of the process (do not reset the device
      between calls); make that first call before any stream capture.
    - All calls on a device share the array. Each call rewrites everything it reads, so no
      clearing is needed, but calls whose work overlaps on the GPU race on it: order them
      (one stream, or events).
   Arguments and errors as for precond_apply; p->stream selects the stream. */
int precond_apply_static(const aao_problem* p, const double* v_dev, double* z_dev);

/* ---- Batched solves (many independent instances in one persistent launch) ----
   A batch holds n problems (each with its own nx, nt, coefficients, alpha) solved by
   right-preconditioned FGMRES(m) exactly as fgmres_solve does with precision AAO_MIXED.
   One CTA owns one instance at a time and runs its whole solve (preconditioner, matvec,
   Gram-Schmidt, Givens, convergence test) with no host round trip; instances are taken from
   a queue, largest first, so uneven sizes balance across the GPU. Each instance has its own
   status. The work of one instance does not depend on the others: its result is the same
   whatever else is in the batch. */
typedef struct aao_batch aao_batch;

/* Build tables and workspace for n problems (all precision AAO_MIXED, op AAO_OP_BS or
   AAO_OP_LOCALVOL, 2 <= nt <= 4096 with prime factors 2, 3, 5 and 7 only (a power of two takes
   the register FFT tile, any other nt the mixed-radix one), 2 <= nx <= 4096) with restart length
   1 <= m <= 40. The FFT column tile of each nt class is autotuned here. Work is ordered after
   ps[0].stream. Errors: AAO_EINVAL (names the first bad problem), AAO_ENOMEM, AAO_ECUDA. */
int aao_batch_create(const aao_problem* ps, int n, int m, aao_batch** bt);

/* b_dev[i] <- the right-hand side of instance i (as aao_rhs). b_dev: n device pointers to
   nx_i*nt_i doubles. */
int aao_batch_rhs(aao_batch* bt, double* const* b_dev);

/* Solve instance i: M_i x_dev[i] = b_dev[i] from the initial guess in x_dev[i], to relative
   residual tol, at most maxit inner iterations each. One persistent kernel launch, replayed
   from a CUDA graph captured on the first call (re-captured if tol or maxit change).
   Blocks until done. st (may be NULL) receives n records; ms is the wall time of the call.
   Returns AAO_OK if every instance converged, else the first failing instance's status. */
int batch_submit(aao_batch* bt, double* const* b_dev, double* const* x_dev, double tol, int maxit,
                 aao_stats* st);

/* Replace the alpha of every instance (alpha[i], 0 < alpha <= 1) and rebuild the tables that
   depend on it (Lambda_alpha, lambda_{1,k}, lambda_{2,k}); used to sweep alpha. */
int aao_batch_set_alpha(aao_batch* bt, const double* alpha);

/* Free the batch (NULL accepted). */
int aao_batch_destroy(aao_batch* bt);

/* ---- The alpha/m predictor (a learned choice of the free parameter alpha of Sec. 3.1) ----
   The paper leaves alpha to the user (alpha = 0.1 or 0.01 "suffices", too small an alpha
   amplifies roundoff in steps (a) and (c), end of Sec. 4). This small network maps problem
   features to the alpha and restart length m that minimised the mixed-precision solver's
   iteration count on synthetic instances; the caller falls back to alpha = 1e-3 whenever a
   prediction does not converge. MLP 6 -> 64 -> 64 -> 2 with ReLU, FP32 parameters (4738:
   W1[64][6], b1[64], W2[64][64], b2[64], W3[2][64], b3[2], row-major), trained by the
   library's CUDA kernels (forward/backward, Adam), queried in BF16.
   Normalised features: x_i = (f_i - mean_i) / scale_i with f = (sigma, r, T, log2 nx,
   log2 nt, cv) (cv = relative variation of the time-dependent operator, 0 for constant
   coefficients); normalised targets y = ((log10 alpha - ym_0)/ys_0, (m - ym_1)/ys_1); the
   constants come from aao_mlp_normalization. Loss: mean over samples of 1/2 ||y - target||^2. */
typedef struct aao_mlp aao_mlp;

/* Create with the 4738 initial parameters (host, FP32); work runs on `stream`. */
int aao_mlp_create(const float* init_params, void* stream, aao_mlp** out);
int aao_mlp_destroy(aao_mlp* h);
/* Copy the current parameters to host (4738 floats). */
int aao_mlp_params(aao_mlp* h, float* params_host);
/* Loss and its gradient over B samples: X_dev B x 6, Y_dev B x 2 (normalised, FP32, device,
   row-major); grad_host 4738 floats, loss_host 1 float. Deterministic (fixed-order sums). */
int aao_mlp_grad(aao_mlp* h, const float* X_dev, const float* Y_dev, int B, float* grad_host, float* loss_host);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with gradient grad_dev (4738
   floats, device). */
int aao_mlp_adam_step(aao_mlp* h, const float* grad_dev, float lr);
/* Train: `epochs` passes over the B samples in minibatches, order shuffled per epoch by a
   seeded 64-bit LCG; loss_host (may be NULL) receives the final full-batch loss. */
int aao_mlp_train(aao_mlp* h, const float* X_dev, const float* Y_dev, int B, int epochs, int minibatch, float lr,
                  unsigned long long seed, float* loss_host);
/* Forward pass of B samples (normalised X_dev B x 6 -> Y_dev B x 2, device); bf16 != 0 rounds
   weights and activations to bfloat16 (FP32 accumulation). */
int aao_mlp_forward(aao_mlp* h, const float* X_dev, float* Y_dev, int B, int bf16);
/* The normalisation constants: feat_mean[6], feat_scale[6], y_mean[2], y_scale[2]. */
int aao_mlp_normalization(double* feat_mean, double* feat_scale, double* y_mean, double* y_scale);
/* Predict (alpha, m) for raw features feats = (sigma, r, T, nx, nt, cv) with the BF16 forward;
   alpha is clamped to [1e-5, 0.1] and m rounded up to the next of {5, 10, 20, 30, 40}. */
int alpha_mlp_predict(aao_mlp* h, const float feats[6], double* alpha, int* m);

/* Fault injection for tests of the failure path (the paper has no counterpart). With mask bit
   AAO_INJECT_TC_NO_LOAD set, the tensor-core products of the symmetric Riesz operator's spectral
   step (b) issue no operator load, so the first bounded wait for an operator tile runs out with
   nothing in flight: the products skip their output and precond_apply / fgmres_solve on h return
   AAO_TIMEOUT. wait_ms > 0 replaces the 2 s bound of those waits (so that a test ends quickly);
   mask 0 with wait_ms <= 0 restores normal operation. No GPU fault is raised: the kernels return
   and the context stays usable. Errors: AAO_EINVAL for a NULL handle or an unknown bit. */
#define AAO_INJECT_TC_NO_LOAD 1
int aao_fault_inject(aao_handle* h, int mask, double wait_ms);

/* Dense symmetric eigendecomposition on the host, FP64: A = Q diag(w) Q^T. A_host (n*n doubles,
   row-major, symmetric; only its values are used, the upper and lower triangles must agree) is
   overwritten with Q^T (row j = the unit eigenvector of w[j]); w_host receives the n eigenvalues
   (unsorted). Householder tridiagonalisation, then the symmetric QR iteration with the Wilkinson
   shift (Golub and Van Loan, Matrix Computations, Sec. 8.3). This is the
   setup of the spectral step (b) for a symmetric spatial operator (AAO_OP_RIESZ with
   r = sigma^2/2), exported for tests and for callers with their own symmetric operator. Needs no
   GPU. Errors: AAO_EINVAL (n < 1 or a NULL pointer), AAO_BREAKDOWN (the QR iteration did not
   converge within 64 steps per eigenvalue found). */
int aao_sym_eig(int n, double* A_host, double* w_host);

/* Bounds-checked build (diagnostics; the paper has no counterpart). A library compiled with
   -DAAO_CHECK (libaao_check.so) tests the index of every guarded global store in the
   preconditioner, solver, Riesz and Heston kernels; a failed test skips the store (no fault) and
   marks its source file. This call synchronises the device and returns how many source files saw a
   failed test since the last call (0 in the normal build, whose tests compile away). */
unsigned int aao_check_failures(void);

/* Message of the calling thread's most recent failure ("" if none). */
const char* aao_last_error(void);

/* Number of kernels this library has launched in this process (monotone counter). */
uint64_t aao_launch_count(void);

/* Kernel classes for per-kernel device timing (diagnostics; no counterpart in the paper). */
#define AAO_K_FFT_FWD 0  /* step (a) of Eq. 3.2: scaling + forward FFT along t    */
#define AAO_K_TRIDIAG 1  /* step (b): shifted tridiagonal solves                  */
#define AAO_K_FFT_INV 2  /* step (c): inverse FFT along t + unscaling             */
#define AAO_K_MATVEC 3   /* y = M x and r = b - M x                               */
#define AAO_K_ARNOLDI 4  /* Gram-Schmidt projections, updates, normalisation      */
#define AAO_K_OTHER 5    /* reductions, Givens, least squares, solution update    */
#define AAO_K_COUNT 6

/* Time the kernel classes whose bit (1 << AAO_K_*) is set in mask with CUDA events recorded
   on the launching stream around each launch, and clear what was accumulated; mask 0 turns
   timing off (the default). */
int aao_profile_enable(int mask);

/* For kernel class cls since the last aao_profile_enable: launches timed, their total device
   milliseconds, the algorithmic bytes they move (what each launch must read and write once,
   by its arguments' sizes) and their algorithmic FP64 flops (an FMA counts 2). Synchronises
   the recorded events. */
int aao_profile_read(int cls, int64_t* launches, double* total_ms, double* bytes, double* fp64_flops);

#ifdef __cplusplus
}
#endif

#endif /* AAO_H */
