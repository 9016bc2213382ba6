/*
 * efgp.h - C ABI of the GB300 library for equispaced-Fourier Gaussian-process
 * regression (EFGP): the posterior mean of a GP with a translation-invariant
 * kernel from N noisy observations in [0,1]^d, d = 1, 2 or 3.
 *
 * The method (Sec. 3.2, Algorithm "GP posterior mean using equispaced Fourier
 * representation"): approximate the kernel by M = (2m+1)^d complex
 * exponentials on an equispaced frequency grid of spacing h (eq. 110), solve
 * the weight-space system (Phi^* Phi + sigma^2 I) beta = Phi^* y (eq. be) by
 * conjugate gradients with an FFT Toeplitz matrix-vector product (Algorithm
 * "Fast product of Toeplitz matrix F^*F with a vector", eq. 97), and evaluate
 * mu(z) = sum_j beta_j phi_j(z) (eq. muws) at targets with a type-2
 * nonuniform FFT.  All steps after input validation run as CUDA kernels on
 * the calling process's current device; there is no CPU fallback.
 *
 * Conventions used by every entry point:
 *  - Status: every function returns an efgp_status (0 = success).
 *  - Points x are N x d, row-major (point n at x[n*d .. n*d+d-1]) unless
 *    efgp_options.x_layout says structure-of-arrays (axis a at x[a*N ..]).
 *    Targets use the same layout flag.
 *  - Pointers are device pointers on the current device unless
 *    efgp_options.host_io is 1, in which case x, y, targets and mu_out are
 *    host pointers (pinned memory is fastest) and the library copies them.
 *  - The library never frees or retains caller memory: it copies what it
 *    needs into its own workspace.  Caller buffers may be reused once the
 *    call has returned (all calls synchronise the handle's stream before
 *    returning, except efgp_apply_system_device, which only orders its work
 *    on that stream).
 *  - Frequency multi-indices j in {-m..m}^d are stored row-major with the
 *    first coordinate slowest: j sits at flat index sum_l (j_l+m)(2m+1)^(d-1-l).
 *    Complex vectors are interleaved (re, im) float64 pairs.
 *  - Sign convention: F_{nj} = exp(+2 pi i h j.x_n); the Toeplitz entries are
 *    w_k = sum_n exp(-2 pi i h k.x_n) (the conjugate of the printed eq. 88).
 */
#ifndef EFGP_H
#define EFGP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EFGP_OK = 0,
  EFGP_EINVAL = 1,    /* bad argument (NULL pointer, d outside 1..3, sigma <= 0, ...) */
  EFGP_ERANGE = 2,    /* a point or target outside [0,1]^d, or a NaN/Inf coordinate  */
  EFGP_ENOMEM = 3,    /* a device or host allocation failed                           */
  EFGP_ENOTCONV = 4,  /* CG hit max_iter before the residual target; beta still valid */
  EFGP_ETIMEOUT = 5,  /* a bounded device-side wait ran out                            */
  EFGP_ECUDA = 6,     /* a CUDA runtime call failed (message: efgp_last_error())       */
  EFGP_ESTATE = 7,    /* call out of order (e.g. predict before solve)                 */
  EFGP_EUNSUPPORTED = 8 /* a size or option the library does not support                */
} efgp_status;

typedef enum { EFGP_KERNEL_SE = 0, EFGP_KERNEL_MATERN = 1 } efgp_kernel_family;
/* EFGP_MIXED: FP32 spreading, fine-grid and Toeplitz FFTs, FP64 CG vectors and
 * scalars; EFGP_FP64: everything FP64; EFGP_MIXED_CG64: FP32 spreading (FP32
 * records and tiles, FP64 flush), FP64 fine grid, Toeplitz FFTs, CG and type-2
 * (for systems whose FP32
 * Toeplitz product error, ~1e-7 N max D^2, would exceed sigma^2); the type-1
 * fine grid and its FFT are FP64 there too, for the same reason. */
typedef enum { EFGP_MIXED = 0, EFGP_FP64 = 1, EFGP_MIXED_CG64 = 2 } efgp_precision;
typedef enum { EFGP_F32 = 0, EFGP_F64 = 1 } efgp_dtype;

/* Covariance kernel (eqs. Gker and Cker), scaled by `variance` (k(0)). */
typedef struct {
  int family;          /* efgp_kernel_family                                  */
  double nu;           /* Matern smoothness (> 0); ignored for SE              */
  double lengthscale;  /* ell > 0                                              */
  double variance;     /* k(0) > 0; 0 is read as 1                              */
} efgp_kernel;

/* Options.  Zero-initialise (or call efgp_default_options) and set fields. */
typedef struct {
  int precision;        /* efgp_precision                                                   */
  int coord_dtype;      /* dtype of x and targets (efgp_dtype)                            */
  int value_dtype;      /* dtype of y and mu_out (efgp_dtype)                              */
  int x_layout;         /* 0: row-major N x d; 1: structure of arrays d x N               */
  int host_io;          /* 0: device pointers; 1: host pointers, copied by the library    */
  double cg_tol;        /* relative residual rho (0: the default of efgp_solve; the       */
                        /* Algorithm's step 4 uses rho ~ eps)                              */
  int64_t max_iter;     /* CG iteration cap (0: 100000)                                   */
  double nufft_tol;     /* NUFFT accuracy (0: eps/10, Sec. 5.1)                           */
  int m_override;       /* > 0: use this m instead of the Sec. 4.2 choice                 */
  double h_override;    /* > 0: use this h instead of the Sec. 4.2 choice                 */
  int fft_len_override; /* > 0: Toeplitz FFT length L per dim (>= 4m+1, 2,3,5,7-smooth)   */
  double upsampfac;     /* > 0: NUFFT fine-grid upsampling factor (else chosen)           */
  int es_width;         /* > 0: ES kernel width in grid points (else chosen)              */
  int iters_per_launch; /* CG iterations per captured CUDA graph launch (0: 32)           */
  int autotune;         /* 1: before the first solve, time each line pass of the Toeplitz  */
                        /* product at a few line batches, thread counts and orders of its */
                        /* Stockham radices (once per pass shape and precision in the     */
                        /* process) and keep the fastest, for every CG form              */
  int profile;          /* 1: time each phase with CUDA events (efgp_get_phase_times)     */
  int cg_mode;          /* 0: choose (one problem: 1; a batch: 3);                      */
                        /* 1: graph-captured kernels per iteration;                        */
                        /* 2: one persistent launch, a thread-block cluster per problem     */
                        /*    (small problems);                                            */
                        /* 3: one launch whose blocks claim work items (FFT line batches,   */
                        /*    vector chunks) of any problem's current CG phase;            */
                        /* 4: one cooperative launch over the whole GPU, grid barriers      */
                        /*    between the passes (bounded waits: ETIMEOUT)                 */
  void* stream;         /* cudaStream_t to order work on (NULL: a private stream)         */
  int setup_path;       /* set-up kernels: 0 or 1: three passes (tile count, sorting     */
                        /* scatter, spread; fastest); 2: fused chunked sort-and-spread,  */
                        /* bitwise reproducible, compensated FP64 tile sums (2D, FP32 x */
                        /* and y, row-major, 16-byte aligned, mixed precision; other    */
                        /* problems take the three passes)                              */
  int precond;          /* 1: Jacobi-preconditioned CG, M = diag(A) = D_j^2 w_0 + sigma^2  */
                        /* (Sec. 6 leaves preconditioning open); the stopping rule stays  */
                        /* ||r|| <= rho ||b|| with a default rho ten times smaller (a     */
                        /* preconditioned iterate's mean error at a given residual is     */
                        /* larger; see efgp_solve).  Graph-captured and scheduled CG    */
                        /* (cg_mode 0, 1 or 3; cg_mode 2 or 4 gives EUNSUPPORTED)         */
} efgp_options;

/* Discretisation and NUFFT parameters chosen for a problem. */
typedef struct {
  int d;
  double h;             /* frequency grid spacing (Sec. 4.2)                    */
  int m;                /* half-width: J_m = {-m..m}^d                           */
  int64_t M;            /* (2m+1)^d unknowns                                     */
  int L;                /* Toeplitz FFT length per dim (>= 4m+1)                 */
  int nf1, w1;          /* type-1 fine grid per dim and ES width                 */
  double beta1, upsamp1;
  int nf2, w2;          /* type-2 fine grid per dim and ES width                 */
  double beta2, upsamp2;
  int poly_deg1, poly_deg2; /* degree of the piecewise polynomial ES evaluation  */
  double es_err1, es_err2;  /* estimated relative NUFFT error (sup norm)        */
  int tile;             /* spread tile edge (fine-grid cells)                    */
  double kernel_l2norm; /* ||k||_{L2[-1,1]^d} (Matern heuristic; 0 for SE)      */
} efgp_params;

typedef struct {
  int64_t iters;        /* CG iterations taken                                   */
  double rel_residual;  /* ||r||/||b|| of the recursively updated residual        */
  double true_rel_residual; /* ||b - A beta||/||b|| recomputed at exit             */
  int converged;        /* 1 if rel_residual <= rho                              */
  double solve_ms;      /* device time of the CG loop                            */
} efgp_solve_info;

/* Per-phase device times accumulated over all calls on a handle (filled when
 * efgp_options.profile = 1; launch counts are always kept). */
typedef struct {
  double bin_count_ms;   /* tile histogram of the points                         */
  double bin_scatter_ms; /* bin sort scatter                                      */
  double spread_ms;      /* type-1 spreading (shared-memory tiles, FP64 flush)   */
  double fine_fft_ms;    /* fold, fine-grid FFT, deconvolution and split          */
  double what_ms;        /* FFT of the Toeplitz generating vector                 */
  double cg_ms;          /* CG iterations                                         */
  double predict_fft_ms; /* type-2 precorrection, inverse FFT, unfold             */
  double interp_ms;      /* type-2 interpolation at the targets                   */
  int64_t n_setup, n_solve, n_predict;  /* calls timed                           */
  int64_t launches;      /* kernels this handle has launched (graph nodes count)  */
  int64_t cg_iters;      /* CG iterations run                                     */
  int64_t setups_fused;  /* set-ups that took the fused chunked kernels (the rest */
                         /* took the three passes; see efgp_options.setup_path)   */
} efgp_phase_times;

typedef struct efgp_handle efgp_handle;

/* Fill *opt with defaults (mixed precision, FP32 inputs, device pointers). */
int efgp_default_options(efgp_options* opt);

/* Text for a status code; static storage, never NULL. */
const char* efgp_status_string(int status);

/* Message of the last error on this thread (CUDA error text etc.). */
const char* efgp_last_error(void);

/* Host-only: the (h, m) of Sec. 4.2 and the NUFFT/FFT sizes for a problem of
 * dimension d with N points, without touching a GPU.  Needs no device. */
int efgp_plan(int d, int64_t N, const efgp_kernel* kern, double sigma, double eps,
              const efgp_options* opt, efgp_params* out);

/* Steps 1-3 of the Algorithm: choose (h, m), bin-sort the points, spread them
 * with a type-1 NUFFT to get the Toeplitz vector w (eq. 88) and Phi^* y
 * (eq. rhs), and take the FFT of w.  x: N x d coordinates in [0,1]^d; y: N
 * values.  On success *out owns all device workspace (free with
 * efgp_destroy).  N may be 0 (the mean is then 0).  Errors: EINVAL, ERANGE
 * (a coordinate outside [0,1] or not finite), ENOMEM, ECUDA. */
int efgp_setup(const void* x, const void* y, int64_t N, int d, const efgp_kernel* kern,
               double sigma, double eps, const efgp_options* opt, efgp_handle** out);

/* Step 4: conjugate gradients on (D F^*F D + sigma^2 I) beta = D F^* y
 * (eqs. 97, be) from beta = 0, stopping at ||r||/||b|| <= rho or max_iter.
 * The default rho is eps/10 * min(1, sqrt(1e7 / kappa)) with
 * kappa = 1 + N D_0^2 / sigma^2 (D_0^2 = h^d khat(0)), divided by a further 10
 * with the Jacobi preconditioner: one or more digits below the paper's
 * rho ~ eps, so that the posterior mean stays within 10 eps max|y| of the
 * exact solution of the same discretised system (measured at N = 1e9: with
 * rho = eps that error reaches 15-25 eps max|y| at kappa ~ 4e7, and rho =
 * eps/10 leaves 44 eps max|y| at kappa ~ 2e9).  info may be NULL.  Returns
 * ENOTCONV if max_iter was reached (beta is then the last iterate and
 * predict still works). */
int efgp_solve(efgp_handle* h, efgp_solve_info* info);

/* Step 6: mu(z_i) = sum_j D_j beta_j exp(2 pi i h j.z_i) for q targets in
 * [0,1]^d by a type-2 NUFFT.  mu_out: q values of value_dtype.  Errors:
 * ESTATE before a solve, ERANGE for a target outside [0,1]^d. */
int efgp_predict(efgp_handle* h, const void* targets, int64_t q, void* mu_out);

/* Allocation-free form of efgp_predict, for callers that cannot allocate
 * device memory when they predict: real-time serving loops that must not
 * block in an allocator, and host applications that reserve all device memory
 * up front and forbid plug-ins from allocating.  The paper has no
 * counterpart: it is an interface convenience.  Arguments and results are
 * those of efgp_predict, with device pointers only (a handle set up with
 * host_io = 1 gives EFGP_EINVAL).  The two type-2 scratch grids live in one
 * fixed 16 MiB device array inside the library instead of handle memory; a
 * problem whose grids need more (fine grid nf2^d complex plus extended grid
 * nE2^d real, see efgp_get_params) gives EFGP_EUNSUPPORTED with the sizes in
 * efgp_last_error().  The first call on each device looks up the array's
 * device address (once per device, with that device current).  Like
 * efgp_predict, the call ends by copying the target range flag to the host
 * and synchronising the handle's stream, so it returns only when mu_out is
 * written.  All calls share the one array, which keeps the previous call's
 * contents (the part that must start at zero is cleared by every call), so
 * calls whose work overlaps on the GPU (different streams or threads) race:
 * order them.  No cudaMalloc, cudaFree or other allocating call is made. */
int efgp_predict_noalloc(efgp_handle* h, const void* targets, int64_t q, void* mu_out);

/* Release everything the handle owns.  NULL is ignored. */
void efgp_destroy(efgp_handle* h);

/* Parameters of a set-up problem. */
int efgp_get_params(const efgp_handle* h, efgp_params* out);

/* Accumulated phase times and launch counts of a handle. */
int efgp_get_phase_times(const efgp_handle* h, efgp_phase_times* out);

/* Copy beta (M complex float64, interleaved) to host memory. */
int efgp_get_beta(const efgp_handle* h, double* beta_host);

/* Replace beta by caller-supplied weights (M complex float64, host memory,
 * same order as efgp_get_beta); efgp_predict then evaluates
 * f(z) = Re sum_j D_j beta_j exp(2 pi i h j.z).  With beta iid standard
 * complex normal and beta_{-j} = conj(beta_j) this draws a sample of the GP
 * prior with covariance ktilde (eq. 110), as suggested in Sec. 6; the random
 * numbers are the caller's.  Marks the handle solved.  N may be 0 at set-up. */
int efgp_set_beta(efgp_handle* h, const double* beta_host);

/* Copy the Toeplitz vector w ((4m+1)^d complex) and/or the right-hand side
 * b = D F^* y (M complex) to host memory; either pointer may be NULL. */
int efgp_get_system(const efgp_handle* h, double* w_host, double* b_host);

/* Apply the system matrix once: out = (D F^*F D + sigma^2 I) in, both M
 * complex float64 in host memory (a test accessor for the Toeplitz matvec). */
int efgp_apply_system(efgp_handle* h, const double* in_host, double* out_host);

/* The same product on device arrays (M complex float64 each, interleaved),
 * enqueued on the handle's stream without synchronising (for timing the
 * Toeplitz matvec, Algorithm 1 steps 3-6, in place).  in and out must not
 * overlap; the handle's FFT scratch is used, so calls on one handle must not
 * run concurrently with its solve. */
int efgp_apply_system_device(efgp_handle* h, const void* in_dev, void* out_dev);

/* ---- batched problems: one CG launch sequence for many problems ---------- */

typedef struct {
  const void* x;        /* N x d coordinates (layout/dtype from the options)   */
  const void* y;        /* N values                                            */
  int64_t N;
  int d;
  efgp_kernel kern;
  double sigma;
  double eps;
} efgp_problem;

typedef struct efgp_batch efgp_batch;

/* Set up nprob independent problems (steps 1-3 of the Algorithm for each).
 * The options apply to all problems.  On failure nothing is leaked and
 * *failed_index (if non-NULL) names the problem that failed. */
int efgp_batch_setup(const efgp_problem* probs, int nprob, const efgp_options* opt,
                     efgp_batch** out, int* failed_index);

/* Solve all problems (step 4 for each), each to its own tolerance.  By
 * default (cg_mode 0 or 3) one launch of a work-claiming scheduler runs every
 * problem's CG: resident blocks claim work items (FFT line batches, vector
 * chunks) of any problem's current phase, and the block finishing a phase
 * reduces it and publishes the next; its device-side waits for work are
 * bounded (ETIMEOUT).  cg_mode 1 captures a CUDA graph per group of
 * iterations with a branch per problem; cg_mode 2 runs one thread-block
 * cluster per problem.  info: nprob entries or NULL (true_rel_residual is
 * -1: not recomputed).  Returns ENOTCONV if any problem hit its cap. */
int efgp_batch_solve(efgp_batch* b, efgp_solve_info* info);

/* Predict problem `index` of the batch at q targets. */
int efgp_batch_predict(efgp_batch* b, int index, const void* targets, int64_t q, void* mu_out);

/* Parameters / handle of one problem of the batch (owned by the batch). */
int efgp_batch_get_params(const efgp_batch* b, int index, efgp_params* out);
efgp_handle* efgp_batch_handle(efgp_batch* b, int index);

void efgp_batch_destroy(efgp_batch* b);

/* Library version string. */
const char* efgp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* EFGP_H */
