/*
 * fio.h -- C ABI of the GB300 (sm_103a) library that applies discrete Fourier
 * integral operators with the wedge-factorised algorithm of Candes, Demanet and
 * Ying, "Fast Computation of Fourier Integral Operators".
 *
 * The operator (Sec. 1.2, Eq. dfio with the unitary DFT of Eq. dft):
 *
 *     (Lf)(x) = (1/N) sum_{xi in Omega} a(x,xi) exp(2 pi i Phi(x,xi)) fhat(xi),
 *     fhat(xi) = (1/N) sum_{x in X} exp(-2 pi i x.xi) f(x),
 *
 * on X = {(n1/N, n2/N) : 0 <= n1, n2 < N} and Omega = [-N/2, N/2)^2 (N even).
 *
 * Data layout shared by every call:
 *   - an N x N grid function is N*N interleaved complex numbers (re, im),
 *     index n1*N + n2 holds the value at x = (n1/N, n2/N);
 *   - a batch of B grid functions is B such arrays back to back;
 *   - precision FIO_MIXED uses complex64 (two floats), FIO_FP64 complex128;
 *   - a spectrum (fio_dft2) is in centred order: index (k1 + N/2)*N + (k2 + N/2)
 *     holds xi = (k1, k2).
 *
 * Pointers named f, g, out, in are DEVICE pointers owned by the caller.  The
 * plan owns its own device memory.  `stream` is a cudaStream_t (NULL = the
 * legacy default stream); every apply call is asynchronous on it and does no
 * host synchronisation.
 *
 * Errors: every call returns a status code and never throws.  A CUDA error from
 * an asynchronous launch is reported by that call if the launch fails, or by a
 * later call (fio_plan_sync).  fio_last_error() returns a thread-local message
 * describing the last failure of the calling thread.
 */
#ifndef FIO_H_
#define FIO_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fio_plan_s *fio_plan;
typedef struct fio_surrogate_s *fio_surrogate;

typedef enum {
  FIO_OK = 0,
  FIO_EINVAL = 1,        /* invalid argument (N odd or out of range, eps, NaN params, ...) */
  FIO_ENOMEM = 2,        /* a device or host allocation failed; nothing leaks */
  FIO_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
  FIO_ERANK = 4,         /* the adaptive sample count exceeded rank_cap (Sec. 3.2) */
  FIO_ETIMEOUT = 5,      /* a bounded device wait gave up */
  FIO_EUNSUPPORTED = 6   /* valid request this build does not implement */
} fio_status;

/* Phase functions Phi(x, xi) = x.xi + Psi(x, xi), homogeneous of degree 1 in xi.
 * theta = arg(xi) = atan2(xi2, xi1); every phase is 0 at xi = 0. */
typedef enum {
  /* Psi = -x0.xi + c|xi|; params {x01, x02, c}.  Translation by x0 and the
   * constant-speed wave propagator of Sec. 1.1 (Eq. wave_solution). */
  FIO_PHASE_SHIFT_WAVE = 0,
  /* Psi = sqrt(c1(x)^2 xi1^2 + c2(x)^2 xi2^2) with
   * c1 = A1 + B1 sin(2 pi x1) sin(2 pi x2), c2 = A2 + B2 cos(2 pi x1) cos(2 pi x2);
   * params {A1, B1, A2, B2}.  The ellipse phase family of Sec. 4 (Eq. nrphase). */
  FIO_PHASE_ELLIPSE = 1,
  /* Psi = |xi| tau(x, theta), tau = sum_j a_j cos(2 pi (k1_j x1 + k2_j x2) + m_j theta + p_j);
   * params: nmodes rows {a_j, k1_j, k2_j, m_j, p_j}, m_j an integer in [-8, 8]. */
  FIO_PHASE_TAU_MODES = 2,
  /* Psi = sqrt(r1(x)^2 xi1^2 + r2(x)^2 xi2^2) with product-form axes
   * r1 = s1 (a1 + sin 4 pi x1)(a1 + sin 4 pi x2), r2 = s2 (a2 + cos 4 pi x1)(a2 + cos 4 pi x2);
   * params {a1, s1, a2, s2}.  The axes of the paper's own experiments (Sec. 4,
   * Eq. nrphase and the separation tests of Tables 1-3): a1 = a2 = 2, s1 = s2 = 1/9. */
  FIO_PHASE_ELLIPSE_PRODUCT = 3
} fio_phase_kind;

typedef struct {
  int kind;              /* fio_phase_kind */
  int nmodes;            /* FIO_PHASE_TAU_MODES only */
  const double *params;  /* HOST memory, read during fio_plan_create only */
} fio_phase;

typedef enum {
  FIO_AMP_ONE = 0,       /* a = 1 (the Egorov operator of Sec. 3) */
  FIO_AMP_SEPARABLE = 1, /* a = (1 + a1 sin 2 pi x1)(1 + a2 cos theta), cos theta := 1 at xi = 0 */
  FIO_AMP_HANKEL = 2     /* integration along ellipses (Appendix A, Eq. ellipses_amp): with
                            s = a1 (+1 or -1) and rho = s (Phi(x, xi) - x.xi) >= 0,
                            a = (J0(2 pi rho) + i s Y0(2 pi rho)) exp(-2 pi i s rho) / (4 pi);
                            the Y0 term is dropped where rho <= 0 (xi = 0).  a2 is unused.
                            L+ (s = +1, Phi = x.xi + rho) plus L- (s = -1, Phi = x.xi - rho)
                            integrates f along the ellipses of axes r1, r2 */
} fio_amp_kind;

typedef struct {
  int kind;              /* fio_amp_kind */
  double a1, a2;
} fio_amplitude;

typedef enum {
  FIO_MIXED = 0,  /* complex64 FFT / NUFFT / accumulation; FP64 plan */
  FIO_FP64 = 1    /* complex128 everywhere */
} fio_precision;

/* Storage of the x-side factors gamma^x of the separated kernel (Sec. 3.2).
 * FIO_ALPHA_STORED keeps gamma^x_t(x) for every x, wedge and rank term:
 * L N^2 q complex values (4.7 GB at N = 1024, eps = 1e-4), read by every apply.
 * FIO_ALPHA_RECOMPUTE keeps only what Eq. probnewfac needs to form them again,
 * gamma^x = A_[C] V S^-1 (the sampled columns xi_c of each wedge and the r x q
 * matrix V S^-1), plus per-x phase data, and forms gamma^x in every apply and
 * adjoint, a few wedges at a time, into a buffer the plan owns.  The operator is
 * the same to rounding: complex64 plans form the entries A_{x,xi_c} in single
 * precision from cancellation-free forms of the residual phase, FP64 plans with
 * the plan's own FP64 evaluation.  Not available for the Hankel amplitude on
 * complex64 plans (FIO_EUNSUPPORTED): its demodulated Bessel functions need FP64.
 * Complex64 recompute plans keep the plain warped points even when a surrogate
 * is given (the single-precision forms assume the exact gradient as the warp). */
typedef enum {
  FIO_ALPHA_STORED = 0,
  FIO_ALPHA_RECOMPUTE = 1
} fio_alpha_mode;

typedef struct {
  int precision;              /* fio_precision (default FIO_MIXED) */
  int L;                      /* number of wedges; 0 = ceil(sqrt(N)) rounded up to a multiple of 8 */
  double sigma;               /* NUFFT oversampling factor; 0 = 2 */
  int kb_width;               /* Kaiser-Bessel width in grid cells; 0 = ceil(log10(45/eps)) */
  unsigned long long seed;    /* seed of the random column/row samples of Sec. 3.2 */
  int r0;                     /* initial sample count r; 0 = 8 */
  int rank_cap;               /* largest r before FIO_ERANK; 0 = 1024 */
  int max_batch;              /* largest batch the plan's workspace holds; 0 = 1 */
  fio_surrogate surrogate;    /* trained phase surrogate (tau-mode phases), or NULL; see below */
  double surrogate_warp_budget; /* largest judged warp error, in cycles at |xi| = N/sqrt 2, for
                                   which the surrogate's warped points are used; 0 = 0.5 */
  double sep_cut;             /* singular values of A_[C] above sep_cut * eps * s_1 are kept
                                 (Sec. 3.2 step 2); 0 = 0.25, at most 1 */
  double sep_target;          /* a sample is accepted when the validated separation error is
                                 at most sep_target * eps and q <= r/3; 0 = 0.5, at most 1 */
  int alpha_mode;             /* fio_alpha_mode (default FIO_ALPHA_STORED) */
  int alpha_group;            /* FIO_ALPHA_RECOMPUTE: wedges whose gamma^x is formed at a time
                                 (the buffer holds that many wedges' factors); 0 = 4 */
} fio_options;

/* Fill *opt with the defaults listed above.  Returns FIO_EINVAL for NULL. */
fio_status fio_options_default(fio_options *opt);

/* Build a plan for L on an N x N grid (Sec. 1.3 wedges; Sec. 3.2 randomized
 * separation of a(x,xi) exp(2 pi i Phi_l(x,xi)) to relative accuracy eps; Sec. 3.4
 * shear/translate boxes and NUFFT grids).
 *   N      even, 8 <= N <= 2048
 *   phase  host descriptor, copied; NaN or Inf parameters give FIO_EINVAL
 *   amp    NULL means a = 1
 *   eps    separation threshold, 1e-12 <= eps <= 0.1 (singular values below
 *          eps * s_1 are dropped)
 *   opt    NULL means defaults
 * Uses the current CUDA device; synchronises it.  On failure *out_plan = NULL and
 * every allocation made so far is released. */
fio_status fio_plan_create(int N, const fio_phase *phase, const fio_amplitude *amp, double eps,
                           const fio_options *opt, fio_plan *out_plan);

/* out = L f for `batch` inputs (Sec. 3.4 evaluation: FFT, windowed scatter by
 * gamma^xi, type-2 NUFFT at the warped points, gamma^x multiply and sum).
 * f, out: device arrays of batch*N*N complex (complex64 for FIO_MIXED plans,
 * complex128 for FIO_FP64).  1 <= batch <= max_batch.  out must not alias f.
 * One plan must not be used on two streams at the same time (shared workspace).
 * The sum over wedges is accumulated with atomic adds into out, so the last bit
 * of a result may differ between runs (the order of the additions is not
 * fixed); every other step, and the whole adjoint, is deterministic: the same
 * call gives the same bits.  The order of the adjoint's spread sums depends on
 * the batch size, so one input may differ in its last bits between batch sizes. */
fio_status fio_apply(fio_plan plan, const void *f, void *out, int batch, void *stream);

/* out = L f for a real f (Eq. dft applied to f(x) + 0i): the same operator and
 * result as fio_apply on the complex array with zero imaginary parts.
 * f: device array of batch*N*N real values, float for FIO_MIXED plans and
 * double for FIO_FP64, half the bytes of its complex form; out as for fio_apply
 * (complex).  Same rules as fio_apply; out must not overlap f. */
fio_status fio_apply_real(fio_plan plan, const void *f, void *out, int batch, void *stream);

/* out = L* g (Sec. 3.5: gamma^x-conjugate multiply, type-1 NUFFT, conj(gamma^xi)
 * windowed gather, inverse FFT).  Same layout and rules as fio_apply.  The result
 * is the exact conjugate transpose of the fast forward operator, so
 * <L f, g> = <f, L* g> holds to rounding. */
fio_status fio_apply_adjoint(fio_plan plan, const void *g, void *out, int batch, void *stream);

/* out = L* L f, the normal operator (imaging's "migration of the modelled data",
 * the paper's Figure 2 setting), in one call: fio_apply, then fio_apply_adjoint
 * of its result, queued on `stream` with no host synchronisation in between.
 * The intermediate L f is held in out itself (the adjoint reads all of its input
 * before it writes its output), so the call needs no memory beyond the plan's.
 * Same layout and rules as fio_apply; out must not alias f.  The result equals
 * fio_apply_adjoint(fio_apply(f)) up to the rounding order of fio_apply's
 * atomic sum over wedges. */
fio_status fio_apply_normal(fio_plan plan, const void *f, void *out, int batch, void *stream);

/* ---------------------------------------------------------------------------
 * Forward apply that allocates nothing.
 *
 * Some callers cannot allocate device memory while they run: a framework that
 * owns all device memory through its own pool and forbids other allocations,
 * a real-time loop that cannot pay the latency or risk the failure of a
 * cudaMalloc, or a process that has already handed the rest of the GPU to
 * other work.  fio_apply_noalloc computes exactly what fio_apply computes, but
 * its NUFFT grids and spectrum live in one fixed scratch array compiled into
 * this library (a file-scope device array of FIO_NOALLOC_SCRATCH_BYTES, held
 * by every GPU that loads the library until the process exits) instead of the
 * plan's workspace.  It calls no cudaMalloc, cudaFree or other allocating
 * routine, and records no timing events.  The paper has no counterpart; this
 * is an interface convenience.
 *
 *   - Limit: grid_points * batch + N * N * batch complex values (complex64 for
 *     FIO_MIXED, complex128 for FIO_FP64) must fit in FIO_NOALLOC_SCRATCH_BYTES;
 *     larger requests return FIO_EINVAL with the sizes in fio_last_error().
 *   - Set-up: the first call on a device looks up the scratch array's device
 *     address (cudaGetSymbolAddress) with that device current, and the plan's
 *     device must be the current device.  Make that first call before any
 *     stream capture.  The address is kept for the life of the process: after
 *     cudaDeviceReset (which also destroys every plan on that device) no call
 *     may follow.
 *   - Sharing: every call uses the same array, which keeps the last call's
 *     contents.  The forward path writes every scratch value before reading it,
 *     so nothing has to be cleared, but two calls that may overlap on the GPU
 *     (different streams, or different host threads without ordering) race on
 *     the array: serialise them.
 * f, out, batch and stream as for fio_apply; batch is not limited by the plan's
 * max_batch, only by the scratch size. */
#define FIO_NOALLOC_SCRATCH_BYTES (32u << 20)
fio_status fio_apply_noalloc(fio_plan plan, const void *f, void *out, int batch, void *stream);

/* ---------------------------------------------------------------------------
 * Learned phase surrogate (tau-mode phases Phi = x.xi + |xi| tau(x, theta)).
 *
 * A 4 -> 64 -> 64 -> 3 tanh network maps (x1, x2, cos theta, sin theta) to
 * (tau, d tau/d x1, d tau/d x2); d tau/d theta is its directional derivative.  It
 * is trained on the GPU on `nsamples` plain evaluations (the literal sum over the
 * modes, FP64) with Adam, BF16 tensor-core products and FP32 accumulation, then
 * judged on 65536 held-out plain samples.
 *
 * fio_plan_create uses it for the warped points y_l(x) = grad_xi Phi(x, xihat_l)
 * only when the judged warp error, in cycles at |xi| = N/sqrt 2, is within
 * surrogate_warp_budget: any smooth warp keeps the factorisation of
 * a exp(2 pi i Phi) exact (the residual is always formed from the plain phase),
 * only the separation rank changes.  Its residual-phase error in cycles is
 * reported; the plain phase stays the residual's judge and is always used.
 *
 * Parameter vector (FP32, fio_surrogate_nparams() values): W1[4][64], b1[64],
 * W2[64][64], b2[64], W3[64][3], b3[3], row-major with the input index first.
 * Outputs are scaled by tau_scale (tau) and dx_scale (x-derivatives) of
 * fio_surrogate_info.  All pointers below are DEVICE pointers unless stated. */
typedef struct {
  int nparams, nsamples, epochs;
  long long steps;
  double train_seconds, final_loss;   /* mean squared error of the scaled outputs */
  double tau_scale, dx_scale;
  double heldout_tau_maxerr;          /* max |tau_net - tau| on held-out samples */
  double heldout_dx_maxerr;           /* max over x1, x2 of the derivative errors */
  double heldout_dtheta_maxerr;       /* max |d_theta tau_net - d_theta tau| */
  double heldout_tau_relrms;          /* RMS error of tau relative to RMS tau */
} fio_surrogate_info;

fio_status fio_surrogate_train(const fio_phase *phase, int nsamples, int epochs, int batch,
                               unsigned long long seed, fio_surrogate *out);
void fio_surrogate_destroy(fio_surrogate s);
fio_status fio_surrogate_get_info(fio_surrogate s, fio_surrogate_info *info);
/* Copy the FP32 parameters to (set = 0) or from (set = 1) the HOST array params. */
fio_status fio_surrogate_params(fio_surrogate s, float *params, int set);
/* y4[i] = (tau, d tau/d x1, d tau/d x2, d tau/d theta) for x4[i] = (x1, x2, cos, sin). */
fio_status fio_surrogate_eval(fio_surrogate s, int n, const float *x4, float *y4, void *stream);
/* Mean squared error of the scaled outputs against t3 (n x 3, scaled targets) and
 * its gradient with respect to the parameters (grad: nparams floats). */
fio_status fio_surrogate_loss_grad(fio_surrogate s, int n, const float *x4, const float *t3,
                                   float *grad, double *loss);
/* The plain-evaluation samples the training uses: x4 (n x 4 floats) and
 * t4 = (tau, d1, d2, d_theta) in FP64 (n x 4 doubles). */
fio_status fio_surrogate_samples(const fio_phase *phase, int n, unsigned long long seed, float *x4,
                                 double *t4);
int fio_surrogate_nparams(void);

/* Wait for the plan's work on `stream` and report any pending CUDA error. */
fio_status fio_plan_sync(fio_plan plan, void *stream);

typedef struct {
  int N, L, precision, kb_width, max_batch;
  double sigma, kb_beta, eps;
  int q_max, q_min, r_max;
  double q_mean;
  unsigned long long bytes_alpha;   /* gamma^x factors on the device */
  unsigned long long bytes_beta;    /* gamma^xi factors */
  unsigned long long bytes_warp;    /* warped points */
  unsigned long long bytes_grid;    /* NUFFT grids for max_batch inputs */
  unsigned long long bytes_total;   /* all device memory the plan holds */
  unsigned long long grid_points;   /* sum over wedges of m1*m2*q (one input) */
  unsigned long long alg_bytes_apply; /* algorithmic HBM bytes of one batch-1 apply */
  double plan_seconds;              /* wall time of fio_plan_create */
  unsigned long long kernel_launches; /* this plan's kernel launches so far (all applies) */
  int surrogate_warp;               /* 1 if the warped points came from the surrogate */
  double surrogate_warp_cycles;     /* the surrogate's judged warp error (cycles), or 0 */
  double surrogate_residual_cycles; /* its judged residual-phase error (cycles), or 0 */
  int max_bin_points;               /* most points in one bin (the points of a wedge are sorted
                                       by window-start cell; a bin is 16 x 16 start cells) */
  double mean_bin_points;           /* mean points per non-empty bin */
  int max_spread_candidates;        /* most points whose windows reach one bin's cells */
  double sep_error;                 /* largest per-wedge estimate of the relative Frobenius
                                       error of the separated factors (Sec. 4, Table 1's
                                       estimator over every column, on 200 random rows) */
  int alpha_mode;                   /* fio_alpha_mode of the plan */
  int alpha_groups;                 /* recompute mode: regeneration groups per apply, else 0 */
  unsigned long long bytes_recompute; /* recompute mode: sampled columns, V S^-1 and per-x phase
                                       data (bytes_alpha is then the regeneration buffer) */
} fio_plan_info;

/* Plan summary (host struct filled). */
fio_status fio_plan_get_info(fio_plan plan, fio_plan_info *info);

typedef struct {
  int M[4];          /* shear: xi'' = M xi, row-major integer matrix, det 1 */
  int xc1, xc2;      /* box centre xi_c: xi' = M xi - xi_c */
  int b1, n1, b2, n2; /* box: xi'_1 in [b1, b1+n1), xi'_2 in [b2, b2+n2) */
  int m1, m2;        /* oversampled grid */
  int q;             /* separation rank */
  int r;             /* final random sample count */
  int npts;          /* |W_l|: frequencies owned by this wedge */
} fio_wedge_info;

/* Stages of the apply path, for per-stage timing (Sec. 3.4 and 3.5 steps). */
typedef enum {
  FIO_STAGE_S0_DFT = 0,      /* unitary 2D DFT of the input */
  FIO_STAGE_S1_SCATTER = 1,  /* beta' fhat placed in the grids, row FFTs */
  FIO_STAGE_S2_COLFFT = 2,   /* column FFTs of the grids */
  FIO_STAGE_S3_INTERP = 3,   /* KB interpolation, alpha' multiply, sums over t and l */
  FIO_STAGE_S4A_SPREAD = 4,  /* adjoint: type-1 spread of conj(alpha') g */
  FIO_STAGE_S4B_COLFFT = 5,  /* adjoint: column FFTs, box rows kept */
  FIO_STAGE_S4B_ROWFFT = 6,  /* adjoint: row FFTs, wedge runs kept */
  FIO_STAGE_S4C_GATHER = 7,  /* adjoint: sum_t conj(beta') Ghat into the owner wedge */
  FIO_STAGE_S4D_IDFT = 8,    /* adjoint: inverse unitary 2D DFT */
  FIO_NUM_STAGES = 9
} fio_stage;

/* Turn per-stage timing on or off.  When on, every apply records a pair of CUDA
 * events around each stage on the launch stream (a few microseconds each). */
fio_status fio_plan_set_timing(fio_plan plan, int on);

/* Stage times accumulated since the previous call: ms[s] = summed event time of
 * stage s in milliseconds, count[s] = its number of timed executions (host
 * arrays of FIO_NUM_STAGES; either may be NULL).  Synchronises on the recorded
 * events, then resets the accumulators. */
fio_status fio_plan_stage_times(fio_plan plan, double *ms, long long *count);

/* Geometry and rank of wedge l (0 <= l < L). */
fio_status fio_plan_get_wedge(fio_plan plan, int l, fio_wedge_info *info);

/* Export the separated factors of wedge l to HOST arrays (complex128):
 *   alpha[t*N*N + x] = gamma^x_{l t}(x)  (columns of U, Sec. 3.2),
 *   beta[t*npts + p] = gamma^xi_{l t}(xi_p) (rows of T), with xi_p = (k1[p], k2[p]).
 * Any pointer may be NULL.  Sizes: alpha q*N*N, beta q*npts, k1/k2 npts.  For tests
 * of the separation error (the estimator of Sec. 4, Table 1). */
fio_status fio_plan_export_wedge(fio_plan plan, int l, double *alpha, double *beta, int *k1,
                                 int *k2);

/* Export the warped points of wedge l as the plan stores them: y[2*x + d] =
 * (M^-T grad_xi Phi(x, xihat_l))_d mod 1, rounded to 32-bit fractions (HOST
 * array of 2*N*N doubles).  With the factors of fio_plan_export_wedge,
 * exp(2 pi i Phi(x,xi)) a(x,xi) ~ exp(2 pi i y(x).(M xi)) sum_t alpha_t(x) beta_t(xi)
 * for xi in W_l (Sec. 1.4 and Sec. 3.2). */
fio_status fio_plan_export_warp(fio_plan plan, int l, double *y);

void fio_plan_destroy(fio_plan plan);

/* Write the plan to the file `path` (host path), so that fio_plan_load can
 * rebuild it without repeating the preprocessing of Sec. 3.2: the factors
 * alpha' and beta', the warped points, the point order, the wedge tables and the
 * work lists, as the plan holds them (about bytes_total minus the workspace).
 * Synchronises the device.  FIO_EINVAL if the file cannot be opened, FIO_ECUDA
 * if a copy or a write fails. */
fio_status fio_plan_save(fio_plan plan, const char *path);

/* Rebuild a plan saved by fio_plan_save, on the current device.  max_batch > 0
 * sizes the new workspace (0 = the saved plan's).  The loaded plan applies the
 * same operator with the same arithmetic as the saved one.  FIO_EINVAL for a
 * missing file, a file of another format or version, or a corrupt or truncated
 * file (checked before any device allocation where the header tells);
 * FIO_ENOMEM if the device allocations fail.  On failure *out_plan = NULL and
 * nothing leaks. */
fio_status fio_plan_load(const char *path, int max_batch, fio_plan *out_plan);

/* Unitary 2D DFT of Eq. dft (inverse = 0) or its inverse (inverse = 1) on the
 * GPU, spectrum in centred order.  in/out: device arrays of batch*N*N complex
 * (precision as above); in == out is allowed.  N = 2^a 3^b 5^c, 8 <= N <= 4096. */
fio_status fio_dft2(int N, int precision, const void *in, void *out, int batch, int inverse,
                    void *stream);

/* ---------------------------------------------------------------------------
 * Host utilities.  They run on the CPU only (no CUDA call), so the host logic
 * of the plan can be inspected and tested without a GPU.
 * ------------------------------------------------------------------------- */

/* Default wedge count for N: ceil(sqrt N) (Sec. 1.3 takes sqrt N wedges)
 * rounded up to a multiple of 8, so that both diagonals are wedge centres. */
int fio_default_wedges(int N);

/* wedge_of[(k1 + N/2)*N + (k2 + N/2)] = l with
 * (2l - 1) pi / L <= arg xi < (2l + 1) pi / L (Sec. 1.3); xi = 0 is put in wedge 0.
 * wedge_of: host array of N*N ints. */
fio_status fio_wedge_map(int N, int L, int *wedge_of);

/* Box and grid of wedge l as fio_plan_create builds them (Sec. 3.4), for
 * oversampling sigma and KB width kb_width (q and r are returned as 0). */
fio_status fio_wedge_geometry(int N, int L, double sigma, int kb_width, int l,
                              fio_wedge_info *info);

/* Kaiser-Bessel kernel phi(s) = I0(beta sqrt(1 - (2s/w)^2)) / I0(beta) (0 for
 * |s| >= w/2) at n points s[], and its Fourier transform
 * phihat(nu) = int phi(s) exp(-2 pi i nu s) ds at n points nu[] (host arrays;
 * phi / phihat may be NULL to skip).  beta <= 0 selects the default shape
 * pi sqrt((w/sigma)^2 (sigma - 1/2)^2 - 0.8) for sigma = 2. */
fio_status fio_kb_eval(int w, double beta, int n, const double *s, double *phi, const double *nu,
                       double *phihat);

/* Default KB width for a separation threshold eps: ceil(log10(45 / eps)). */
int fio_kb_width_for(double eps);

/* Eigendecomposition of a Hermitian n x n complex matrix (host, row-major,
 * interleaved re/im, n <= 1024) by Householder tridiagonalisation and implicit
 * symmetric QR steps with Wilkinson shifts: evals descending, V's columns the
 * eigenvectors (row-major interleaved).  A host utility; the randomized
 * separation does not form Gram matrices (see fio_host_svd). */
fio_status fio_host_eigh(int n, const double *A, double *evals, double *V);

/* Singular value decomposition of an m x n complex matrix (host, row-major,
 * interleaved re/im; 1 <= m <= 1 << 20, 1 <= n <= 1024) by one-sided Jacobi
 * rotations: s (n values, descending), AV = A V (m x n; column j is s_j times
 * the j-th left singular vector, or a zero column where s_j = 0) and V (n x n,
 * columns the right singular vectors).  The randomized separation (Sec. 3.2)
 * applies it to the triangular factor of A_[C] = Q R and to U_[R]; small
 * singular values keep an absolute accuracy of about 1e-16 s_1.  Any output
 * pointer may be NULL. */
fio_status fio_host_svd(int m, int n, const double *A, double *s, double *AV, double *V);

/* Singular values s (descending) and right singular vectors V (columns, n x n
 * row-major interleaved) of a square n x n complex matrix R (host; n <= 2048) by
 * one-sided Jacobi preconditioned with a column-pivoted QR: R P = Q1 R1, then
 * Jacobi on R1^H, which converges in a few sweeps.  This is the solver the
 * randomized separation (Sec. 3.2) applies to the triangular factor of A_[C].
 * A column of V whose singular value is 0 is returned as zeros. */
fio_status fio_host_svd_right(int n, const double *R, double *s, double *V);

const char *fio_status_string(fio_status s);
const char *fio_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int fio_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FIO_H_ */
