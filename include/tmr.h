/*
 * tmr.h -- C ABI of libtmr, GB300 (sm_103a) reference-less transmission-matrix
 * (TM) retrieval with FFT-structured probing, after Zhong et al.,
 * "Efficient reference-less transmission matrix retrieval for a multimode
 * fiber using fast Fourier transform" (arXiv 2302.13524).
 *
 * Problem (Sec. 2.2).  The TM has M rows (output pixels, on an ny x nx grid,
 * row = a*nx + b) of N complex entries (input modes).  Row t is probed by
 * Q = [F D_1; ...; F D_J] (Eq. probingmatrix), F the unnormalised N-point DFT
 * F x[k] = sum_n x[n] exp(-2 pi i k n / N) and D_j = diag(d_j), |d_j[n]| = 1.
 * Each row yields K = J*N intensities y[j*N + k] = |(F (d_j .* t))[k]|^2
 * (Eq. forwardmodel / Eq. optTMsmall2).  Retrieval minimises, independently
 * per row, f(t) = ||y - |Q t|^2||^2 (Eq. optTMsmall2) by L-BFGS (Algorithm 1),
 * then fits one phase offset per row from defocus intensities (Sec. 2.3,
 * Eq. optphase) and returns diag(e^{i phi}) T_est (Eq. phaseoffset).
 *
 * Data layout (all row-major, complex values interleaved re,im):
 *   masks  complex64 [J][N]
 *   T      complex64 [M][N]
 *   y      float32   [M][J][N]   (pattern index i = j*N + k within a row)
 *   y_def  float32   [n_defocus][M]
 *   G      complex64 [M][N]      gradient packed as df/dRe t + i df/dIm t
 *
 * Pointers.  Unless stated otherwise an array argument may be a device
 * pointer or a host pointer (pinned or pageable); the library checks with
 * cudaPointerGetAttributes and stages host arrays through device buffers it
 * owns, copying results back before the call returns.  With device pointers
 * every call is asynchronous on the handle's stream; argument errors are
 * returned synchronously; numerical trouble of a single row is reported in
 * row_status.  The caller owns every array it passes; the library never
 * keeps a caller pointer past the call (masks and H are copied at create).
 *
 * Errors.  Every entry point returns a tmr_status; on failure
 * tmr_last_error() returns a message for the calling thread.  No entry point
 * falls back to the CPU: sizes without a GPU path return TMR_ERR_UNSUPPORTED.
 * A handle is not thread-safe.
 */
#ifndef TMR_H
#define TMR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tmr_handle tmr_handle; /* opaque, owned by the library */

typedef enum {
    TMR_OK = 0,
    TMR_ERR_INVALID_ARG = 1, /* bad size, NULL where not allowed, bad option     */
    TMR_ERR_UNSUPPORTED = 2, /* no GPU path for this N, J or option              */
    TMR_ERR_OOM = 3,         /* device allocation failed or over workspace_limit */
    TMR_ERR_CUDA = 4,        /* a CUDA runtime call failed                       */
    TMR_ERR_TIMEOUT = 5,     /* tmr_sync gave up waiting                         */
    TMR_ERR_NUMERIC = 6      /* a row reported non-finite values (tmr_sync)      */
} tmr_status;

/* Initial value of each row (Algorithm 1, first step). */
enum {
    TMR_INIT_RANDOM = 0,   /* Philox4x32-10 complex normal, scaled to ||t||^2 = sum(y)/(J N) */
    TMR_INIT_BP = 1,       /* back-propagation t0 = Q^H sqrt(y) / (J N), Eq. backpropagation */
    TMR_INIT_SPECTRAL = 2, /* power iteration on Q^H diag(min(y/mean y, clip)) Q / (J N)    */
    TMR_INIT_LEARNED = 3   /* the network of tmr_set_init_model proposes t0 from sqrt(y); the
                              proposal seeds the spectral power iteration (power_iters
                              steps) in place of the Philox vector, and a row whose
                              proposal is not finite or is zero keeps the Philox seed (the
                              plain spectral start).  With power_iters = 0 the solver keeps,
                              per row, whichever of the proposal and the random start has
                              the lower loss                                             */
};

/* Per-row outcome written to row_status. */
enum {
    TMR_ROW_MAXITER = 0,   /* ran all iterations                                   */
    TMR_ROW_CONVERGED = 1, /* stopped early: tolerance met, zero loss or gradient  */
    TMR_ROW_ZERO = 2,      /* all intensities zero: t = 0, no iteration (Sec. 2.2,
                              rows outside the fiber mask)                        */
    TMR_ROW_NUMERIC = 3    /* non-finite intensity or iterate; t = 0 or last value */
};

/* Arithmetic of tmr_retrieve (and of tmr_forward / tmr_grad on the handle).
 * TMR_PREC_FP32: FP32 FFTs, FP32 intensities and L-BFGS pairs.
 * TMR_PREC_MIXED (N = 256, 1024, 2048 or 4096; not an arithmetic of the
 * paper, which works in double precision): intensities stored as FP16 after
 * dividing each row by its largest |y| (the handle packs them, M*J*N*2
 * bytes); L-BFGS pairs stored as BF16 (the iterate, gradient and direction
 * stay FP32); each length-N DFT as radix-16 and radix-8 passes whose small
 * DFTs run on the tensor cores as split BF16 (hi + lo) GEMMs with FP32
 * accumulation, about 1e-5 relative error per transform; the last 10 L-BFGS iterations (when iters > 10) go
 * back to FP32 transforms after a fresh FP32 evaluation of f and g at the
 * current iterate, which restarts the history.  The phase-offset fit is FP64
 * either way. */
enum { TMR_PREC_FP32 = 0, TMR_PREC_MIXED = 1 };

/* Defocus operator of the phase-offset fit (Sec. 2.3).  Two kinds.
 *
 * TMR_DEFOCUS_SAME_GRID (kind 0): the defocus field of pattern n is D c_n
 * with c_n[row] = (Q t_row)[n] (the first n_defocus probe patterns) and
 * D x = ifft2(H .* fft2(x)) on the ny x nx pixel grid; the defocus images are
 * float [n_defocus][M].  H: device or host complex64 [ny][nx], or NULL for the
 * quadratic phase H[a][b] = exp(-i coef (ky_a^2 + kx_b^2)) on signed integer
 * frequencies (k = idx for 2 idx < n, else idx - n).
 *
 * TMR_DEFOCUS_ANGULAR_2X (kind 1, Eq. angularspectrum and Eq.
 * forwarddefocusImage): n_defocus separate incident fields theta_n (complex64
 * [n_defocus][N], `incident`, copied) give the fields c_n = T theta_n on the
 * half-sampled ny x nx grid (c_n[row] = sum_k T[row][k] theta_n[k]), and the
 * image of pattern n is |K2^H P diag(h) K1 c_n|^2 on the full 2ny x 2nx grid:
 * K1 the 2D DFT of the half grid, h the angular-spectrum kernel
 * exp(i 2 pi / wavelength sqrt(1 - (wavelength u)^2 - (wavelength v)^2) z_d)
 * inside the pupil wavelength sqrt(u^2 + v^2) <= na (0 outside), with
 * u = kx / (nx pixel), v = ky / (ny pixel) on signed frequencies, P the zero
 * padding of the spectrum to the 2ny x 2nx grid and K2^H its inverse DFT
 * divided by ny nx (so that with h = 1 the even full-grid pixels equal the
 * half grid).  The images are float [n_defocus][4 M], each row-major
 * 2ny x 2nx.  H non-NULL replaces the computed h ([ny][nx], FFT order).
 * wavelength, pixel and z_d share one length unit. */
enum { TMR_DEFOCUS_SAME_GRID = 0, TMR_DEFOCUS_ANGULAR_2X = 1 };

typedef struct {
    int ny, nx;      /* ny * nx == M                                   */
    const void *H;   /* copied at tmr_create; NULL = made from the parameters */
    double coef;     /* kind 0: quadratic coefficient (0.05 in the workloads) */
    int n_defocus;   /* kind 0: 1..J*N; kind 1: 1..65536               */
    int kind;        /* TMR_DEFOCUS_SAME_GRID (0) or TMR_DEFOCUS_ANGULAR_2X */
    double wavelength, na, z_d, pixel;  /* kind 1: > 0, > 0, finite, > 0 */
    const void *incident;  /* kind 1: device or host complex64 [n_defocus][N] */
} tmr_defocus_op;

typedef struct {
    int m;                  /* L-BFGS memory, 1..6 (default 5)                       */
    int init;               /* TMR_INIT_* (default spectral)                         */
    unsigned long long seed;/* Philox key for random/spectral starts (default 0)     */
    int power_iters;        /* spectral start: power iterations, or Lanczos steps (default 100) */
    double clip;            /* spectral intensity clip, <= 0: none (default 2.0)     */
    double tol;             /* early exit when |f_prev - f| / f_prev < tol; 0 = off  */
    int phase_iters;        /* L-BFGS iterations of the phase-offset fit (default 100) */
    int precision;          /* TMR_PREC_FP32 (default) or TMR_PREC_MIXED             */
    int use_graph;          /* replay tmr_retrieve from a captured CUDA graph (default 0) */
    size_t workspace_limit; /* max device bytes the handle may allocate; 0 = no cap  */
    int schedule;           /* solver layout: 1, 2 or 4 = masks per CTA (must divide J),
                               a cluster of J/G CTAs per row, 8 points per thread;
                               16 = one CTA per row (FP32, N = 512..2048 with
                               J N / 16 <= 512 threads, 16 points per thread, L-BFGS
                               pairs, and the Lanczos vectors where they fit, in the
                               SM's tensor memory: no device workspace for them);
                               32 = for 2048 < N <= 2731, one mask per CTA with the
                               full-length Bluestein plan (FFTs of L = 8192) instead
                               of the split outputs at L = 4096 of schedule 1;
                               0 = chosen by the autotuner (default)                 */
    const char *tune_cache; /* JSON file caching autotuned schedules per device, N, J,
                               m; NULL = this process only                           */
    long long wait_spins;   /* bound on each device-side wait of the phase-offset fit's
                               grid barrier, in polls (default 1 << 24, about one
                               second); when a wait runs out the fit stops, every CTA
                               returns, phi keeps its last value and tmr_sync
                               returns TMR_ERR_TIMEOUT                               */
    int withhold_release;   /* test hook, 0 in normal use: 1 = the fit's grid barrier
                               is never released, so every wait runs out after
                               wait_spins polls (exercises the bounded wait)         */
    int probe_n1;           /* 0 (default): K is the 1D DFT of length N.  n1 > 0: K is
                               the paper's 2D DFT (Sec. 2.2, Eq. probingmatrix) of the
                               row read as an n1 x (N/n1) array (element a*(N/n1) + b
                               is row a, column b), its spectrum X[k1][k2] stored as
                               pattern k1 + n1*k2 of each mask (y, forward, gradient,
                               defocus fields).  FP32 only; N = 512 with n1 = 8 or 64,
                               or N = 4096 with n1 = 8, 64 or 512 (the strides at which
                               a pass of the register FFT starts); cluster schedules */
    int lanczos;            /* 0 (default): the spectral start runs power_iters power
                               iterations.  1: it runs power_iters (1..16) Lanczos
                               steps instead (the same leading eigenvector in far
                               fewer operator products; not in the paper): each step
                               one product with A, w orthogonalised against every
                               earlier Lanczos vector by two passes of classical
                               Gram-Schmidt, stop at an invariant subspace
                               (beta_j <= 1e-6 alpha_0); the start is the Ritz vector
                               of the largest eigenvalue of the tridiagonal,
                               signed so that its first coefficient is >= 0.  The
                               handle holds power_iters N complex64 per resident
                               CTA (one CTA per row) or cluster, up to 2 per SM.
                               Applies to TMR_INIT_SPECTRAL and TMR_INIT_LEARNED
                               (the proposal seeds the first Lanczos vector). */
    int cost;               /* TMR_COST_INTENSITY (default): Eq. optTMsmall2 with the
                               exact quartic line search.  TMR_COST_AMPLITUDE: the
                               Discussion's cost for Poisson noise,
                               f = sum (sqrt(y) - |Q t|)^2, real gradient
                               2 Q^H((|z| - sqrt(y)) z / |z|) (0 where z = 0), and a
                               line search that brackets the first sign change of
                               f'(t + al p) at al = 1, 2, 4, ... (40 doublings at
                               most) and finds it by Newton steps kept inside the
                               bracket (to 1e-6 al, 30 steps at most).  Applies to
                               tmr_grad and tmr_retrieve (the row loss reported is
                               this cost); the start and the defocus fit are
                               unchanged. */
    double phase_tol;       /* 0 (default): the phase-offset fit runs phase_iters
                               L-BFGS iterations or until a backtracking fails.
                               > 0: it also stops after an accepted step that
                               lowers g(phi) (Eq. optphase) by at most phase_tol
                               g -- the loss has reached its noise floor. */
    int dense;              /* 0 (default): the probing operator by FFTs.  1 or 2: the
                               paper's "without FFT" evaluation (Table 1) for
                               tmr_forward and tmr_grad: Q (J N x N, complex64,
                               Q[j N + k][n] = exp(-2 pi i k n / N) d_j[n]) is built
                               on the device at the first call (8 J N^2 bytes, plus
                               two J N x M scratch products), and Z = T Q^T and
                               G = -4 (Z .* r) conj(Q) (amplitude cost: its
                               coefficient) run as complex matrix products over
                               all rows (cuBLAS): 1 = FP32, 2 = FP32 emulated on
                               the tensor cores with three BF16 terms per operand.
                               tmr_retrieve then runs Algorithm 1 with every FFT
                               replaced by the matrix-vector product with the DFT
                               matrix (one mask per CTA, N^2 multiply-adds per
                               transform, the table of W_N^m in shared memory):
                               the paper's "TM retrieval without FFT", without
                               the phase-offset fit (y_def must be NULL; the
                               defocus calls return TMR_ERR_UNSUPPORTED).  FP32,
                               probe_n1 0, N a power of two in 64..4096. */
} tmr_options;

enum { TMR_COST_INTENSITY = 0, TMR_COST_AMPLITUDE = 1 };

/* Fill *opt with the defaults above. */
void tmr_default_options(tmr_options *opt);

/* Create a handle for M rows of length N probed with J masks.  With
 * opt->schedule == 0 the first handle for a (device, N, J, m) times every
 * solver schedule that fits (G masks per CTA with a cluster of J/G CTAs per
 * row, and one CTA per row) on synthetic rows and keeps the fastest; the
 * choice is cached in memory and, when opt->tune_cache names a file, in that
 * JSON file.
 *   masks      complex64 [J][N], |d| = 1 (not checked), copied.
 *   defocus_op NULL: no phase-offset fit; else copied (H copied).
 *   opt        NULL: defaults.
 *   stream     cudaStream_t for all work; NULL = the legacy default stream (with
 *              use_graph, a blocking stream the handle creates, which orders
 *              itself with the legacy default stream).
 * Supported on the GPU: 1 <= J <= 8 and N a power of two with
 * 64 <= N <= 4096 (one register FFT of length N), or any other N with
 * 16 <= N <= 4096 (Bluestein's chirp-z form of the same DFT through FFTs of
 * a power-of-two length L >= 2N - 1, or, for 2048 < N <= 2731, through
 * 4096-point FFTs with the outputs split in two halves; one mask per CTA).  When no solver
 * schedule fits the per-row state of (N, J, opt->m) in shared memory the
 * handle is still made (tmr_forward, tmr_grad and tmr_defocus_forward work),
 * tmr_schedule reports 0 and tmr_retrieve returns UNSUPPORTED.
 * Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
tmr_status tmr_create(tmr_handle **out, int N, int M, int J, const void *masks,
                      const tmr_defocus_op *defocus_op, const tmr_options *opt,
                      void *stream);

/* Forward model (Eq. optTMsmall2): Y[r][j][k] = |F(d_j .* T[r])[k]|^2.
 *   T complex64 [M][N] in, Y float32 [M][J][N] out. */
tmr_status tmr_forward(tmr_handle *h, const void *T, float *Y);

/* Loss and gradient (Eq. optTMsmall2, Eq. derivative, App. A):
 *   loss[r] = ||Y[r] - |Q T[r]|^2||^2,
 *   G[r]    = -4 Q^H diag(Q T[r]) (Y[r] - |Q T[r]|^2).
 * loss float32 [M] (may be NULL), G complex64 [M][N] (may be NULL). */
tmr_status tmr_grad(tmr_handle *h, const void *T, const float *Y, float *loss, void *G);

/* The whole path: initialise every row (opt.init), run `iters` L-BFGS
 * iterations of Algorithm 1 with an exact line search on the quartic
 * f(t + alpha p), then, when y_def != NULL and the handle has a defocus
 * operator, fit the phase offsets (Eq. optphase) from phi = 0 and write
 * T_out = diag(e^{i phi}) T_est (Eq. phaseoffset), phi shifted so that
 * arg(sum_r ||t_r||^2 e^{i phi_r}) = 0.
 *   y          float32 [M][J][N]
 *   y_def      float32 [n_defocus][M] or NULL (skip the phase fit)
 *   iters      >= 0
 *   T_out      complex64 [M][N]
 *   row_status int32 [M], row_iters int32 [M], row_loss float32 [M]: each may
 *              be NULL.
 * Rows whose intensities are all zero come back as t = 0 with status ZERO. */
tmr_status tmr_retrieve(tmr_handle *h, const float *y, const float *y_def, int iters,
                        void *T_out, int *row_status, int *row_iters, float *row_loss);

/* As tmr_retrieve, starting every row from T_init (complex64 [M][N]) with an
 * empty L-BFGS history (restart or resume from a checkpoint). */
tmr_status tmr_retrieve_from(tmr_handle *h, const void *T_init, const float *y,
                             const float *y_def, int iters, void *T_out, int *row_status,
                             int *row_iters, float *row_loss);

/* Defocus intensities of T (Eq. forwarddefocusImage with the handle's
 * operator): Y_def[n][r] = |(D c_n)[r]|^2, c_n[r] = (Q T[r])[n].
 *   Y_def float32 [n_defocus][M].  UNSUPPORTED without a defocus operator. */
tmr_status tmr_defocus_forward(tmr_handle *h, const void *T, float *Y_def);

/* Phase-offset fit alone (Sec. 2.3): given T_est and y_def, run the L-BFGS /
 * Armijo fit of Eq. optphase from phi = 0, write phi (float64 [M], may be
 * NULL) and T_out = diag(e^{i phi}) T_est (complex64 [M][N], may be NULL). */
tmr_status tmr_defocus_fit(tmr_handle *h, const void *T_est, const float *y_def, double *phi,
                           void *T_out);

/* Wait for the handle's stream, at most timeout_s seconds (<= 0: no limit),
 * polling.  Returns TMR_ERR_TIMEOUT when the work is still running or when a
 * grid-barrier wait of the last phase-offset fit (tmr_retrieve with y_def, or
 * tmr_defocus_fit) ran out (opt.wait_spins), TMR_ERR_NUMERIC when a row of
 * the last retrieve reported non-finite values. */
tmr_status tmr_sync(tmr_handle *h, double timeout_s);

/* Loss g(phi) (Eq. optphase) at the phi of the last phase-offset fit and its
 * accepted L-BFGS iterations (either pointer may be NULL); waits for the
 * handle's stream.  UNSUPPORTED without a defocus operator, INVALID_ARG
 * before the first fit. */
tmr_status tmr_phase_fit_report(tmr_handle *h, double *loss, int *iters);

/* Message describing the calling thread's last error ("" if none). */
const char *tmr_last_error(void);

/* Device bytes currently held by the handle. */
size_t tmr_workspace_bytes(const tmr_handle *h);

/* ---- learned initialiser (not in the paper: a network proposes t0) ----
 * A perceptron x -> GELU(W1 x + b1) -> GELU(W2 h1 + b2) -> W3 h2 + b3 with
 * FP32 master weights, BF16 copies feeding tensor-core products and FP32
 * accumulation.  Parameters are one flat FP32 vector W1 [h1][in], b1,
 * W2 [h2][h1], b2, W3 [out][h2], b3 (row-major).  For tmr_retrieve the input
 * is the row's sqrt(y) / sqrt(mean y) (in = J*N) and the output the real and
 * imaginary parts of t0 (out = 2*N), rescaled to ||t0||^2 = sum(y) / (J N).
 * X, T, Y, loss and grad are device arrays; all work runs on `stream`. */
typedef struct tmr_mlp tmr_mlp;

/* Weights drawn from U(-sqrt(3/fan_in), sqrt(3/fan_in)) by Philox(seed), biases 0. */
tmr_status tmr_mlp_create(tmr_mlp **out, int n_in, int n_h1, int n_h2, int n_out,
                          unsigned long long seed, void *stream);
size_t tmr_mlp_num_params(const tmr_mlp *m);
/* Copy (host or device) parameters in; resets the Adam state. */
tmr_status tmr_mlp_set_params(tmr_mlp *m, const float *params);
tmr_status tmr_mlp_get_params(tmr_mlp *m, float *params);
/* Y[B][out] = network(X[B][in]). */
tmr_status tmr_mlp_forward(tmr_mlp *m, const float *X, int B, float *Y);
/* Loss of tmr_mlp_grad and tmr_mlp_train_step.  TMR_LOSS_MSE (default):
 * L = sum (Y - T)^2 / (B out).  TMR_LOSS_PHASE (out even): each row is read
 * as a complex vector y = Y[:out/2] + i Y[out/2:] (likewise t from T) and
 * compared with the nearest global-phase rotation of its target,
 * L = sum_b min_a ||y_b - t_b e^{-i a}||^2 / (B out) -- a TM row is only
 * defined up to such a phase, so this is the loss for rows of T.  Its
 * gradient is that of the mean squared error against the aligned targets
 * t_b conj(c_b) / |c_b|, c_b = <y_b, t_b> (unrotated where c_b = 0). */
enum { TMR_LOSS_MSE = 0, TMR_LOSS_PHASE = 1 };
tmr_status tmr_mlp_set_loss(tmr_mlp *m, int kind);
/* The loss of the batch into *loss (may be NULL) and its gradient w.r.t.
 * every parameter into grad (may be NULL). */
tmr_status tmr_mlp_grad(tmr_mlp *m, const float *X, const float *T, int B, float *loss,
                        float *grad);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the batch. */
tmr_status tmr_mlp_train_step(tmr_mlp *m, const float *X, const float *T, int B, float lr,
                              float *loss);
void tmr_mlp_destroy(tmr_mlp *m);

/* The network's BF16 product on the tensor cores (tcgen05.mma, FP32
 * accumulation in tensor memory, TMA-fed): C[M][N] = A B^T with A [M][K] and
 * B [N][K] BF16 (bit patterns in uint16 storage), rows K-contiguous with
 * strides lda, ldb elements; C float32 with row stride ldc >= N.  Device
 * arrays of the current device.  Needs M, N >= 128, K >= 64, K, lda and ldb
 * multiples of 8 and 16-byte aligned A and B (UNSUPPORTED otherwise; the
 * network falls back to its mma.sync kernel there).  Synchronises `stream`;
 * TMR_ERR_TIMEOUT if a barrier wait of the kernel ran out. */
tmr_status tmr_gemm_bf16(int M, int N, int K, const void *A, int lda, const void *B, int ldb, float *C, int ldc,
                         void *stream);

/* Network used by TMR_INIT_LEARNED (not owned; keep it alive while the handle
 * uses it).  Its sizes must be in = J*N and out = 2*N. */
tmr_status tmr_set_init_model(tmr_handle *h, tmr_mlp *model);
/* Rows of the last completed learned-start retrieve whose proposal was used
 * (seeded the power iteration, or won the loss comparison when power_iters
 * is 0); synchronises the handle's stream; -1 when there was none. */
long long tmr_learned_rows(tmr_handle *h);

/* The solver schedule the handle uses (after autotuning): 1, 2 or 4 masks per
 * CTA, 16 for one CTA per row, 32 for the full-length Bluestein plan; 0 for a
 * NULL handle or when no schedule fits (see tmr_create). */
int tmr_schedule(const tmr_handle *h);
/* The schedules the autotuner timed when this handle was made, and the mean
 * time of their timed runs in milliseconds (each: 4 power and 6 L-BFGS
 * iterations on 608 synthetic rows): writes up to cap entries, returns their
 * number (0 when the schedule was given, cached, or the only one). */
int tmr_autotune_report(const tmr_handle *h, int *codes, float *ms, int cap);

/* Release the handle and everything it allocated.  NULL is allowed. */
void tmr_destroy(tmr_handle *h);

/* Per-row retrieval without any allocation and without a handle.
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that must not call cudaMalloc: code running under an allocator that owns
 * the whole device memory budget, loops that cannot afford the device-wide
 * synchronisation a first cudaMalloc may cause, or hosts that forbid device
 * allocation after start-up.  It runs the same persistent solver as
 * tmr_retrieve (initialisation, then `iters` of the same L-BFGS iterations;
 * no phase-offset fit) with the caller's arrays, all of which must be device
 * memory of the current device: masks complex64 [J][N], y float32 [M][J][N],
 * T_out complex64 [M][N], row_status / row_iters int32 [M] and row_loss
 * float32 [M] (each may be NULL).
 * opt: NULL for the defaults; workspace_limit, use_graph, schedule and tune_cache
 * are ignored (one mask per CTA); opt->precision must be TMR_PREC_FP32,
 * opt->probe_n1 0 and opt->lanczos 0 (TMR_ERR_UNSUPPORTED otherwise).
 * stream: cudaStream_t, NULL for the legacy default stream.
 *
 * Its only scratch (a row work counter and the FFT twiddle table) lives in
 * one static 64 KiB device array that every GPU which loads the library holds
 * until the process exits.  Limits: N a power of two in 64..4096, J <= 8,
 * 1 <= opt->m <= 6; larger sizes return TMR_ERR_UNSUPPORTED with a message.
 * It calls no cudaMalloc, cudaFree or other allocating routine.  The first
 * call on a device looks up the array's device address (once per device, with
 * that device current) and keeps it until the process exits; make that first
 * call before any stream capture, and do not use the entry point on a device
 * after a cudaDeviceReset of that device (the array may have moved).
 * Every call on a device shares the array and rewrites it (the counter is
 * cleared, the table refilled), so calls whose work overlaps on the GPU -- on
 * different streams, or from different threads -- race and must be ordered
 * by the caller.  Asynchronous on `stream`; errors via tmr_last_error(). */
tmr_status tmr_retrieve_rows_static(int N, int M, int J, const void *masks, const float *y,
                                    int iters, const tmr_options *opt, void *T_out,
                                    int *row_status, int *row_iters, float *row_loss,
                                    void *stream);

/* ---- Camera preprocessing (Sec. 2.2, the procedure after Algorithm 1) ----
 *
 * Before the per-row solves the paper shrinks the problem in two steps:
 * half-sampling keeps every other pixel of each intensity image in both
 * directions (the kept grid samples the transmitted field at twice the camera
 * pixel size, still enough for the fiber's NA), and a binary fiber mask on
 * the half grid, whose one-region holds 99.9 % of the total intensity,
 * decides which rows are solved; the others are zero.
 *
 * Half grid.  Rows and columns offset, offset + 2, ... of an H x W frame are
 * kept (offset 0 reads the paper's "odd indexes" counted from one; 1 keeps
 * the other phase): ny = (H - offset + 1) / 2, nx = (W - offset + 1) / 2,
 * M = ny * nx, and grid pixel p = a * nx + b is camera pixel
 * (2a + offset, 2b + offset).  This p is the row index of T and y.
 *
 * Energy and mask.  E[p] = sum over the K frames of frame_i(p): exact in
 * 64-bit integers for uint16 frames, FP64 for float32 frames, summed in a
 * fixed order (repeated calls agree bitwise).  With the pixels sorted by E
 * descending, c is the smallest count whose leading energies sum to at least
 * energy_frac * sum(E) (compared in FP64), tau is the c-th largest energy and
 * mask[p] = (E[p] >= tau): ties with the last pixel taken are included.
 * All-dark frames (sum(E) = 0) give an empty mask. */
enum { TMR_PIX_U16 = 0, TMR_PIX_F32 = 1 }; /* frame pixel types */

/* Device scratch tmr_preprocess needs for K frames of H x W at this offset,
 * about 8 * M * (ceil(K / 256) + 1) + M bytes; 0 for invalid sizes. */
size_t tmr_preprocess_workspace_bytes(int K, int H, int W, int offset);

/* Camera frames -> the rows of the retrieval problem.
 *   frames     device, [K][H][W] uint16 (TMR_PIX_U16) or float32 (TMR_PIX_F32),
 *              frame i = probe pattern i = j * N + k (mask-major, as in y);
 *              float32 frames must be non-negative and finite
 *   y          device float32 [M][K] (the layout [M][J][N] of tmr_retrieve):
 *              y[p][i] = frame i at grid pixel p, zero where mask[p] == 0
 *   mask       device uint8 [M] or NULL: 1 inside the fiber mask
 *   energy     device float64 [M] or NULL: E[p]
 *   n_inside   device int32 [1] or NULL: pixels inside the mask; -1 when a
 *              float32 frame set gave a negative or non-finite energy (the
 *              mask is then empty and y all zero)
 *   workspace  device scratch of at least tmr_preprocess_workspace_bytes
 *   stream     cudaStream_t, NULL for the legacy default stream
 * All arrays are the caller's and must be device memory.  Argument errors
 * (sizes, offset not 0/1, energy_frac outside (0, 1], pixel_type, NULL or
 * host pointers, a short workspace, K above 65535 * 256) return
 * TMR_ERR_INVALID_ARG synchronously; otherwise the call is asynchronous on
 * `stream` and allocates nothing. */
tmr_status tmr_preprocess(const void *frames, int pixel_type, int K, int H, int W, int offset,
                          double energy_frac, float *y, unsigned char *mask, double *energy,
                          int *n_inside, void *workspace, size_t workspace_bytes, void *stream);

/* Half-sampling alone: out[i][p] = frame i at grid pixel p, for n frames
 * [n][H][W] (uint16 or float32, device) into device float32 [n][M].  Used for
 * the defocus images, whose layout [n_defocus][M] is already y_def's.  Same
 * argument rules as tmr_preprocess; asynchronous on `stream`. */
tmr_status tmr_half_sample(const void *frames, int pixel_type, int n, int H, int W, int offset,
                           float *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TMR_H */
