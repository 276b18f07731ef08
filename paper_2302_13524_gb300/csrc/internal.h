// internal.h -- launchers shared between the C-ABI layer and the kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>

struct tmr_mlp;

namespace tmr {

// Message returned by tmr_last_error() on this thread (fixed buffer, no heap).
void set_last_error(const char *msg);

// Where a caller array lives: PTR_DEVICE for memory of the current device (or
// managed memory), PTR_OTHER_DEVICE for device memory of another GPU (which a
// kernel of this device must not touch: without peer access it faults),
// PTR_HOST for NULL, host memory and pointers the runtime does not know (the
// lookup error is cleared).
enum { PTR_HOST = 0, PTR_DEVICE = 1, PTR_OTHER_DEVICE = 2 };
int pointer_class(const void *p);
// pointer_class(p) == PTR_DEVICE
bool is_device_ptr(const void *p);

// Twiddle table of the block FFT for length N (FP64 on the host, rounded to
// FP32); returns its length in float2, writes it to out when out != NULL.
int fft_table(int N, float2 *out);
int fft_table_len(int N);
bool fft_supported(int N);  // powers of two 64..4096 (one register FFT)

// Transform constants of length N (xform.cuh): the FFT table for powers of
// two, [twiddles | half Bluestein filter | chirp] for the other lengths.
// xform_supported: powers of two 64..4096 and every other N in 16..4096.
bool xform_supported(int N);
// Bluestein shape of a non-power-of-two N: FFT length L (4096 with split
// outputs for N in (2048, 2731]) and registers per
// thread (the instantiated variant); false when N has none.
bool xform_blue_shape(int N, int *L, int *ne);
int xform_table(int N, float2 *out);  // length in float2; writes when out != NULL
// For 2048 < N <= 2731 the other Bluestein plan: the full convolution at
// L = 8192 (XfBlue<8192, 6>) instead of the split outputs at L = 4096; the
// table of the solver schedule kBlueFullSchedule.
int xform_table_blue_full(int N, float2 *out);
// The 2D probing DFT (N = 512 or 4096, n1 and N / n1 pass boundaries: 8, 64,
// 512): the forward and adjoint twiddle tables and (n1, N/n1); -1 otherwise.
// The kernels take it as transform kind 2 (the `prec` argument below).
int fft_table_2d(int N, int n1, float2 *out);
// Mixed precision (TMR_PREC_MIXED): N = 256, 1024, 2048 or 4096; its table is
// [FP32 twiddles | tensor-core DFT fragments (radix 16, radix 8) | roots W_N^k].
bool mixed_supported(int N);
int xform_table_prec(int N, int prec, float2 *out);

// ---- fused forward model and gradient (kernels.cu) -------------------------
// prec: transform kind: TMR_PREC_FP32 (0, FP32, 1D probing DFT), TMR_PREC_MIXED
// (1, tensor-core transforms) or 2 (FP32, 2D probing DFT, table fft_table_2d)
cudaError_t launch_forward(int N, int M, int J, const float2 *T, const float2 *masks,
                           const float2 *tw, float *Y, cudaStream_t s, int prec = 0);
cudaError_t launch_grad(int N, int M, int J, const float2 *T, const float2 *masks,
                        const float2 *tw, const float *Y, float *loss, float2 *G, cudaStream_t s,
                        int prec = 0, int cost = 0);
// c_n[r] = (Q T[r])[n] for n < Nd, written as Zd[n][r] (the defocus fields).
cudaError_t launch_fields(int N, int M, int J, int Nd, const float2 *T, const float2 *masks,
                          const float2 *tw, float2 *Zd, cudaStream_t s, int prec = 0);
// y (float32 [M][K]) -> y16 (FP16, each row divided by its largest |y|) and the row scales
cudaError_t launch_pack_f16(int M, size_t K, const float *y, void *y16, float *ysc, cudaStream_t s);
// T[r] *= exp(i phi[r])
cudaError_t launch_apply_phase(int N, int M, const double *phi, const float2 *Tin, float2 *Tout,
                               cudaStream_t s);

// ---- persistent per-row solver (solver.cu) ---------------------------------
struct SolverParams {
    const float2 *masks;  // [J][N]
    const float2 *tw;     // transform constants (xform_table)
    const float *y;       // [M][J][N]
    const void *y16;      // [M][J][N] FP16, row-normalised (mixed precision), else unused
    const float *ysc;     // [M] row scales of y16
    const float2 *T_init; // [M][N] or NULL
    float2 *T_out;        // [M][N]
    int *row_status;      // [M]
    int *row_iters;       // [M]
    float *row_loss;      // [M]
    float2 *Zd;           // [Nd][M] defocus fields of the final iterate, or NULL
    const float2 *T_cand; // [M][N] proposed starts (learned initialiser), or NULL
    int seed_from_cand;   // the proposal (when finite, nonzero) replaces the Philox seed
                          //   vector of the random/spectral start
    int judge_cand;       // per row, the proposal replaces the start when its loss is lower
    unsigned *cand_wins;  // rows whose proposed start was kept
    unsigned *queue;      // row work counter, zeroed before the launch
    float2 *pairs;        // one-CTA-per-row schedule: non-null when it may run (its L-BFGS
    int pair_ctas;        //   pairs are in tensor memory); pair_ctas = its resident CTAs
    int lanczos;          // spectral start by power_iters Lanczos steps (else the power iteration)
    int cost;             // COST_INTENSITY (Eq. optTMsmall2) or COST_AMPLITUDE (cost.cuh)
    float2 *krylov;       // Lanczos vectors: krylov_units regions of lanczos_region(N, power_iters)
    int krylov_units;     //   float2, one per CTA (one CTA per row) or cluster; launches use at most that many
    int N, Nd, M, J, iters, m, init, power_iters;
    int prec;             // TMR_PREC_FP32 or TMR_PREC_MIXED
    unsigned long long seed;
    float clip;
    double tol;
};
// Variants: G masks per CTA (G in {1, 2, 4}, G divides J), cluster of J/G CTAs;
// or G = kRowSchedule (16): one CTA per row holding all J masks at 16 points
// per thread, FP32, N = 512 .. 2048 with J N / 16 <= 512, L-BFGS pairs in the
// global workspace p.pairs (solver_row.cuh).
constexpr int kRowSchedule = 16;
// Lanczos steps of the spectral start at most: the 2 k values of a
// Gram-Schmidt reduction fit one warp
constexpr int kMaxLanczos = 16;
// float2 per Lanczos workspace region (one CTA, or one cluster of up to 8
// CTAs): k vectors of length N, then one kMaxLanczos^2 Gram matrix per CTA
__host__ __device__ inline size_t lanczos_region(int N, int k)
{
    return (size_t)k * N + (size_t)8 * kMaxLanczos * kMaxLanczos;
}
// G = kBlueFullSchedule (32): for 2048 < N <= 2731, one mask per CTA with the
// full-length Bluestein plan (L = 8192) and its own transform table.
constexpr int kBlueFullSchedule = 32;
long long solver_dispatch_blue8192(int N, int ne, int what, const SolverParams *p, cudaStream_t s,
                                   int *clusters_out);
// The amplitude cost's solvers (p.cost == 1): one CTA per row (N = 512, 1024,
// 2048), clusters with G = 1, 2, 4 for powers of two, and G = 1 for the
// Bluestein lengths with L <= 4096 (other N: none).
cudaError_t launch_solver_row_amp(int N, const SolverParams &p, cudaStream_t s, int *ctas_out);
cudaError_t launch_solver_amp(int N, int G, const SolverParams &p, cudaStream_t s, int *clusters_out);
bool solver_cost_supported(int N, int G, int prec, int cost);
bool solver_variant_exists(int N, int G, int prec = 0);
// transform kind 3: the matrix-vector DFT (solver_dense.cu, the "without FFT" solver)
long long solver_dispatch_dense(int N, int G, int what, const SolverParams *p, cudaStream_t s, int *clusters_out);
int dense_mv_table(int N, float2 *out);
// schedule G usable for (N, J): variant exists, J % G == 0 for cluster schedules
bool solver_schedule_valid(int N, int J, int G, int prec = 0);
// one-CTA-per-row schedule: CTAs resident at once (the pair regions a launch needs)
int solver_row_max_ctas(int N, int J, int m);
size_t solver_row_pair_stride(int N, int m);  // float2 per CTA region
size_t solver_smem_bytes(int N, int J, int m, int G, int prec = 0);
cudaError_t launch_solver(int N, int G, const SolverParams &p, cudaStream_t s, int *clusters_out);
// the Bluestein variants (solver_bs.cu); what == 0: shared bytes, 1: launch
long long solver_dispatch_blue(int N, int G, int what, const SolverParams *p, cudaStream_t s, int *clusters_out);
// the one-CTA-per-row variants (solver_row.cu)
long long solver_dispatch_row(int N, int what, const SolverParams *p, cudaStream_t s, int *ctas_out);
// the 2D-probing-DFT variants (solver_2d.cu)
long long solver_dispatch_2d(int N, int G, int what, const SolverParams *p, cudaStream_t s, int *clusters_out);
// the mixed-precision variants (solver_mx.cu)
long long solver_dispatch_mixed(int N, int G, int what, const SolverParams *p, cudaStream_t s, int *clusters_out);
// Synthetic positive intensities for timing runs (autotuner).
cudaError_t launch_fill_synthetic(float *y, size_t n, unsigned seed, cudaStream_t s);

// ---- BF16 tensor-core GEMM (gemm_tc.cu) ---------------------------------------
// C[M][N] (FP32, row stride ldc) = A B^T with A [M][K], B [N][K] BF16, K-contiguous
// rows of stride lda, ldb.  Needs M, N >= 128, K >= 64, K, lda, ldb multiples of 8
// and 16-byte aligned A, B; *err (device) is raised when a barrier wait ran out.
bool gemm_tc_supported(int M, int N, int K, const void *A, int lda, const void *B, int ldb);
cudaError_t gemm_tc(int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb,
                    float *C, int ldc, int *err, cudaStream_t s);

// ---- learned initialiser (mlp.cu) --------------------------------------------
// rows of y (B of them) -> features -> network -> starts T scaled to the
// Parseval norm
cudaError_t mlp_propose(tmr_mlp *m, const float *y, int B, int N, int J, float2 *T, cudaStream_t s);
int mlp_in(const tmr_mlp *m);
int mlp_out(const tmr_mlp *m);

// ---- defocus operator and phase-offset fit (defocus.cu) --------------------
struct PhaseFitParams {
    const float2 *Zd;    // [Nd][P] fields c_n (P = ny*nx = M)
    const float *Ydef;   // [Nd][P]
    const float2 *H;     // [P] transfer function
    const float2 *twy;   // FFT table for ny
    const float2 *twx;   // FFT table for nx
    const float *wts;    // [P] weights of the constant-phase normalisation
    double *phi;         // [P] out
    int Nd, ny, nx, iters, m;
    // workspace (allocated by the caller, see phase_fit_workspace)
    double *ws;
    unsigned *sync;      // grid barrier words (2), zeroed before the launch
    int *err;            // error flag, zeroed before the launch
    int *iters_done;     // [1]
    double *loss_out;    // [1]
    long long wait_spins;   // polls before a grid-barrier wait gives up
    bool withhold_release;  // test hook: the barrier is never released
    int kind;               // 0: same-grid operator; 1: angular spectrum with 2x padding (Ydef [Nd][4P])
    double tol;             // > 0: stop after an accepted step lowering g by at most tol g
};
size_t phase_fit_workspace_doubles(int P, int Nd, int m, int grid);
int phase_fit_grid(int ny, int nx, int Nd);
// The probing operator as an explicit dense matrix (dense.cu, the paper's
// "without FFT" evaluation): Q [J N][N] and cuBLAS, made on first use.
// mode 1: FP32 complex products; 2: FP32 emulated on the tensor cores (BF16x9).
struct DenseState {
    void *blas = nullptr;  // cublasHandle_t
    float2 *Q = nullptr, *Z = nullptr, *C = nullptr;
    ~DenseState();
    void release();
};
cudaError_t dense_prepare(DenseState &ds, int N, int M, int J, const float2 *masks, cudaStream_t s,
                          size_t *bytes_out);
cudaError_t dense_forward(DenseState &ds, int mode, int N, int M, int J, const float2 *T, float *Y, cudaStream_t s);
cudaError_t dense_grad(DenseState &ds, int mode, int N, int M, int J, const float2 *T, const float *y, float *loss,
                       float2 *G, int cost, cudaStream_t s);
bool defocus_supported(int ny, int nx);
bool defocus2x_supported(int ny, int nx);
cudaError_t launch_make_H2x(int ny, int nx, double wavelength, double na, double zd, double pixel, float2 *H,
                            cudaStream_t s);
cudaError_t launch_incident_fields(int M, int N, int Nd, const float2 *T, const float2 *inc, float2 *Zd,
                                   cudaStream_t s);
cudaError_t launch_defocus_forward2x(int ny, int nx, int Nd, const float2 *Zd, const float2 *H, float *Ydef,
                                     cudaStream_t s);
cudaError_t launch_phase_fit(const PhaseFitParams &p, cudaStream_t s);
cudaError_t launch_defocus_forward(int ny, int nx, int Nd, const float2 *Zd, const float2 *H,
                                   const float2 *twy, const float2 *twx, float *Ydef,
                                   cudaStream_t s);
cudaError_t launch_make_quadratic_H(int ny, int nx, double coef, float2 *H, cudaStream_t s);
cudaError_t launch_row_energy(int N, int M, const float2 *T, float *w, cudaStream_t s);

}  // namespace tmr
