/*
 * oracle.c -- plain, slow, FP64 CPU oracle for reference-less transmission-matrix
 * (TM) retrieval with FFT-structured probing (arXiv 2302.13524).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * load it.  It shares no code with the CUDA library.
 *
 * Every transform here is the textbook definition evaluated directly:
 *   - the DFT is the O(N^2) sum with an exact (k*n mod N) index into an FP64
 *     twiddle table made by libm cos/sin;
 *   - the probing operator Q = [F D_1; ...; F D_J] (Eq. probingmatrix, Sec. 2.2)
 *     is applied mask by mask, never stored as a matrix;
 *   - the loss and gradient are Eq. optTMsmall2 and Eq. derivative (App. A);
 *   - the per-row solver follows Algorithm 1 with L-BFGS (two-loop recursion,
 *     Nocedal & Wright Alg. 7.4) and an exact line search on the quartic
 *     f(t + alpha p);
 *   - the defocus phase-offset fit follows Eq. phaseoffset, Eq. optphase and
 *     Eq. phasederive (App. B) with L-BFGS and Armijo backtracking.
 *
 * Conventions (binding for both implementations):
 *   DFT      F x[k] = sum_n x[n] exp(-2 pi i k n / N)   (unnormalised)
 *   probing  z[j*N + k] = (F (d_j .* t))[k],  pattern index i = j*N + k
 *   adjoint  (Q^H v)[n] = sum_j conj(d_j[n]) sum_k exp(+2 pi i k n / N) v[j*N+k]
 *   complex arrays are interleaved (re, im) doubles, row-major.
 *
 * Row status codes: 0 = ran all iterations, 1 = converged early (tolerance met,
 * zero loss or zero gradient), 2 = all-zero row (t = 0, no iteration),
 * 3 = non-finite input or iterate.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef double complex cplx;

/* |x|^2 */
static double abs2(cplx x) { return creal(x) * creal(x) + cimag(x) * cimag(x); }

enum { ROW_MAXITER = 0, ROW_CONVERGED = 1, ROW_ZERO = 2, ROW_NUMERIC = 3 };
enum { INIT_RANDOM = 0, INIT_BP = 1, INIT_SPECTRAL = 2, INIT_GIVEN = 3, INIT_LANCZOS = 4 };

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* DFT                                                                       */
/* ------------------------------------------------------------------------ */

/* tw[m] = exp(-2 pi i m / N), m = 0..N-1, from libm in FP64. */
static cplx *make_twiddles(int N)
{
    cplx *tw = malloc(sizeof(cplx) * (size_t)N);
    for (int m = 0; m < N; m++) {
        double a = 2.0 * M_PI * (double)m / (double)N;
        tw[m] = cos(a) - I * sin(a);
    }
    return tw;
}

/* X[k] = sum_n x[n] exp(sign * 2 pi i k n / N), sign = -1 (forward) or +1
 * (backward, no 1/N).  Direct O(N^2) sum; the twiddle of (k, n) is
 * tw[(k*n) mod N], the index advanced exactly in integers. */
static void dft_naive(const cplx *x, cplx *X, int N, int sign, const cplx *tw)
{
    for (int k = 0; k < N; k++) {
        cplx acc = 0;
        long idx = 0; /* (k * n) mod N */
        for (int n = 0; n < N; n++) {
            cplx w = sign < 0 ? tw[idx] : conj(tw[idx]);
            acc += x[n] * w;
            idx += k;
            if (idx >= N) idx -= N;
        }
        X[k] = acc;
    }
}

int orc_dft(const double *x, double *X, int N, int sign)
{
    if (N <= 0) return -1;
    cplx *tw = make_twiddles(N);
    dft_naive((const cplx *)x, (cplx *)X, N, sign, tw);
    free(tw);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Probing operator Q and its adjoint (Eq. probingmatrix, Eq. optTMsmall2)    */
/* ------------------------------------------------------------------------ */

/* The probing DFT K (Eq. probingmatrix): the 1D DFT of length N (default),
 * or, after orc_set_probe_2d(n1, N), the 2D DFT of the vector read as an
 * n1 x n2 array (n2 = N / n1; element a*n2 + b is row a, column b) -- the
 * paper's "2D Fourier transform matrix for an N_kx x 2N_ky matrix".  The 2D
 * spectrum X[k1][k2] is stored at pattern index k1 + n1*k2 (column by
 * column).  A process-wide setting of this test oracle (read-only while a
 * computation runs). */
static int g_probe_n1 = 0, g_probe_N = 0;
static cplx *g_tw1 = NULL, *g_tw2 = NULL;

int orc_set_probe_2d(int n1, int N)
{
    free(g_tw1);
    free(g_tw2);
    g_tw1 = g_tw2 = NULL;
    g_probe_n1 = g_probe_N = 0;
    if (n1 == 0) return 0;
    if (n1 < 1 || N <= 0 || N % n1) return -1;
    g_probe_n1 = n1;
    g_probe_N = N;
    g_tw1 = make_twiddles(n1);
    g_tw2 = make_twiddles(N / n1);
    return 0;
}

/* Z[k1 + n1 k2] = sum_{a, b} s[a n2 + b] W_n1^(a k1 sign) W_n2^(b k2 sign) (forward
 * layout), or, for the adjoint layout, out[a n2 + b] = the same double sum of
 * V[k1 + n1 k2] with the conjugate kernel.  Separable: the n2-point sums along
 * each row, then the n1-point sums along each column.  scratch: 2 N entries. */
static void dft2_probe(const cplx *in, cplx *out, int N, int sign, int adjoint_layout, cplx *scratch)
{
    const int n1 = g_probe_n1, n2 = N / n1;
    cplx *A = scratch, *col = scratch + N;  /* A[a][k2] (or A[k1][b]) */
    if (!adjoint_layout) {
        for (int a = 0; a < n1; a++) dft_naive(in + (size_t)a * n2, A + (size_t)a * n2, n2, sign, g_tw2);
        for (int k2 = 0; k2 < n2; k2++) {
            for (int a = 0; a < n1; a++) col[a] = A[(size_t)a * n2 + k2];
            dft_naive(col, out + (size_t)n1 * k2, n1, sign, g_tw1);  /* out[k1 + n1 k2] */
        }
    } else {
        /* in[k1 + n1 k2]: the n1-point sums over k1 for each k2 give A2[a][k2]
           (held as A[k2 * n1 + a]), then the n2-point sums over k2 for each a */
        for (int k2 = 0; k2 < n2; k2++) dft_naive(in + (size_t)n1 * k2, A + (size_t)n1 * k2, n1, sign, g_tw1);
        for (int a = 0; a < n1; a++) {
            for (int k2 = 0; k2 < n2; k2++) col[k2] = A[(size_t)n1 * k2 + a];
            dft_naive(col, out + (size_t)a * n2, n2, sign, g_tw2);
        }
    }
}

/* z = Q t : z[j*N + k] = K(d_j .* t)[k].  scratch: 3 N entries. */
static void apply_Q(const cplx *t, const cplx *d, int N, int J, const cplx *tw,
                    cplx *z, cplx *scratch)
{
    for (int j = 0; j < J; j++) {
        for (int n = 0; n < N; n++) scratch[n] = d[(size_t)j * N + n] * t[n];
        if (g_probe_n1 && g_probe_N == N) dft2_probe(scratch, z + (size_t)j * N, N, -1, 0, scratch + N);
        else dft_naive(scratch, z + (size_t)j * N, N, -1, tw);
    }
}

/* out = Q^H v : out[n] = sum_j conj(d_j[n]) * (K^H v_j)[n].  scratch: 3 N entries. */
static void apply_QH(const cplx *v, const cplx *d, int N, int J, const cplx *tw,
                     cplx *out, cplx *scratch)
{
    for (int n = 0; n < N; n++) out[n] = 0;
    for (int j = 0; j < J; j++) {
        if (g_probe_n1 && g_probe_N == N) dft2_probe(v + (size_t)j * N, scratch, N, +1, 1, scratch + N);
        else dft_naive(v + (size_t)j * N, scratch, N, +1, tw);
        for (int n = 0; n < N; n++) out[n] += conj(d[(size_t)j * N + n]) * scratch[n];
    }
}

/* Forward model, Eq. forwardmodel restricted to one pixel (Eq. optTMsmall2):
 * Y[row][i] = |(Q t_row)[i]|^2, optionally also Z = Q t. */
int orc_forward(const double *T, const double *masks, int M, int N, int J,
                double *Z, double *Y)
{
    if (M < 0 || N <= 0 || J <= 0) return -1;
    const cplx *Tc = (const cplx *)T, *d = (const cplx *)masks;
    cplx *tw = make_twiddles(N);
    size_t K = (size_t)J * N;
#pragma omp parallel
    {
        cplx *z = malloc(sizeof(cplx) * K), *sc = malloc(sizeof(cplx) * 3 * (size_t)N);
#pragma omp for schedule(dynamic)
        for (int r = 0; r < M; r++) {
            apply_Q(Tc + (size_t)r * N, d, N, J, tw, z, sc);
            for (size_t i = 0; i < K; i++) Y[(size_t)r * K + i] = abs2(z[i]);
            if (Z) memcpy((cplx *)Z + (size_t)r * K, z, sizeof(cplx) * K);
        }
        free(z);
        free(sc);
    }
    free(tw);
    return 0;
}

/* Row-batched adjoint: out[row] = Q^H V[row]. */
int orc_adjoint(const double *V, const double *masks, int M, int N, int J, double *out)
{
    if (M < 0 || N <= 0 || J <= 0) return -1;
    const cplx *d = (const cplx *)masks;
    cplx *tw = make_twiddles(N);
    size_t K = (size_t)J * N;
#pragma omp parallel
    {
        cplx *sc = malloc(sizeof(cplx) * 3 * (size_t)N);
#pragma omp for schedule(dynamic)
        for (int r = 0; r < M; r++)
            apply_QH((const cplx *)V + (size_t)r * K, d, N, J, tw, (cplx *)out + (size_t)r * N, sc);
        free(sc);
    }
    free(tw);
    return 0;
}

/* Loss and gradient of one row.
 *   f(t) = || y - |Q t|^2 ||^2                           (Eq. optTMsmall2)
 *   g    = (df/dt)^H = -4 Q^H diag(Q t)(y - |Q t|^2)      (Eq. derivative)
 * with g packed as df/dRe(t) + i df/dIm(t).  Work: z, rz (K each), sc (N). */
/* Cost of the per-row problem.  Intensity (Eq. optTMsmall2, the paper's):
 * f = sum_i (y_i - |z_i|^2)^2, real gradient g = -4 Q^H (z .* r), r = y - |z|^2
 * (Eq. derivative).  Amplitude (the Discussion's alternative for Poisson noise,
 * after Yeh et al. 2015), after orc_set_cost(1): f = sum_i (a_i - |z_i|)^2 with
 * a = sqrt(y), real gradient g = 2 Q^H ((|z| - a) z / |z|), the term taken as 0
 * where z_i = 0.  (Real gradient: d f / d Re t + i d f / d Im t.)  A
 * process-wide setting of this test oracle, like the probing DFT's. */
static int g_cost = 0;

int orc_set_cost(int cost)
{
    if (cost != 0 && cost != 1) return -1;
    g_cost = cost;
    return 0;
}

static double loss_grad_row(const cplx *t, const double *y, const cplx *d, int N, int J,
                            const cplx *tw, cplx *g, cplx *z, cplx *rz, cplx *sc)
{
    size_t K = (size_t)J * N;
    apply_Q(t, d, N, J, tw, z, sc);
    double f = 0;
    for (size_t i = 0; i < K; i++) {
        if (g_cost == 1) {
            double a = sqrt(y[i] > 0 ? y[i] : 0.0), m = cabs(z[i]);
            f += (a - m) * (a - m);
            rz[i] = m > 0 ? z[i] * ((m - a) / m) : 0;
        } else {
            double r = y[i] - abs2(z[i]);
            f += r * r;
            rz[i] = z[i] * r;
        }
    }
    if (g) {
        apply_QH(rz, d, N, J, tw, g, sc);
        for (int n = 0; n < N; n++) g[n] *= g_cost == 1 ? 2.0 : -4.0;
    }
    return f;
}

int orc_loss_grad(const double *T, const double *masks, const double *Y, int M, int N, int J,
                  double *loss, double *G)
{
    if (M < 0 || N <= 0 || J <= 0) return -1;
    const cplx *d = (const cplx *)masks;
    cplx *tw = make_twiddles(N);
    size_t K = (size_t)J * N;
#pragma omp parallel
    {
        cplx *z = malloc(sizeof(cplx) * K), *rz = malloc(sizeof(cplx) * K);
        cplx *sc = malloc(sizeof(cplx) * 3 * (size_t)N);
#pragma omp for schedule(dynamic)
        for (int r = 0; r < M; r++) {
            double f = loss_grad_row((const cplx *)T + (size_t)r * N, Y + (size_t)r * K, d, N, J, tw,
                                     G ? (cplx *)G + (size_t)r * N : NULL, z, rz, sc);
            if (loss) loss[r] = f;
        }
        free(z);
        free(rz);
        free(sc);
    }
    free(tw);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)                         */
/* ------------------------------------------------------------------------ */

/* One application of the 10-round Philox4x32 bijection to counter c under key k:
 * each round multiplies words 0 and 2 by the round multipliers, XORs the high
 * halves with words 1/3 and the key, and the key is bumped by the Weyl
 * constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Standard complex normal draw for element n of row `row`:
 * counter (n, row, 0, 0), key (seed lo, seed hi); words 0 and 1 become
 * uniforms u = (x + 1/2) 2^-32 in (0,1); Box-Muller gives
 * rho = sqrt(-2 ln u0), value = rho (cos 2 pi u1 + i sin 2 pi u1). */
static cplx philox_cnormal(uint64_t seed, uint32_t row, uint32_t n)
{
    uint32_t c[4] = {n, row, 0u, 0u}, k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)}, o[4];
    orc_philox4x32_10(c, k, o);
    double u0 = ((double)o[0] + 0.5) * 0x1p-32;
    double u1 = ((double)o[1] + 0.5) * 0x1p-32;
    double rho = sqrt(-2.0 * log(u0));
    return rho * cos(2.0 * M_PI * u1) + I * rho * sin(2.0 * M_PI * u1);
}

int orc_random_cnormal(uint64_t seed, int row, int N, double *out)
{
    for (int n = 0; n < N; n++) ((cplx *)out)[n] = philox_cnormal(seed, (uint32_t)row, (uint32_t)n);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Initialisation                                                            */
/* ------------------------------------------------------------------------ */

static double norm2(const cplx *x, int n)
{
    double s = 0;
    for (int i = 0; i < n; i++) s += creal(x[i]) * creal(x[i]) + cimag(x[i]) * cimag(x[i]);
    return s;
}

/* Real inner product <a, b> = Re(a^H b) on C^n viewed as R^(2n). */
static double rdot(const cplx *a, const cplx *b, int n)
{
    double s = 0;
    for (int i = 0; i < n; i++) s += creal(a[i]) * creal(b[i]) + cimag(a[i]) * cimag(b[i]);
    return s;
}

/* Eigenvalues and eigenvectors of a symmetric n x n matrix by the cyclic
 * Jacobi method (rotations that zero one off-diagonal entry at a time, swept
 * until the off-diagonal part vanishes).  A (row-major) is overwritten; on
 * return ev[i] = A[i][i] and column i of V is its eigenvector. */
static void jacobi_eig(int n, double *A, double *V, double *ev)
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) V[i * n + j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0, dia = 0;
        for (int p = 0; p < n; p++) {
            dia += A[p * n + p] * A[p * n + p];
            for (int q = p + 1; q < n; q++) off += A[p * n + q] * A[p * n + q];
        }
        if (off <= 1e-32 * dia || off == 0) break;
        for (int p = 0; p < n; p++)
            for (int q = p + 1; q < n; q++) {
                double apq = A[p * n + q];
                if (apq == 0) continue;
                /* J = [[c, s], [-s, c]] in the (p, q) plane; A <- J^T A J with
                 * t = s / c the smaller root of t^2 + 2 theta t - 1 = 0 */
                double theta = (A[q * n + q] - A[p * n + p]) / (2 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1));
                double c = 1 / sqrt(t * t + 1), s = t * c;
                for (int k = 0; k < n; k++) {
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; k++) {
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; k++) {
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < n; i++) ev[i] = A[i * n + i];
}

/* The leading eigenvector of A = Q^H diag(tau) Q / (J N) by the Lanczos method
 * (the spectral start's eigenvector in fewer products than the power
 * iteration; not in the paper).  From v_0 = t / ||t||, step j forms
 * w = A v_j, orthogonalises w against v_0 .. v_j by two passes of classical
 * Gram-Schmidt (coefficients h_l = <v_l, w>, w <- w - sum_l h_l v_l), takes
 * alpha_j = the real part of v_j's two coefficients and beta_j = ||w||, and
 * stops after k steps or when beta_j <= 1e-6 alpha_0 (an invariant subspace);
 * else v_{j+1} = w / beta_j.  The tridiagonal T (alpha on the diagonal, beta
 * beside it) is diagonalised, and t <- sum_l s_l v_l with s the eigenvector of
 * its largest eigenvalue, signed so that s_0 >= 0.  Work: z (K), sc (3N). */
static void lanczos_row(const double *tau, const cplx *d, int N, int J, const cplx *tw, int k,
                        cplx *t, cplx *z, cplx *sc)
{
    size_t K = (size_t)J * N;
    cplx *V = malloc(sizeof(cplx) * (size_t)k * N), *w = malloc(sizeof(cplx) * (size_t)N);
    cplx *h = malloc(sizeof(cplx) * (size_t)k);
    double *al = calloc((size_t)k, sizeof(double)), *be = calloc((size_t)k, sizeof(double));
    double nt = sqrt(norm2(t, N));
    for (int n = 0; n < N; n++) V[n] = nt > 0 ? t[n] / nt : 0;
    int kk = k;
    for (int j = 0; j < k; j++) {
        cplx *vj = V + (size_t)j * N;
        apply_Q(vj, d, N, J, tw, z, sc);
        for (size_t i = 0; i < K; i++) z[i] *= tau[i];
        apply_QH(z, d, N, J, tw, w, sc);
        for (int n = 0; n < N; n++) w[n] /= (double)J * N;
        al[j] = 0;
        for (int pass = 0; pass < 2; pass++) {
            for (int l = 0; l <= j; l++) {
                cplx s = 0;
                for (int n = 0; n < N; n++) s += conj(V[(size_t)l * N + n]) * w[n];
                h[l] = s;
            }
            for (int l = 0; l <= j; l++)
                for (int n = 0; n < N; n++) w[n] -= h[l] * V[(size_t)l * N + n];
            al[j] += creal(h[j]);
        }
        be[j] = sqrt(norm2(w, N));
        if (j == k - 1 || !(be[j] > 1e-6 * al[0])) {
            kk = j + 1;
            break;
        }
        for (int n = 0; n < N; n++) V[(size_t)(j + 1) * N + n] = w[n] / be[j];
    }
    double *Tm = calloc((size_t)kk * kk, sizeof(double)), *E = malloc(sizeof(double) * kk * kk);
    double *ev = malloc(sizeof(double) * kk);
    for (int j = 0; j < kk; j++) {
        Tm[j * kk + j] = al[j];
        if (j + 1 < kk) Tm[j * kk + j + 1] = Tm[(j + 1) * kk + j] = be[j];
    }
    jacobi_eig(kk, Tm, E, ev);
    int top = 0;
    for (int j = 1; j < kk; j++)
        if (ev[j] > ev[top]) top = j;
    double sg = E[0 * kk + top] < 0 ? -1.0 : 1.0;
    for (int n = 0; n < N; n++) {
        cplx s = 0;
        for (int l = 0; l < kk; l++) s += sg * E[l * kk + top] * V[(size_t)l * N + n];
        t[n] = s;
    }
    free(V); free(w); free(h); free(al); free(be); free(Tm); free(E); free(ev);
}

/* t0 for one row.
 *  random   : Philox complex normal, rescaled to the Parseval norm
 *             ||t||^2 = sum(y) / (J N)  (Q^H Q = J N I for unit-modulus masks).
 *  bp       : t0 = (Q^H Q)^-1 Q^H sqrt(y) = Q^H sqrt(y) / (J N), the first line
 *             of Eq. backpropagation with the unnormalised DFT.
 *  spectral : `power_iters` power iterations t <- A t / ||A t|| on
 *             A = Q^H diag(tau) Q / (J N), tau_i = min(y_i / mean(y), clip)
 *             (clip <= 0: tau = y / mean(y)), started from the random vector,
 *             then rescaled to the Parseval norm.
 *  lanczos  : the same eigenvector by `power_iters` Lanczos steps from the
 *             random vector (lanczos_row), then rescaled to the Parseval norm.
 * Work: z (K), sc (N). */
static void init_row(const double *y, const cplx *d, int N, int J, const cplx *tw, int init,
                     uint64_t seed, int row, int power_iters, double clip, cplx *t, cplx *z,
                     cplx *sc)
{
    size_t K = (size_t)J * N;
    double sy = 0;
    for (size_t i = 0; i < K; i++) sy += y[i];
    double target = sqrt(sy / ((double)J * N));
    if (init == INIT_BP) {
        for (size_t i = 0; i < K; i++) z[i] = sqrt(y[i]);
        apply_QH(z, d, N, J, tw, t, sc);
        for (int n = 0; n < N; n++) t[n] /= (double)J * N;
        return;
    }
    for (int n = 0; n < N; n++) t[n] = philox_cnormal(seed, (uint32_t)row, (uint32_t)n);
    if (init == INIT_LANCZOS && power_iters > 0) {
        double mean = sy / (double)K;
        double *tau = malloc(sizeof(double) * K);
        for (size_t i = 0; i < K; i++) {
            tau[i] = mean > 0 ? y[i] / mean : 0.0;
            if (clip > 0 && tau[i] > clip) tau[i] = clip;
        }
        lanczos_row(tau, d, N, J, tw, power_iters, t, z, sc);
        free(tau);
    }
    if (init == INIT_SPECTRAL) {
        double mean = sy / (double)K;
        for (int it = 0; it < power_iters; it++) {
            apply_Q(t, d, N, J, tw, z, sc);
            for (size_t i = 0; i < K; i++) {
                double tau = mean > 0 ? y[i] / mean : 0.0;
                if (clip > 0 && tau > clip) tau = clip;
                z[i] *= tau;
            }
            apply_QH(z, d, N, J, tw, t, sc);
            for (int n = 0; n < N; n++) t[n] /= (double)J * N;
            double nt = sqrt(norm2(t, N));
            if (nt > 0)
                for (int n = 0; n < N; n++) t[n] /= nt;
        }
    }
    double nt = sqrt(norm2(t, N));
    for (int n = 0; n < N; n++) t[n] = nt > 0 ? t[n] * (target / nt) : 0;
}

/* Batched init; row_ids gives the global row index of each row (Philox counter),
 * NULL meaning 0..M-1. */
int orc_init(const double *Y, const double *masks, int M, int N, int J, const int *row_ids,
             int init, uint64_t seed, int power_iters, double clip, double *T0)
{
    if (M < 0 || N <= 0 || J <= 0) return -1;
    const cplx *d = (const cplx *)masks;
    cplx *tw = make_twiddles(N);
    size_t K = (size_t)J * N;
#pragma omp parallel
    {
        cplx *z = malloc(sizeof(cplx) * K), *sc = malloc(sizeof(cplx) * 3 * (size_t)N);
#pragma omp for schedule(dynamic)
        for (int r = 0; r < M; r++)
            init_row(Y + (size_t)r * K, d, N, J, tw, init, seed, row_ids ? row_ids[r] : r,
                     power_iters, clip, (cplx *)T0 + (size_t)r * N, z, sc);
        free(z);
        free(sc);
    }
    free(tw);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exact line search on the quartic                                          */
/* ------------------------------------------------------------------------ */

/* phi(alpha) = f(t + alpha p) = sum_i (r_i - 2 alpha a_i - alpha^2 b_i)^2
 *            = c0 + c1 a + c2 a^2 + c3 a^3 + c4 a^4
 * with a_i = Re(conj(z_i) w_i), b_i = |w_i|^2, w = Q p.  Returns the global
 * minimiser over the real line, taken among the real roots of phi'(alpha)
 * (a cubic); ties go to the smallest positive root.  c4 = sum b^2 >= 0; c4 == 0
 * means w == 0 and gives alpha = 0. */
static double quartic_val(const double c[5], double a)
{
    return (((c[4] * a + c[3]) * a + c[2]) * a + c[1]) * a + c[0];
}

static double cubic_newton(const double c[5], double x)
{
    for (int it = 0; it < 3; it++) {
        double f1 = ((4 * c[4] * x + 3 * c[3]) * x + 2 * c[2]) * x + c[1];
        double f2 = (12 * c[4] * x + 6 * c[3]) * x + 2 * c[2];
        if (f2 == 0) break;
        double nx = x - f1 / f2;
        if (!isfinite(nx)) break;
        x = nx;
    }
    return x;
}

double orc_quartic_argmin(const double c[5])
{
    if (!(c[4] > 0)) {
        if (c[2] > 0 && c[3] == 0) return -c[1] / (2 * c[2]);
        return 0.0;
    }
    /* phi'(a)/(4 c4) = a^3 + B a^2 + C a + D */
    double B = 3 * c[3] / (4 * c[4]), C = 2 * c[2] / (4 * c[4]), D = c[1] / (4 * c[4]);
    /* depressed: a = x - B/3, x^3 + p x + q = 0 */
    double p = C - B * B / 3.0;
    double q = 2 * B * B * B / 27.0 - B * C / 3.0 + D;
    double roots[3];
    int nr = 0;
    double disc = q * q / 4.0 + p * p * p / 27.0;
    if (disc > 0) {
        double sq = sqrt(disc);
        double u = cbrt(-q / 2.0 + (q > 0 ? -sq : sq));
        double x = (u != 0) ? u - p / (3.0 * u) : 0.0;
        roots[nr++] = x - B / 3.0;
    } else if (p == 0) {
        roots[nr++] = -B / 3.0;
    } else {
        double m = 2.0 * sqrt(-p / 3.0);
        double arg = 3.0 * q / (p * m);
        if (arg > 1) arg = 1;
        if (arg < -1) arg = -1;
        double th = acos(arg) / 3.0;
        for (int k = 0; k < 3; k++) roots[nr++] = m * cos(th - 2.0 * M_PI * k / 3.0) - B / 3.0;
    }
    double best = 0, bestv = INFINITY;
    int have = 0;
    for (int k = 0; k < nr; k++) {
        double a = cubic_newton(c, roots[k]);
        double v = quartic_val(c, a);
        if (!have || v < bestv || (v == bestv && a > 0 && (best <= 0 || a < best))) {
            best = a;
            bestv = v;
            have = 1;
        }
    }
    return best;
}

/* The five coefficients of phi(alpha) from r, z, w (length K). */
/* Line search of the amplitude cost along t + alpha p (fields z + alpha w,
 * w = Q p): phi(alpha) = sum_i (a_i - |u_i|)^2 with u = z + alpha w, m = |u|.
 * Half its derivatives: phi'/2 = sum (m - a) Re(conj(u) w) / m and
 * phi''/2 = sum |w|^2 - a Im(conj(u) w)^2 / m^3 (a term with m = 0 adds |w|^2
 * to the second and nothing to the first, as in the gradient).  phi is not a
 * polynomial, so the step is the root of phi' found in two stages:
 *   bracket: alpha = 1, 2, 4, ... (at most 40 doublings) until phi' >= 0,
 *     the lower end the last point with phi' < 0 (alpha = 0 at first: p is a
 *     descent direction); if phi' stays negative, the farthest point tried;
 *   root: Newton steps from the lower end kept inside the bracket (the
 *     midpoint when a step would leave it or phi'' <= 0), the bracket shrunk
 *     by the sign of phi' at every point, until a step is below tol alpha.
 * The oracle stops at tol = 1e-13 (at most 200 steps). */
static void amp_derivs(const cplx *z, const cplx *w, const double *y, size_t K, double al, double *d1,
                       double *d2)
{
    double s1 = 0, s2 = 0;
    for (size_t i = 0; i < K; i++) {
        double a = sqrt(y[i] > 0 ? y[i] : 0.0);
        cplx u = z[i] + al * w[i], cw = conj(u) * w[i];
        double m = cabs(u);
        s2 += abs2(w[i]);
        if (m > 0) {
            s1 += (m - a) * creal(cw) / m;
            s2 -= a * cimag(cw) * cimag(cw) / (m * m * m);
        }
    }
    *d1 = s1;
    *d2 = s2;
}

double orc_amp_step(const double *zr, const double *wr, const double *y, size_t K)
{
    const cplx *z = (const cplx *)zr, *w = (const cplx *)wr;
    double lo = 0, hi = 0, d1lo, d2lo, d1, d2, al = 1;
    amp_derivs(z, w, y, K, 0.0, &d1lo, &d2lo);
    int bracketed = 0;
    for (int k = 0; k <= 40; k++) {
        amp_derivs(z, w, y, K, al, &d1, &d2);
        if (!(d1 < 0)) {
            hi = al;
            bracketed = 1;
            break;
        }
        lo = al;
        d1lo = d1;
        d2lo = d2;
        al *= 2;
    }
    if (!bracketed) return lo;
    double x = d2lo > 0 ? lo - d1lo / d2lo : NAN;
    if (!(x > lo && x < hi)) x = 0.5 * (lo + hi);
    for (int it = 0; it < 200; it++) {
        amp_derivs(z, w, y, K, x, &d1, &d2);
        if (d1 == 0) return x;
        if (d1 < 0) lo = x;
        else hi = x;
        double xn = d2 > 0 ? x - d1 / d2 : NAN;
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        if (fabs(xn - x) <= 1e-13 * x) return xn;
        x = xn;
    }
    return x;
}

static void quartic_coeffs(const double *r, const cplx *z, const cplx *w, size_t K, double c[5])
{
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0;
    for (size_t i = 0; i < K; i++) {
        double a = creal(z[i]) * creal(w[i]) + cimag(z[i]) * cimag(w[i]);
        double b = creal(w[i]) * creal(w[i]) + cimag(w[i]) * cimag(w[i]);
        s0 += r[i] * r[i];
        s1 += -4.0 * r[i] * a;
        s2 += 4.0 * a * a - 2.0 * r[i] * b;
        s3 += 4.0 * a * b;
        s4 += b * b;
    }
    c[0] = s0;
    c[1] = s1;
    c[2] = s2;
    c[3] = s3;
    c[4] = s4;
}

/* ------------------------------------------------------------------------ */
/* L-BFGS two-loop recursion (Nocedal & Wright, Algorithm 7.4)               */
/* ------------------------------------------------------------------------ */

/* p = -H g for vectors in R^n.  S and Yh hold `np` pairs, oldest first
 * (pair i at S + i*n).  H0 = gamma I with gamma = s^T y / y^T y of the newest
 * pair (gamma = 1 with no pairs).  q: scratch of n, alpha: scratch of np. */
static void two_loop(int n, const double *g, const double *S, const double *Yh, int np, double *p,
                     double *alpha)
{
    for (int i = 0; i < n; i++) p[i] = g[i];
    for (int k = np - 1; k >= 0; k--) {
        const double *s = S + (size_t)k * n, *y = Yh + (size_t)k * n;
        double sy = 0, sq = 0;
        for (int i = 0; i < n; i++) {
            sy += s[i] * y[i];
            sq += s[i] * p[i];
        }
        alpha[k] = sq / sy;
        for (int i = 0; i < n; i++) p[i] -= alpha[k] * y[i];
    }
    if (np > 0) {
        const double *s = S + (size_t)(np - 1) * n, *y = Yh + (size_t)(np - 1) * n;
        double sy = 0, yy = 0;
        for (int i = 0; i < n; i++) {
            sy += s[i] * y[i];
            yy += y[i] * y[i];
        }
        double gamma = sy / yy;
        for (int i = 0; i < n; i++) p[i] *= gamma;
    }
    for (int k = 0; k < np; k++) {
        const double *s = S + (size_t)k * n, *y = Yh + (size_t)k * n;
        double sy = 0, yr = 0;
        for (int i = 0; i < n; i++) {
            sy += s[i] * y[i];
            yr += y[i] * p[i];
        }
        double beta = yr / sy;
        for (int i = 0; i < n; i++) p[i] += s[i] * (alpha[k] - beta);
    }
    for (int i = 0; i < n; i++) p[i] = -p[i];
}

int orc_lbfgs_direction(int n, const double *g, const double *S, const double *Yh, int np,
                        double *p)
{
    double *alpha = malloc(sizeof(double) * (size_t)(np > 0 ? np : 1));
    two_loop(n, g, S, Yh, np, p, alpha);
    free(alpha);
    return 0;
}

/* Curvature-pair acceptance shared by both L-BFGS loops. */
static int accept_pair(const double *s, const double *y, int n)
{
    double sy = 0, ss = 0, yy = 0;
    for (int i = 0; i < n; i++) {
        sy += s[i] * y[i];
        ss += s[i] * s[i];
        yy += y[i] * y[i];
    }
    return sy > 1e-10 * sqrt(ss) * sqrt(yy) && sy > 0;
}

/* Ring of m (s, y) pairs kept oldest-first in contiguous storage. */
static void push_pair(double *S, double *Yh, int *np, int m, int n, const double *s,
                      const double *y)
{
    if (*np == m) {
        memmove(S, S + n, sizeof(double) * (size_t)n * (m - 1));
        memmove(Yh, Yh + n, sizeof(double) * (size_t)n * (m - 1));
        (*np)--;
    }
    memcpy(S + (size_t)(*np) * n, s, sizeof(double) * n);
    memcpy(Yh + (size_t)(*np) * n, y, sizeof(double) * n);
    (*np)++;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1: per-row retrieval                                            */
/* ------------------------------------------------------------------------ */

typedef struct {
    int iters, m, init, power_iters;
    uint64_t seed;
    double clip, tol;
} solve_opts;

static int all_finite(const double *y, size_t K)
{
    for (size_t i = 0; i < K; i++)
        if (!isfinite(y[i])) return 0;
    return 1;
}

/* One row of Algorithm 1.  t holds the initial value on entry when
 * init == INIT_GIVEN.  Each iteration evaluates f and its gradient at the
 * current iterate from their definitions, forms the L-BFGS direction, takes
 * the exact quartic line-search step and updates t. */
static void solve_row(const double *y, const cplx *d, int N, int J, const cplx *tw,
                      const solve_opts *o, int row, cplx *t, double *loss_out, int *iters_out,
                      int *status_out)
{
    size_t K = (size_t)J * N;
    int n2 = 2 * N, m = o->m > 0 ? o->m : 1;
    int zero = 1;
    for (size_t i = 0; i < K; i++)
        if (y[i] != 0) zero = 0;
    if (!all_finite(y, K)) {
        for (int n = 0; n < N; n++) t[n] = 0;
        *loss_out = NAN;
        *iters_out = 0;
        *status_out = ROW_NUMERIC;
        return;
    }
    if (zero) {
        for (int n = 0; n < N; n++) t[n] = 0;
        *loss_out = 0;
        *iters_out = 0;
        *status_out = ROW_ZERO;
        return;
    }
    cplx *z = malloc(sizeof(cplx) * K), *w = malloc(sizeof(cplx) * K), *rz = malloc(sizeof(cplx) * K);
    cplx *sc = malloc(sizeof(cplx) * 3 * (size_t)N), *g = malloc(sizeof(cplx) * (size_t)N);
    cplx *gn = malloc(sizeof(cplx) * (size_t)N), *p = malloc(sizeof(cplx) * (size_t)N);
    cplx *tn = malloc(sizeof(cplx) * (size_t)N);
    double *r = malloc(sizeof(double) * K);
    double *S = malloc(sizeof(double) * (size_t)m * n2), *Yh = malloc(sizeof(double) * (size_t)m * n2);
    double *sv = malloc(sizeof(double) * n2), *yv = malloc(sizeof(double) * n2);
    double *alpha = malloc(sizeof(double) * m);
    int np = 0, status = ROW_MAXITER, done = 0;

    if (o->init != INIT_GIVEN)
        init_row(y, d, N, J, tw, o->init, o->seed, row, o->power_iters, o->clip, t, z, sc);

    double f = loss_grad_row(t, y, d, N, J, tw, g, z, rz, sc);
    for (int it = 0; it < o->iters; it++) {
        if (f == 0 || norm2(g, N) == 0) {
            status = ROW_CONVERGED;
            break;
        }
        two_loop(n2, (const double *)g, S, Yh, np, (double *)p, alpha);
        if (rdot(p, g, N) >= 0) { /* not a descent direction: restart */
            np = 0;
            for (int n = 0; n < N; n++) p[n] = -g[n];
        }
        /* line search along p; z = Q t is left by the last loss evaluation */
        apply_Q(p, d, N, J, tw, w, sc);
        double alph;
        if (g_cost == 1) {
            alph = orc_amp_step((const double *)z, (const double *)w, y, K);
        } else {
            for (size_t i = 0; i < K; i++) r[i] = y[i] - abs2(z[i]);
            double c[5];
            quartic_coeffs(r, z, w, K, c);
            alph = orc_quartic_argmin(c);
        }
        if (!(alph != 0) || !isfinite(alph)) {
            status = isfinite(alph) ? ROW_CONVERGED : ROW_NUMERIC;
            break;
        }
        for (int n = 0; n < N; n++) tn[n] = t[n] + alph * p[n];
        double fn = loss_grad_row(tn, y, d, N, J, tw, gn, z, rz, sc);
        if (!isfinite(fn)) {
            status = ROW_NUMERIC;
            break;
        }
        for (int n = 0; n < N; n++) {
            cplx s = tn[n] - t[n], yy = gn[n] - g[n];
            sv[2 * n] = creal(s);
            sv[2 * n + 1] = cimag(s);
            yv[2 * n] = creal(yy);
            yv[2 * n + 1] = cimag(yy);
        }
        if (accept_pair(sv, yv, n2)) push_pair(S, Yh, &np, m, n2, sv, yv);
        double rel = fabs(f - fn) / fmax(f, 1e-30);
        memcpy(t, tn, sizeof(cplx) * N);
        memcpy(g, gn, sizeof(cplx) * N);
        f = fn;
        done = it + 1;
        if (o->tol > 0 && rel < o->tol) {
            status = ROW_CONVERGED;
            break;
        }
    }
    *loss_out = f;
    *iters_out = done;
    *status_out = status;
    free(z); free(w); free(rz); free(sc); free(g); free(gn); free(p); free(tn); free(r);
    free(S); free(Yh); free(sv); free(yv); free(alpha);
}

/* Retrieve rows of the TM.  T (in/out): initial values when init == 3 (given),
 * otherwise output only.  row_ids: global row index per row (Philox counter). */
int orc_retrieve(const double *Y, const double *masks, int M, int N, int J, const int *row_ids,
                 int iters, int m, int init, uint64_t seed, int power_iters, double clip,
                 double tol, double *T, double *loss, int *iters_done, int *status)
{
    if (M < 0 || N <= 0 || J <= 0 || iters < 0 || m <= 0) return -1;
    const cplx *d = (const cplx *)masks;
    cplx *tw = make_twiddles(N);
    size_t K = (size_t)J * N;
    solve_opts o = {iters, m, init, power_iters, seed, clip, tol};
#pragma omp parallel for schedule(dynamic)
    for (int r = 0; r < M; r++)
        solve_row(Y + (size_t)r * K, d, N, J, tw, &o, row_ids ? row_ids[r] : r,
                  (cplx *)T + (size_t)r * N, &loss[r], &iters_done[r], &status[r]);
    free(tw);
    return 0;
}

/* One L-BFGS step of Algorithm 1 from a given state, for step-level parity:
 * given t, the history pairs (oldest first, as R^(2N) vectors) and the row's
 * data, returns the direction p, the quartic coefficients, alpha, the new t and
 * its loss and gradient. */
int orc_lbfgs_step(const double *y, const double *masks, int N, int J, const double *t,
                   const double *S, const double *Yh, int np, double *p_out, double *coef_out,
                   double *alpha_out, double *t_out, double *loss_out, double *g_out)
{
    if (N <= 0 || J <= 0 || np < 0) return -1;
    const cplx *d = (const cplx *)masks;
    cplx *tw = make_twiddles(N);
    size_t K = (size_t)J * N;
    int n2 = 2 * N;
    cplx *z = malloc(sizeof(cplx) * K), *w = malloc(sizeof(cplx) * K), *rz = malloc(sizeof(cplx) * K);
    cplx *sc = malloc(sizeof(cplx) * 3 * (size_t)N), *g = malloc(sizeof(cplx) * N), *p = (cplx *)p_out;
    double *r = calloc(K, sizeof(double)), *alpha = malloc(sizeof(double) * (np > 0 ? np : 1));
    loss_grad_row((const cplx *)t, y, d, N, J, tw, g, z, rz, sc);
    two_loop(n2, (const double *)g, S, Yh, np, (double *)p, alpha);
    if (rdot(p, g, N) >= 0)
        for (int n = 0; n < N; n++) p[n] = -g[n];
    apply_Q((const cplx *)t, d, N, J, tw, z, sc);
    for (size_t i = 0; i < K; i++) r[i] = y[i] - abs2(z[i]);
    apply_Q(p, d, N, J, tw, w, sc);
    double al;
    if (g_cost == 1) {  /* no quartic: its coefficients are returned as 0 */
        for (int k = 0; k < 5; k++) coef_out[k] = 0;
        al = orc_amp_step((const double *)z, (const double *)w, y, K);
    } else {
        quartic_coeffs(r, z, w, K, coef_out);
        al = orc_quartic_argmin(coef_out);
    }
    *alpha_out = al;
    for (int n = 0; n < N; n++) ((cplx *)t_out)[n] = ((const cplx *)t)[n] + al * p[n];
    *loss_out = loss_grad_row((const cplx *)t_out, y, d, N, J, tw, (cplx *)g_out, z, rz, sc);
    free(z); free(w); free(rz); free(sc); free(g); free(r); free(alpha); free(tw);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Defocus operator and phase-offset fit (Sec. 2.3, App. B)                  */
/* ------------------------------------------------------------------------ */

/* Signed FFT-order frequency of index idx on an axis of length n. */
static int signed_freq(int idx, int n) { return 2 * idx < n ? idx : idx - n; }

/* H[a][b] = exp(-i coef (ky_a^2 + kx_b^2)) on integer frequencies, or the
 * caller's table when H != NULL. */
static cplx *make_transfer(int ny, int nx, const double *H, double coef)
{
    cplx *h = malloc(sizeof(cplx) * (size_t)ny * nx);
    for (int a = 0; a < ny; a++)
        for (int b = 0; b < nx; b++) {
            size_t i = (size_t)a * nx + b;
            if (H) {
                h[i] = ((const cplx *)H)[i];
            } else {
                double ky = signed_freq(a, ny), kx = signed_freq(b, nx);
                double ph = -coef * (ky * ky + kx * kx);
                h[i] = cos(ph) + I * sin(ph);
            }
        }
    return h;
}

/* 2D DFT of an ny x nx array (row-major) as F_ny (x) F_nx: the 1D naive DFT
 * along every row, then along every column. */
static void dft2_naive(const cplx *x, cplx *X, int ny, int nx, int sign, const cplx *twy,
                       const cplx *twx, cplx *col_in, cplx *col_out)
{
    for (int a = 0; a < ny; a++) dft_naive(x + (size_t)a * nx, X + (size_t)a * nx, nx, sign, twx);
    for (int b = 0; b < nx; b++) {
        for (int a = 0; a < ny; a++) col_in[a] = X[(size_t)a * nx + b];
        dft_naive(col_in, col_out, ny, sign, twy);
        for (int a = 0; a < ny; a++) X[(size_t)a * nx + b] = col_out[a];
    }
}

typedef struct {
    int ny, nx;
    cplx *h, *twy, *twx;
} defocus_ctx;

static void ctx_init(defocus_ctx *c, int ny, int nx, const double *H, double coef)
{
    c->ny = ny;
    c->nx = nx;
    c->h = make_transfer(ny, nx, H, coef);
    c->twy = make_twiddles(ny);
    c->twx = make_twiddles(nx);
}

static void ctx_free(defocus_ctx *c)
{
    free(c->h);
    free(c->twy);
    free(c->twx);
}

/* out = D x = ifft2(H .* fft2(x)), or D^H x = ifft2(conj(H) .* fft2(x)).
 * work: ny*nx + 2*max(ny,nx) entries. */
static void defocus_apply(const defocus_ctx *c, const cplx *x, cplx *out, int adjoint, cplx *work)
{
    int ny = c->ny, nx = c->nx;
    size_t P = (size_t)ny * nx;
    cplx *F = work, *ci = work + P, *co = ci + (ny > nx ? ny : nx);
    dft2_naive(x, F, ny, nx, -1, c->twy, c->twx, ci, co);
    for (size_t i = 0; i < P; i++) F[i] *= adjoint ? conj(c->h[i]) : c->h[i];
    dft2_naive(F, out, ny, nx, +1, c->twy, c->twx, ci, co);
    for (size_t i = 0; i < P; i++) out[i] /= (double)P;
}

int orc_defocus_apply(const double *x, int ny, int nx, const double *H, double coef, int adjoint,
                      double *out)
{
    if (ny <= 0 || nx <= 0) return -1;
    defocus_ctx c;
    ctx_init(&c, ny, nx, H, coef);
    size_t P = (size_t)ny * nx;
    cplx *work = malloc(sizeof(cplx) * (P + 2 * (size_t)(ny > nx ? ny : nx)));
    defocus_apply(&c, (const cplx *)x, (cplx *)out, adjoint, work);
    free(work);
    ctx_free(&c);
    return 0;
}

/* Defocus intensities I_n = |D(c_n .* e^{i phi})|^2 (Eq. forwarddefocusImage
 * with the same-grid operator D).  C: [Nd][P] fields c_n; phi: [P] or NULL. */
int orc_defocus_forward(const double *C, int Nd, int ny, int nx, const double *H, double coef,
                        const double *phi, double *Ydef)
{
    if (Nd < 0 || ny <= 0 || nx <= 0) return -1;
    defocus_ctx c;
    ctx_init(&c, ny, nx, H, coef);
    size_t P = (size_t)ny * nx;
#pragma omp parallel
    {
        cplx *x = malloc(sizeof(cplx) * P), *o = malloc(sizeof(cplx) * P);
        cplx *work = malloc(sizeof(cplx) * (P + 2 * (size_t)(ny > nx ? ny : nx)));
#pragma omp for schedule(dynamic)
        for (int n = 0; n < Nd; n++) {
            for (size_t k = 0; k < P; k++) {
                cplx u = phi ? cos(phi[k]) + I * sin(phi[k]) : 1.0;
                x[k] = ((const cplx *)C)[(size_t)n * P + k] * u;
            }
            defocus_apply(&c, x, o, 0, work);
            for (size_t k = 0; k < P; k++) Ydef[(size_t)n * P + k] = abs2(o[k]);
        }
        free(x);
        free(o);
        free(work);
    }
    ctx_free(&c);
    return 0;
}

/* g(phi) = sum_n || I_n - |A_n e^{i phi}|^2 ||^2, A_n = D diag(c_n) (Eq. optphase),
 * dg/dphi = sum_n Re(-4 diag(-i e^{-i phi}) A_n^H diag(A_n e^{i phi}) G_n)
 *         = -4 Im(conj(u) .* sum_n conj(c_n) .* D^H(w_n .* G_n))      (Eq. phasederive)
 * with u = e^{i phi}, w_n = A_n u, G_n = I_n - |w_n|^2.  grad may be NULL.
 * Per-pattern partial sums are added in pattern order. */
static double phase_loss_grad(const defocus_ctx *c, const double *phi, const cplx *C,
                              const double *Ydef, int Nd, double *grad)
{
    size_t P = (size_t)c->ny * c->nx;
    double *fpart = malloc(sizeof(double) * (size_t)(Nd > 0 ? Nd : 1));
    cplx *vpart = grad ? malloc(sizeof(cplx) * P * (size_t)(Nd > 0 ? Nd : 1)) : NULL;
    cplx *u = malloc(sizeof(cplx) * P);
    for (size_t k = 0; k < P; k++) u[k] = cos(phi[k]) + I * sin(phi[k]);
#pragma omp parallel
    {
        cplx *x = malloc(sizeof(cplx) * P), *wv = malloc(sizeof(cplx) * P), *v = malloc(sizeof(cplx) * P);
        cplx *work = malloc(sizeof(cplx) * (P + 2 * (size_t)(c->ny > c->nx ? c->ny : c->nx)));
#pragma omp for schedule(dynamic)
        for (int n = 0; n < Nd; n++) {
            const cplx *cn = C + (size_t)n * P;
            for (size_t k = 0; k < P; k++) x[k] = cn[k] * u[k];
            defocus_apply(c, x, wv, 0, work);
            double f = 0;
            for (size_t k = 0; k < P; k++) {
                double G = Ydef[(size_t)n * P + k] - abs2(wv[k]);
                f += G * G;
                x[k] = wv[k] * G;
            }
            fpart[n] = f;
            if (grad) {
                defocus_apply(c, x, v, 1, work);
                for (size_t k = 0; k < P; k++) vpart[(size_t)n * P + k] = conj(cn[k]) * v[k];
            }
        }
        free(x);
        free(wv);
        free(v);
        free(work);
    }
    double f = 0;
    for (int n = 0; n < Nd; n++) f += fpart[n];
    if (grad) {
        for (size_t k = 0; k < P; k++) {
            cplx v = 0;
            for (int n = 0; n < Nd; n++) v += vpart[(size_t)n * P + k];
            grad[k] = -4.0 * cimag(conj(u[k]) * v);
        }
    }
    free(fpart);
    free(vpart);
    free(u);
    return f;
}

int orc_phase_loss_grad(const double *phi, const double *C, const double *Ydef, int Nd, int ny,
                        int nx, const double *H, double coef, double *loss, double *grad)
{
    if (Nd < 0 || ny <= 0 || nx <= 0) return -1;
    defocus_ctx c;
    ctx_init(&c, ny, nx, H, coef);
    *loss = phase_loss_grad(&c, phi, (const cplx *)C, Ydef, Nd, grad);
    ctx_free(&c);
    return 0;
}

/* L-BFGS over phi from phi = 0 (the initialisation of the paper's phase
 * algorithm) with Armijo backtracking: step 1, halved up to 30 times until
 * g(phi + a p) <= g(phi) + 1e-4 a <grad, p>.  The first direction (and any
 * restart) is -grad / max|grad|, a step of at most one radian.  Stops after
 * `iters` iterations, at a zero gradient or when backtracking fails.
 * Finally phi is shifted by a constant so that arg(sum_k w_k e^{i phi_k}) = 0
 * with weights w (NULL: w = 1). */
/* tol > 0: stop after an accepted step whose decrease f_old - f_new is at
 * most tol f_old (the loss has reached its floor); 0: only the iteration cap
 * and a failed backtracking stop the fit. */
int orc_phase_fit(const double *C, const double *Ydef, int Nd, int ny, int nx, const double *H,
                  double coef, int iters, int m, const double *weights, double *phi,
                  int *iters_done, double *loss_out, double tol)
{
    if (Nd < 0 || ny <= 0 || nx <= 0 || m <= 0) return -1;
    defocus_ctx c;
    ctx_init(&c, ny, nx, H, coef);
    int P = ny * nx;
    double *g = malloc(sizeof(double) * P), *gn = malloc(sizeof(double) * P);
    double *p = malloc(sizeof(double) * P), *pt = malloc(sizeof(double) * P);
    double *S = malloc(sizeof(double) * (size_t)m * P), *Yh = malloc(sizeof(double) * (size_t)m * P);
    double *sv = malloc(sizeof(double) * P), *yv = malloc(sizeof(double) * P);
    double *alpha = malloc(sizeof(double) * m);
    int np = 0, done = 0;
    for (int k = 0; k < P; k++) phi[k] = 0;
    double f = phase_loss_grad(&c, phi, (const cplx *)C, Ydef, Nd, g);
    for (int it = 0; it < iters; it++) {
        double gmax = 0;
        for (int k = 0; k < P; k++) gmax = fmax(gmax, fabs(g[k]));
        if (gmax == 0) break;
        two_loop(P, g, S, Yh, np, p, alpha);
        double gp = 0;
        for (int k = 0; k < P; k++) gp += g[k] * p[k];
        if (np == 0 || gp >= 0) {
            np = 0;
            for (int k = 0; k < P; k++) p[k] = -g[k] / gmax;
            gp = 0;
            for (int k = 0; k < P; k++) gp += g[k] * p[k];
        }
        double a = 1.0, fn = 0;
        int ok = 0;
        for (int h = 0; h <= 30; h++) {
            for (int k = 0; k < P; k++) pt[k] = phi[k] + a * p[k];
            fn = phase_loss_grad(&c, pt, (const cplx *)C, Ydef, Nd, NULL);
            if (fn <= f + 1e-4 * a * gp) {
                ok = 1;
                break;
            }
            a *= 0.5;
        }
        if (!ok) break;
        fn = phase_loss_grad(&c, pt, (const cplx *)C, Ydef, Nd, gn);
        for (int k = 0; k < P; k++) {
            sv[k] = pt[k] - phi[k];
            yv[k] = gn[k] - g[k];
        }
        if (accept_pair(sv, yv, P)) push_pair(S, Yh, &np, m, P, sv, yv);
        memcpy(phi, pt, sizeof(double) * P);
        memcpy(g, gn, sizeof(double) * P);
        const double decrease = f - fn;
        f = fn;
        done = it + 1;
        if (tol > 0 && decrease <= tol * (f + decrease)) break;
    }
    /* remove the free constant: arg(sum_k w_k e^{i phi_k}) = 0 */
    cplx acc = 0;
    for (int k = 0; k < P; k++) acc += (weights ? weights[k] : 1.0) * (cos(phi[k]) + I * sin(phi[k]));
    double shift = carg(acc);
    for (int k = 0; k < P; k++) phi[k] -= shift;
    if (iters_done) *iters_done = done;
    if (loss_out) *loss_out = f;
    free(g); free(gn); free(p); free(pt); free(S); free(Yh); free(sv); free(yv); free(alpha);
    ctx_free(&c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Metrics                                                                   */
/* ------------------------------------------------------------------------ */

/* Row fidelity |<a_r, b_r>| / (||a_r|| ||b_r||), 0 when either row is zero. */
int orc_fidelity_rows(const double *A, const double *B, int M, int N, double *out)
{
    for (int r = 0; r < M; r++) {
        const cplx *a = (const cplx *)A + (size_t)r * N, *b = (const cplx *)B + (size_t)r * N;
        cplx ip = 0;
        for (int n = 0; n < N; n++) ip += conj(a[n]) * b[n];
        double na = sqrt(norm2(a, N)), nb = sqrt(norm2(b, N));
        out[r] = (na > 0 && nb > 0) ? cabs(ip) / (na * nb) : 0.0;
    }
    return 0;
}
