// defocus.cu -- defocus operator and phase-offset fit (Sec. 2.3, App. B).
//
// D x = ifft2(H .* fft2(x)) on the ny x nx pixel grid; the defocus field of
// pattern n is D (c_n .* e^{i phi}) with c_n[r] = (Q t_r)[n] (Eq.
// forwarddefocusImage with the same-grid operator).  The fit minimises
// g(phi) = sum_n ||I_n - |D(c_n .* u)|^2||^2, u = e^{i phi} (Eq. optphase),
// whose gradient is dg/dphi = -4 Im(conj(u) .* sum_n conj(c_n) .* D^H(w_n .* G_n))
// with w_n = D(c_n .* u), G_n = I_n - |w_n|^2 (Eq. phasederive).
//
// The whole fit is one cooperative launch: each CTA owns a set of patterns and
// transforms their grids in shared memory (in-place radix-8/16 2D FFTs, FP32);
// loss and gradient partials are written per CTA and reduced in a fixed order
// (deterministic); the L-BFGS state, the Armijo test and every reduction of the
// fit are FP64.  CTAs meet at a grid barrier whose spin is bounded: on timeout
// the kernel raises an error flag and every CTA returns.
#include <cmath>

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"

namespace tmr {

bool defocus_supported(int ny, int nx)
{
    auto p2 = [](int v) { return v >= 2 && v <= 512 && (v & (v - 1)) == 0; };
    return p2(ny) && p2(nx) && (size_t)(ny) * (nx + 1) * sizeof(float2) <= 160 * 1024;
}

__global__ void k_make_H(int ny, int nx, double coef, float2 *H)
{
    const int P = ny * nx;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        const int a = i / nx, b = i % nx;
        const double ky = 2 * a < ny ? a : a - ny, kx = 2 * b < nx ? b : b - nx;
        double s, c;
        sincos(-coef * (ky * ky + kx * kx), &s, &c);
        H[i] = make_float2((float)c, (float)s);
    }
}

cudaError_t launch_make_quadratic_H(int ny, int nx, double coef, float2 *H, cudaStream_t s)
{
    k_make_H<<<64, 256, 0, s>>>(ny, nx, coef, H);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// shared-memory 2D FFT, in place, radix-2 decimation in time after a
// bit-reversal permutation along each axis.  grid pitch = nx + 1 float2.

// tw[k] = exp(-2 pi i k / n), k < n/2 (twy for ny, twx for nx), made once per CTA.
__device__ void make_tw(float2 *tw, int n)
{
    for (int k = threadIdx.x; k < n / 2; k += blockDim.x) {
        double s, c;
        sincospi(-2.0 * k / n, &s, &c);
        tw[k] = make_float2((float)c, (float)s);
    }
}

// ---------------------------------------------------------------------------
// In-place 2D FFT of an ny x nx grid in shared memory (row pitch nx + 1).
// Each axis of length n = 2^l runs as a few radix-R stages (R = 8, with one
// radix-16, radix-4 or radix-2 stage first when l is not a multiple of 3):
// the forward transform is decimation in frequency from natural order, so
// the spectrum is left in digit-reversed order (spec_freq gives the frequency
// at a position); the inverse is the mirror decimation in time from that
// order back to natural order (unnormalised).  Every product with a spectrum
// (the kernel h, the padding's ramps) indexes it through spec_freq, so no
// reordering pass is needed.  Row stages map consecutive threads to
// consecutive rows and column stages to consecutive columns: with the odd
// pitch both touch shared memory without bank conflicts.

// stage s has radix 2^lr(s): lr0 for the first stage, 3 (radix 8) after it
struct AxisPlan {
    int n, ln, lr0, ns;
    __device__ int lr(int s) const { return s == 0 ? lr0 : 3; }
};

__device__ __forceinline__ AxisPlan axis_plan(int n)
{
    AxisPlan P;
    P.n = n;
    P.ln = __ffs(n) - 1;
    const int l = P.ln;
    P.lr0 = l == 1 ? 1 : (l % 3 == 1 ? 4 : (l % 3 == 2 ? 2 : 3));
    P.ns = 1 + (l - P.lr0) / 3;
    return P;
}

// frequency held at position pos after the forward stages: the digits of pos
// in the stage radices (most significant first) are the frequency's digits
// from the least significant up
__device__ __forceinline__ int axis_freq(const AxisPlan &P, int pos)
{
    int f = 0, lmul = 0, lspan = P.ln;
    for (int s = 0; s < P.ns; s++) {
        const int l = P.lr(s);
        lspan -= l;
        f |= ((pos >> lspan) & ((1 << l) - 1)) << lmul;
        lmul += l;
    }
    return f;
}

// W_n^idx from the half table tw[k] = exp(-2 pi i k / n), k < n / 2, idx < n
__device__ __forceinline__ float2 tw_full(const float2 *tw, int n, int idx)
{
    if (idx < n / 2) return tw[idx];
    const float2 w = tw[idx - n / 2];
    return make_float2(-w.x, -w.y);
}

// One forward (FWD) or inverse stage of radix R and length L on every line
// of one axis.  Along rows (ROWS): element e of line a at a * pitch + e,
// nlines = ny; along columns: element e of line x at e * pitch + x.
template <int R, bool FWD, bool ROWS>
__device__ void fft_stage(float2 *g, int n, int nlines, int pitch, int L, const float2 *tw)
{
    const int m = L / R, per = n / R, total = nlines * per;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int line = i % nlines, q = i / nlines;  // lines fastest
        const int b = q / m, j = q - b * m;
        const int e0 = b * L + j;
        float2 *base = ROWS ? g + line * pitch + e0 : g + e0 * pitch + line;
        const int es = ROWS ? m : m * pitch;
        float2 x[R];
#pragma unroll
        for (int k = 0; k < R; k++) x[k] = base[k * es];
        const int step = j * (n / L);
        if (FWD) {
            dft_small<R, -1>(x);
#pragma unroll
            for (int k = 1; k < R; k++) x[k] = cmul(x[k], tw_full(tw, n, step * k));
        } else {
#pragma unroll
            for (int k = 1; k < R; k++) x[k] = cmulc(x[k], tw_full(tw, n, step * k));
            dft_small<R, 1>(x);
        }
#pragma unroll
        for (int k = 0; k < R; k++) base[k * es] = x[k];
    }
    __syncthreads();
}

template <bool FWD, bool ROWS>
__device__ void fft_axis(float2 *g, const AxisPlan &P, int nlines, int pitch, const float2 *tw)
{
    // forward: stages 0 .. ns-1 (span shrinking); inverse: the reverse order
    for (int t = 0; t < P.ns; t++) {
        const int s = FWD ? t : P.ns - 1 - t;
        int lL = P.ln;
        for (int u = 0; u < s; u++) lL -= P.lr(u);
        const int L = 1 << lL;
        switch (1 << P.lr(s)) {
        case 2: fft_stage<2, FWD, ROWS>(g, P.n, nlines, pitch, L, tw); break;
        case 4: fft_stage<4, FWD, ROWS>(g, P.n, nlines, pitch, L, tw); break;
        case 8: fft_stage<8, FWD, ROWS>(g, P.n, nlines, pitch, L, tw); break;
        default: fft_stage<16, FWD, ROWS>(g, P.n, nlines, pitch, L, tw); break;
        }
    }
}

// forward 2D DFT (exp(-2 pi i ...)), natural order in, digit-reversed out
__device__ void fft2_fwd(float2 *g, int ny, int nx, const float2 *twy, const float2 *twx)
{
    const AxisPlan Px = axis_plan(nx), Py = axis_plan(ny);
    fft_axis<true, true>(g, Px, ny, nx + 1, twx);
    fft_axis<true, false>(g, Py, nx, nx + 1, twy);
}

// unnormalised inverse 2D DFT, digit-reversed order in, natural out
__device__ void fft2_inv(float2 *g, int ny, int nx, const float2 *twy, const float2 *twx)
{
    const AxisPlan Px = axis_plan(nx), Py = axis_plan(ny);
    fft_axis<false, false>(g, Py, nx, nx + 1, twy);
    fft_axis<false, true>(g, Px, ny, nx + 1, twx);
}

// natural frequencies (ky index, kx index) of the spectrum at grid position (a, b)
struct SpecMap {
    AxisPlan py, px;
    __device__ void init(int ny, int nx)
    {
        py = axis_plan(ny);
        px = axis_plan(nx);
    }
    __device__ int fy(int a) const { return axis_freq(py, a); }
    __device__ int fx(int b) const { return axis_freq(px, b); }
};

// g <- D g (adjoint: D^H g), including the 1/P of the inverse transform.
__device__ void defocus_apply_smem(float2 *g, int ny, int nx, const float2 *__restrict__ H,
                                   bool adjoint, const float2 *twy, const float2 *twx)
{
    const int pitch = nx + 1, P = ny * nx, lx = __ffs(nx) - 1;
    SpecMap sm;
    sm.init(ny, nx);
    fft2_fwd(g, ny, nx, twy, twx);
    const float inv = 1.0f / (float)P;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int a = i >> lx, b = i & (nx - 1);
        float2 h = H[sm.fy(a) * nx + sm.fx(b)];
        if (adjoint) h.y = -h.y;
        g[a * pitch + b] = cscale(cmul(g[a * pitch + b], h), inv);
    }
    __syncthreads();
    fft2_inv(g, ny, nx, twy, twx);
}

static size_t defocus_smem(int ny, int nx)
{
    return sizeof(float2) * ((size_t)ny * (nx + 1) + ny / 2 + nx / 2) + 64 * sizeof(double);
}

__global__ void k_defocus_forward(int ny, int nx, int Nd, const float2 *__restrict__ Zd,
                                  const float2 *__restrict__ H, float *__restrict__ Ydef)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = ny * nx, pitch = nx + 1;
    float2 *g = reinterpret_cast<float2 *>(smem_raw);
    float2 *twy = g + (size_t)ny * pitch, *twx = twy + ny / 2;
    make_tw(twy, ny);
    make_tw(twx, nx);
    for (int n = blockIdx.x; n < Nd; n += gridDim.x) {
        for (int i = threadIdx.x; i < P; i += blockDim.x) g[(i / nx) * pitch + i % nx] = Zd[(size_t)n * P + i];
        __syncthreads();
        defocus_apply_smem(g, ny, nx, H, false, twy, twx);
        for (int i = threadIdx.x; i < P; i += blockDim.x) Ydef[(size_t)n * P + i] = cabs2(g[(i / nx) * pitch + i % nx]);
        __syncthreads();
    }
}

cudaError_t launch_defocus_forward(int ny, int nx, int Nd, const float2 *Zd, const float2 *H,
                                   const float2 *, const float2 *, float *Ydef, cudaStream_t s)
{
    if (Nd == 0) return cudaSuccess;
    const size_t sm = defocus_smem(ny, nx);
    cudaError_t e = cudaFuncSetAttribute(k_defocus_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = Nd < nsm ? Nd : nsm;
    k_defocus_forward<<<grid, 512, sm, s>>>(ny, nx, Nd, Zd, H, Ydef);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The paper's defocus model (Sec. 2.3, Eq. angularspectrum, Eq.
// forwarddefocusImage): fields c_n = TM_est e^{j theta_n} of separate incident
// fields, A = K2^H P diag(h) K1 with the angular-spectrum kernel h and its NA
// pupil on the half grid's frequencies, P the zero padding of the spectrum to
// the 2ny x 2nx grid and K2^H the inverse DFT there (divided by ny nx, so that
// with h = 1 the even full-grid pixels reproduce the half grid).  The padded
// inverse is evaluated as four inverse DFTs of the half grid: the full-grid
// pixel (2a + s, 2b + t) is
//   (1 / (ny nx)) sum_{ky,kx} X[ky][kx] e^{i pi (ky s / ny + kx t / nx)} e^{2 pi i (ky a / ny + kx b / nx)}
// (ky, kx the signed frequencies), i.e. the half-grid inverse of X times the
// ramp ry^s rx^t, ry[ky] = e^{i pi ky / ny}, rx[kx] = e^{i pi kx / nx}; the
// adjoint sums the four forward DFTs of the subgrids times the conjugate ramps.

__global__ void k_make_H2x(int ny, int nx, double wavelength, double na, double zd, double pixel, float2 *H)
{
    const int P = ny * nx;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        const int a = i / nx, b = i % nx;
        const double ky = 2 * a < ny ? a : a - ny, kx = 2 * b < nx ? b : b - nx;
        const double lu = wavelength * kx / (nx * pixel), lv = wavelength * ky / (ny * pixel);
        const double rho2 = lu * lu + lv * lv;
        if (sqrt(rho2) <= na) {
            double s, c;
            sincos(2.0 * M_PI / wavelength * sqrt(fmax(1.0 - rho2, 0.0)) * zd, &s, &c);
            H[i] = make_float2((float)c, (float)s);
        } else {
            H[i] = make_float2(0.f, 0.f);
        }
    }
}

cudaError_t launch_make_H2x(int ny, int nx, double wavelength, double na, double zd, double pixel, float2 *H,
                            cudaStream_t s)
{
    k_make_H2x<<<64, 256, 0, s>>>(ny, nx, wavelength, na, zd, pixel, H);
    return cudaGetLastError();
}

// Zd[n][r] = sum_k T[r][k] inc[n][k] (FP32): a tiled complex product, 64 rows
// x 32 fields per CTA, 16 x 16 threads with 4 x 2 outputs each, k in steps of 32.
__global__ void __launch_bounds__(256) k_incident_fields(int M, int N, int Nd, const float2 *__restrict__ T,
                                                         const float2 *__restrict__ inc, float2 *__restrict__ Zd)
{
    __shared__ float2 Ts[64][33], Is[32][33];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int r0 = blockIdx.x * 64, n0 = blockIdx.y * 32;
    float2 acc[4][2];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 2; j++) acc[i][j] = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < N; k0 += 32) {
        for (int e = threadIdx.x; e < 64 * 32; e += 256) {
            const int rr = e >> 5, kk = e & 31;
            Ts[rr][kk] = (r0 + rr < M && k0 + kk < N) ? T[(size_t)(r0 + rr) * N + k0 + kk] : make_float2(0.f, 0.f);
        }
        for (int e = threadIdx.x; e < 32 * 32; e += 256) {
            const int nn = e >> 5, kk = e & 31;
            Is[nn][kk] = (n0 + nn < Nd && k0 + kk < N) ? inc[(size_t)(n0 + nn) * N + k0 + kk] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; kk++) {
            float2 tv[4], iv[2];
#pragma unroll
            for (int i = 0; i < 4; i++) tv[i] = Ts[ty + 16 * i][kk];
#pragma unroll
            for (int j = 0; j < 2; j++) iv[j] = Is[tx + 16 * j][kk];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 2; j++) {
                    acc[i][j].x = fmaf(tv[i].x, iv[j].x, fmaf(-tv[i].y, iv[j].y, acc[i][j].x));
                    acc[i][j].y = fmaf(tv[i].x, iv[j].y, fmaf(tv[i].y, iv[j].x, acc[i][j].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 2; j++) {
            const int r = r0 + ty + 16 * i, n = n0 + tx + 16 * j;
            if (r < M && n < Nd) Zd[(size_t)n * M + r] = acc[i][j];
        }
}

cudaError_t launch_incident_fields(int M, int N, int Nd, const float2 *T, const float2 *inc, float2 *Zd,
                                   cudaStream_t s)
{
    if (M == 0 || Nd == 0) return cudaSuccess;
    dim3 grid((M + 63) / 64, (Nd + 31) / 32);
    k_incident_fields<<<grid, 256, 0, s>>>(M, N, Nd, T, inc, Zd);
    return cudaGetLastError();
}

// ramps of the four subgrids: ry[a] = e^{i pi ky(a) / ny}, rx[b] = e^{i pi kx(b) / nx}
__device__ void make_ramps(float2 *ry, float2 *rx, int ny, int nx)
{
    for (int a = threadIdx.x; a < ny; a += blockDim.x) {
        double s, c;
        sincospi((double)(2 * a < ny ? a : a - ny) / ny, &s, &c);
        ry[a] = make_float2((float)c, (float)s);
    }
    for (int b = threadIdx.x; b < nx; b += blockDim.x) {
        double s, c;
        sincospi((double)(2 * b < nx ? b : b - nx) / nx, &s, &c);
        rx[b] = make_float2((float)c, (float)s);
    }
}

__device__ __forceinline__ float2 ramp_st(int st, int a, int b, const float2 *ry, const float2 *rx)
{
    switch (st) {
    case 0: return make_float2(1.f, 0.f);
    case 1: return rx[b];
    case 2: return ry[a];
    default: return cmul(ry[a], rx[b]);
    }
}

static size_t defocus2x_smem(int ny, int nx, int grids)
{
    return sizeof(float2) * ((size_t)grids * ny * (nx + 1) + ny / 2 + nx / 2 + ny + nx) + 64 * sizeof(double);
}

bool phase_fit2x_fits(int ny, int nx);

bool defocus2x_supported(int ny, int nx)
{
    auto p2 = [](int v) { return v >= 2 && v <= 512 && (v & (v - 1)) == 0; };
    return p2(ny) && p2(nx) && phase_fit2x_fits(ny, nx);
}

// Ydef[n][(2a + s) 2nx + 2b + t] = |A c_n|^2 at the full-grid pixels.
__global__ void k_defocus_forward2x(int ny, int nx, int Nd, const float2 *__restrict__ Zd,
                                    const float2 *__restrict__ H, float *__restrict__ Ydef)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = ny * nx, pitch = nx + 1, lx = __ffs(nx) - 1;
    float2 *g = reinterpret_cast<float2 *>(smem_raw);
    float2 *Xs = g + (size_t)ny * pitch;
    float2 *twy = Xs + (size_t)ny * pitch, *twx = twy + ny / 2, *ry = twx + nx / 2, *rx = ry + ny;
    make_tw(twy, ny);
    make_tw(twx, nx);
    make_ramps(ry, rx, ny, nx);
    SpecMap sm;
    sm.init(ny, nx);
    const float inv = 1.f / (float)P;
    for (int n = blockIdx.x; n < Nd; n += gridDim.x) {
        for (int i = threadIdx.x; i < P; i += blockDim.x) g[(i >> lx) * pitch + (i & (nx - 1))] = Zd[(size_t)n * P + i];
        __syncthreads();
        fft2_fwd(g, ny, nx, twy, twx);
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            const int a = i >> lx, b = i & (nx - 1), gi = a * pitch + b;
            Xs[gi] = cmul(g[gi], H[sm.fy(a) * nx + sm.fx(b)]);
        }
        __syncthreads();
        for (int st = 0; st < 4; st++) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int a = i >> lx, b = i & (nx - 1), gi = a * pitch + b;
                g[gi] = cmul(Xs[gi], ramp_st(st, sm.fy(a), sm.fx(b), ry, rx));
            }
            __syncthreads();
            fft2_inv(g, ny, nx, twy, twx);
            const int s = st >> 1, t = st & 1;
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int a = i >> lx, b = i & (nx - 1);
                Ydef[(size_t)n * 4 * P + (size_t)(2 * a + s) * (2 * nx) + 2 * b + t] =
                    cabs2(cscale(g[a * pitch + b], inv));
            }
            __syncthreads();
        }
    }
}

cudaError_t launch_defocus_forward2x(int ny, int nx, int Nd, const float2 *Zd, const float2 *H, float *Ydef,
                                     cudaStream_t s)
{
    if (Nd == 0) return cudaSuccess;
    const size_t sm = defocus2x_smem(ny, nx, 2);
    cudaError_t e = cudaFuncSetAttribute(k_defocus_forward2x, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = Nd < nsm ? Nd : nsm;
    k_defocus_forward2x<<<grid, 512, sm, s>>>(ny, nx, Nd, Zd, H, Ydef);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Phase-offset fit.

// bounded grid barrier; bar[0] arrival count, bar[1] generation.  A wait gives
// up after `limit` polls (about 64 ns each after the first 4096), raises *err
// and returns false; so does every CTA that sees *err raised.  `withhold`
// (a test hook) keeps the last CTA from releasing the others, so that every
// wait runs out.
__device__ bool grid_sync(unsigned *bar, int *err, long long limit, bool withhold)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = bar + 1;
        volatile int *verr = err;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u) + 1u;
        if (arrived == gridDim.x && !withhold) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            // poll tightly at first (the other CTAs usually arrive within
            // microseconds), then back off; give up after about a second
            long long spins = 0;
            while (*vgen == gen) {
                if (*verr) break;
                if (++spins > limit) {
                    atomicExch(err, 1);
                    break;
                }
                if (spins > 4096) __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int *)err == 0;
}

int phase_fit_grid(int ny, int nx, int Nd)
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    (void)ny;
    (void)nx;
    int g = Nd < nsm ? Nd : nsm;
    return g < 1 ? 1 : g;
}

constexpr int kPfSlots = kMaxMem + 1;
constexpr int kPfDots = 4 * kPfSlots + 4;  // per age 4 dots, then ss, gg, gmax, spare

// workspace (in doubles): phi, p, g, phit, S[m+1], Y[m+1] (P each, chunk-owned),
// fpart[grid], pdot[grid][kPfDots], part[grid][P] (floats), u[P] (float2)
size_t phase_fit_workspace_doubles(int P, int Nd, int m, int grid)
{
    (void)Nd;
    return (size_t)P * (4 + 2 * (m + 1)) + grid + (size_t)grid * kPfDots + ((size_t)grid * P + 1) / 2 +
           2 * (size_t)P + 64;
}

struct PFWork {
    double *phi, *p, *g, *phit, *S, *Y, *fpart, *pdot;
    float *part;
    float2 *u;
    double *gsum;  // [P] the new gradient of an accepted step, summed over the CTAs' partials
};

__device__ PFWork pf_carve(double *ws, int P, int m, int grid)
{
    PFWork w;
    w.phi = ws;
    w.p = w.phi + P;
    w.g = w.p + P;
    w.phit = w.g + P;
    w.S = w.phit + P;
    w.Y = w.S + (size_t)(m + 1) * P;
    w.fpart = w.Y + (size_t)(m + 1) * P;
    w.pdot = w.fpart + grid;
    w.part = reinterpret_cast<float *>(w.pdot + (size_t)grid * kPfDots);
    w.u = reinterpret_cast<float2 *>(w.pdot + (size_t)grid * kPfDots + ((size_t)grid * P + 1) / 2);
    w.gsum = reinterpret_cast<double *>(w.u + P);
    return w;
}

// The cross-CTA sums of the fit, each in a fixed order (deterministic) and
// spread over lanes so that no thread walks all nb partials in sequence.
// out[k] = sum_b part[b P + k] for k in [k0, k1): 8 lanes per element, lane s
// adding b = s, s + 8, ..., then an xor tree over the 8 lanes.
__device__ void pf_part_sums(const float *part, int nb, int P, int k0, int k1, double *out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int sub = lane & 7, slot = lane >> 3;
    for (int base = k0 + 4 * warp; base < k1; base += 4 * nw) {
        const int k = base + slot;
        double s = 0.0;
        if (k < k1)
            for (int b = sub; b < nb; b += 8) s += (double)__ldcg(part + (size_t)b * P + k);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 4);
        if (sub == 0 && k < k1) out[k] = s;
    }
}

// Block sums of 32 values per thread (kPfDots): within each warp a
// transposing xor tree leaves value l's warp sum in lane l (31 additions per
// lane instead of 32 x 5), then 32 threads add the warps' sums in order.
static_assert(kPfDots == 32, "block_sum32 reduces 32 values");
__device__ void block_sum32(double (&v)[32], double *red, double *out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        const bool upper = (lane & h) != 0;
#pragma unroll
        for (int i = 0; i < h; i++) {
            const double send = upper ? v[i] : v[i + h];
            const double keep = upper ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
        }
    }
    red[lane * nw + warp] = v[0];
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = 0.0;
        for (int w = 0; w < nw; w++) s += red[threadIdx.x * nw + w];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// sum_b x[b] over b < nb by the lanes of one warp (lane-strided, xor tree):
// every lane of every warp that calls it gets the same value
__device__ __forceinline__ double warp_sum_nb(const double *x, int nb)
{
    double s = 0.0;
    for (int b = threadIdx.x & 31; b < nb; b += 32) s += __ldcg(x + b);
    for (int o = 1; o < 32; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// L-BFGS scalars of the phase fit (FP64), replicated in every CTA; pairs by age.
struct PFGram {
    double SY[kPfSlots][kPfSlots], YY[kPfSlots][kPfSlots];
    double rD[kPfSlots], Sg[kPfSlots], Yg[kPfSlots], c1[kPfSlots], c2[kPfSlots];
    double gamma, gg, gmax, f, gp, a;
    double red[kPfDots];
    int slot[kPfSlots];
    int np, restart;
    int floor_reached;  // the last accepted step lowered g by at most tol g (PhaseFitParams::tol)
};

// compact-form coefficients (one thread); restart = 1 selects p = -g / max|g|
__device__ void pf_coefficients(PFGram &G)
{
    const int np = G.np;
    for (int i = 0; i < kPfSlots; i++) G.c1[i] = G.c2[i] = 0.0;
    G.restart = 1;
    if (np > 0) {
        const double gamma = G.SY[np - 1][np - 1] / G.YY[np - 1][np - 1];
        double c1[kPfSlots], c2[kPfSlots];
        for (int i = np - 1; i >= 0; i--) {
            double s = -G.Sg[i];
            for (int j = i + 1; j < np; j++) s -= G.SY[i][j] * c2[j];
            c2[i] = s * G.rD[i];
        }
        for (int i = 0; i < np; i++) {
            double rhs = -G.SY[i][i] * c2[i] - gamma * G.Yg[i];
            for (int j = 0; j < np; j++) rhs -= gamma * G.YY[i < j ? i : j][i < j ? j : i] * c2[j];
            for (int j = 0; j < i; j++) rhs -= G.SY[j][i] * c1[j];
            c1[i] = rhs * G.rD[i];
        }
        double pg = gamma * G.gg;
        for (int i = 0; i < np; i++) pg += c1[i] * G.Sg[i] + gamma * c2[i] * G.Yg[i];
        if (pg > 0.0 && isfinite(pg)) {
            G.gamma = gamma;
            for (int i = 0; i < np; i++) {
                G.c1[i] = c1[i];
                G.c2[i] = gamma * c2[i];
            }
            G.gp = -pg;
            G.restart = 0;
            return;
        }
        G.np = 0;
    }
    G.gamma = 1.0;
    G.gp = G.gmax > 0.0 ? -G.gg / G.gmax : 0.0;
}

// The 2x-padded operator's share of pf_eval for pattern n: on return g holds
// A^H(w G) on the half grid, with w = A(c_n u) on the full grid and
// G = I_n - |w|^2, and the loss of the pattern is added to fpl.  Xs and S are
// two more grids: X h, and the accumulated cropped spectrum of w G.
__device__ void pf_pattern2x(const PhaseFitParams &Pp, int n, float2 *g, float2 *Xs, float2 *S, const float2 *twy,
                             const float2 *twx, const float2 *ry, const float2 *rx, float &fpl)
{
    const int ny = Pp.ny, nx = Pp.nx, P = ny * nx, pitch = nx + 1, lx = __ffs(nx) - 1;
    const float *In = Pp.Ydef + (size_t)n * 4 * P;
    const float inv = 1.0f / (float)P;
    SpecMap sm;
    sm.init(ny, nx);
    fft2_fwd(g, ny, nx, twy, twx);
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int a = i >> lx, b = i & (nx - 1), gi = a * pitch + b;
        Xs[gi] = cmul(g[gi], Pp.H[sm.fy(a) * nx + sm.fx(b)]);
        S[gi] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int st = 0; st < 4; st++) {
        const int s = st >> 1, t = st & 1;
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            const int a = i >> lx, b = i & (nx - 1), gi = a * pitch + b;
            g[gi] = cmul(Xs[gi], ramp_st(st, sm.fy(a), sm.fx(b), ry, rx));
        }
        __syncthreads();
        fft2_inv(g, ny, nx, twy, twx);
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            const int a = i >> lx, b = i & (nx - 1), gi = a * pitch + b;
            const float2 w = cscale(g[gi], inv);
            const float Gv = In[(size_t)(2 * a + s) * (2 * nx) + 2 * b + t] - cabs2(w);
            fpl = fmaf(Gv, Gv, fpl);
            g[gi] = cscale(w, Gv);
        }
        __syncthreads();
        fft2_fwd(g, ny, nx, twy, twx);
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            const int a = i >> lx, b = i & (nx - 1), gi = a * pitch + b;
            S[gi] = cadd(S[gi], cmulc(g[gi], ramp_st(st, sm.fy(a), sm.fx(b), ry, rx)));
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int a = i >> lx, b = i & (nx - 1), gi = a * pitch + b;
        g[gi] = cscale(cmulc(S[gi], Pp.H[sm.fy(a) * nx + sm.fx(b)]), inv);
    }
    __syncthreads();
    fft2_inv(g, ny, nx, twy, twx);
}

// Loss and gradient partials of this CTA's patterns for the phase table u:
// part[blockIdx.x][:] (FP32, at most a few patterns per CTA) and fpart (FP64).
// ex (kind 1 only): the grids Xs, S and the ramps ry, rx of pf_pattern2x.
struct PFExtra {
    float2 *Xs, *S;
    const float2 *ry, *rx;
};

__device__ void pf_eval(const PhaseFitParams &Pp, const PFWork &W, float2 *g, const float2 *twy,
                        const float2 *twx, double *red, double *out, const PFExtra &ex)
{
    const int ny = Pp.ny, nx = Pp.nx, P = ny * nx, pitch = nx + 1, lx = __ffs(nx) - 1;
    auto at = [&](int k) { return (k >> lx) * pitch + (k & (nx - 1)); };
    float *part = W.part + (size_t)blockIdx.x * P;
    for (int k = threadIdx.x; k < P; k += blockDim.x) part[k] = 0.f;
    double fl = 0.0;
    if (Pp.kind == 1) {
        for (int n = blockIdx.x; n < Pp.Nd; n += gridDim.x) {
            const float2 *cn = Pp.Zd + (size_t)n * P;
            for (int k = threadIdx.x; k < P; k += blockDim.x) g[at(k)] = cmul(cn[k], __ldcg(W.u + k));
            __syncthreads();
            float fpl = 0.f;
            pf_pattern2x(Pp, n, g, ex.Xs, ex.S, twy, twx, ex.ry, ex.rx, fpl);
            fl += (double)fpl;
            for (int k = threadIdx.x; k < P; k += blockDim.x) {
                const float2 v = cmulc(g[at(k)], cn[k]);  // conj(c_n) A^H(w G)
                const float2 cu = __ldcg(W.u + k);
                part[k] += -4.f * fmaf(cu.x, v.y, -cu.y * v.x);  // -4 Im(conj(u) v)
            }
            __syncthreads();
        }
        double fv[1] = {fl};
        block_sum<1, double>(fv, red, out);
        if (threadIdx.x == 0) W.fpart[blockIdx.x] = out[0];
        return;
    }
    for (int n = blockIdx.x; n < Pp.Nd; n += gridDim.x) {
        const float2 *cn = Pp.Zd + (size_t)n * P;
        const float *In = Pp.Ydef + (size_t)n * P;
        for (int k = threadIdx.x; k < P; k += blockDim.x)
            g[at(k)] = cmul(cn[k], __ldcg(W.u + k));
        __syncthreads();
        defocus_apply_smem(g, ny, nx, Pp.H, false, twy, twx);
        float fpl = 0.f;
        for (int k = threadIdx.x; k < P; k += blockDim.x) {
            const int gi = at(k);
            const float2 w = g[gi];
            const float Gv = In[k] - cabs2(w);
            fpl = fmaf(Gv, Gv, fpl);
            g[gi] = cscale(w, Gv);
        }
        fl += (double)fpl;
        __syncthreads();
        defocus_apply_smem(g, ny, nx, Pp.H, true, twy, twx);
        for (int k = threadIdx.x; k < P; k += blockDim.x) {
            const float2 v = cmulc(g[at(k)], cn[k]);  // conj(c_n) D^H(w G)
            const float2 cu = __ldcg(W.u + k);
            part[k] += -4.f * fmaf(cu.x, v.y, -cu.y * v.x);  // -4 Im(conj(u) v)
        }
        __syncthreads();
    }
    double fv[1] = {fl};
    block_sum<1, double>(fv, red, out);
    if (threadIdx.x == 0) W.fpart[blockIdx.x] = out[0];
}

// The phase-offset fit: L-BFGS over phi from phi = 0 with Armijo backtracking.
// CTA b owns the chunk [k0, k1) of every length-P vector (phi, g, p, the
// pairs); the cross-CTA traffic is the phase table u (written by chunks, read
// whole by every CTA's pattern evaluations), the gradient partials and one
// batched FP64 reduction of dot products per accepted step.  Every CTA holds
// the same FP64 L-BFGS scalars (identical sums in identical order), so all
// take the same decisions.
__global__ void __launch_bounds__(512) k_phase_fit(PhaseFitParams Pp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ny = Pp.ny, nx = Pp.nx, P = ny * nx, m = Pp.m, nb = gridDim.x;
    const int ngrid = Pp.kind == 1 ? 3 : 1;
    float2 *g = reinterpret_cast<float2 *>(smem_raw);
    float2 *twy = g + (size_t)ngrid * ny * (nx + 1), *twx = twy + ny / 2;
    float2 *ry = twx + nx / 2, *rx = ry + ny;
    double *red = reinterpret_cast<double *>(rx + nx + 1);
    double *out = red + 32 * kPfDots;
    __shared__ PFGram G;
    PFWork W = pf_carve(Pp.ws, P, m, nb);
    make_tw(twy, ny);
    make_tw(twx, nx);
    PFExtra ex{g + (size_t)ny * (nx + 1), g + (size_t)2 * ny * (nx + 1), ry, rx};
    if (Pp.kind == 1) make_ramps(ry, rx, ny, nx);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int chunk = (P + nb - 1) / nb, k0 = min(P, blockIdx.x * chunk), k1 = min(P, k0 + chunk);
    double *Sg_ = W.S, *Yg_ = W.Y;

    // reduce kPfDots per-thread values over the grid: block sums to pdot[b], a
    // grid barrier, then every CTA adds the nb partials in order into G.red
    auto grid_dots = [&](double (&v)[kPfDots], double vmax) -> bool {
        block_sum32(v, red, out);
        __shared__ double mx[32];
        double mv = vmax;
        for (int o = 16; o > 0; o >>= 1) mv = fmax(mv, __shfl_xor_sync(0xffffffffu, mv, o));
        if ((tid & 31) == 0) mx[tid >> 5] = mv;
        __syncthreads();
        if (tid < kPfDots) {
            double val = out[tid];
            if (tid == kPfDots - 2) {
                val = 0.0;
                for (int w = 0; w < nt / 32; w++) val = fmax(val, mx[w]);
            }
            W.pdot[(size_t)blockIdx.x * kPfDots + tid] = val;
        }
        if (!grid_sync(Pp.sync, Pp.err, Pp.wait_spins, Pp.withhold_release)) return false;
        {
            // value vi by 16 lanes (b = sub, sub + 16, ...), then an xor tree
            const int vi = tid >> 4, sub = tid & 15;
            const bool is_max = vi == kPfDots - 2;
            double acc = 0.0;
            if (vi < kPfDots)
                for (int b = sub; b < nb; b += 16) {
                    const double x = __ldcg(W.pdot + (size_t)b * kPfDots + vi);
                    acc = is_max ? fmax(acc, x) : acc + x;
                }
            for (int o = 1; o < 16; o <<= 1) {
                const double y = __shfl_xor_sync(0xffffffffu, acc, o);
                acc = is_max ? fmax(acc, y) : acc + y;
            }
            if (sub == 0 && vi < kPfDots) G.red[vi] = acc;
        }
        __syncthreads();
        return true;
    };
    // phase table of phit for my chunk
    auto write_u = [&](const double *ph) {
        for (int k = k0 + tid; k < k1; k += nt) {
            float s, c;
            sincosf((float)ph[k], &s, &c);
            W.u[k] = make_float2(c, s);
        }
    };

    // a wait ran out (or another CTA's did): phi keeps its last accepted value
    // on my chunk, without the constant-phase normalisation, and the CTA returns
    auto bail = [&]() {
        for (int k = k0 + tid; k < k1; k += nt) Pp.phi[k] = W.phi[k];
    };

    // ---- phi = 0: loss and gradient ----
    for (int k = k0 + tid; k < k1; k += nt) {
        W.phi[k] = 0.0;
        W.phit[k] = 0.0;
    }
    write_u(W.phit);
    if (!grid_sync(Pp.sync, Pp.err, Pp.wait_spins, Pp.withhold_release)) {
        bail();
        return;
    }
    pf_eval(Pp, W, g, twy, twx, red, out, ex);
    if (!grid_sync(Pp.sync, Pp.err, Pp.wait_spins, Pp.withhold_release)) {
        bail();
        return;
    }
    {
        pf_part_sums(W.part, nb, P, k0, k1, W.g);
        __syncthreads();
        double v[kPfDots] = {0.0};
        double vmax = 0.0;
        for (int k = k0 + tid; k < k1; k += nt) {
            const double s = W.g[k];
            v[4 * kPfSlots + 1] += s * s;
            vmax = fmax(vmax, fabs(s));
        }
        if (!grid_dots(v, vmax)) {
            bail();
            return;
        }
    }
    const double f_start = warp_sum_nb(W.fpart, nb);
    if (tid == 0) {
        G.f = f_start;
        G.floor_reached = 0;
        G.gg = G.red[4 * kPfSlots + 1];
        G.gmax = G.red[kPfDots - 2];
        G.np = 0;
        for (int i = 0; i < kPfSlots; i++) G.slot[i] = i;
        pf_coefficients(G);
    }
    __syncthreads();

    int done = 0;
    for (int it = 0; it < Pp.iters; it++) {
        if (!(G.gmax > 0.0)) break;
        // ---- direction on my chunk ----
        {
            const double gam = G.gamma, ig = 1.0 / G.gmax;
            const int np = G.np, rs = G.restart;
            for (int k = k0 + tid; k < k1; k += nt) {
                double acc;
                if (rs) {
                    acc = W.g[k] * ig;
                } else {
                    acc = gam * W.g[k];
                    for (int i = 0; i < np; i++) {
                        const size_t sl = (size_t)G.slot[i] * P + k;
                        acc += G.c1[i] * Sg_[sl] + G.c2[i] * Yg_[sl];
                    }
                }
                W.p[k] = -acc;
            }
        }
        // ---- Armijo backtracking ----
        const double f0 = G.f, gp = G.gp;
        double a = 1.0, ft = 0.0;
        bool accepted = false;
        for (int h = 0; h <= 30; h++) {
            for (int k = k0 + tid; k < k1; k += nt) W.phit[k] = W.phi[k] + a * W.p[k];
            write_u(W.phit);
            if (!grid_sync(Pp.sync, Pp.err, Pp.wait_spins, Pp.withhold_release)) {
        bail();
        return;
    }
            pf_eval(Pp, W, g, twy, twx, red, out, ex);
            if (!grid_sync(Pp.sync, Pp.err, Pp.wait_spins, Pp.withhold_release)) {
        bail();
        return;
    }
            ft = warp_sum_nb(W.fpart, nb);
            if (ft <= f0 + 1e-4 * a * gp) {
                accepted = true;
                break;
            }
            a *= 0.5;
        }
        if (!accepted) break;
        // ---- accept: new gradient, pair and dot products on my chunk ----
        {
            const int np = G.np, ns = G.slot[np];
            pf_part_sums(W.part, nb, P, k0, k1, W.gsum);
            __syncthreads();
            double v[kPfDots] = {0.0};
            double vmax = 0.0;
            for (int k = k0 + tid; k < k1; k += nt) {
                const double gn = W.gsum[k];
                const double sv = W.phit[k] - W.phi[k], yv = gn - W.g[k];
                Sg_[(size_t)ns * P + k] = sv;
                Yg_[(size_t)ns * P + k] = yv;
                W.phi[k] = W.phit[k];
                W.g[k] = gn;
                for (int i = 0; i <= np; i++) {
                    const size_t sl = (size_t)G.slot[i] * P + k;
                    const double si = Sg_[sl], yi = Yg_[sl];
                    v[4 * i + 0] += si * yv;
                    v[4 * i + 1] += yi * yv;
                    v[4 * i + 2] += si * gn;
                    v[4 * i + 3] += yi * gn;
                }
                v[4 * kPfSlots + 0] += sv * sv;
                v[4 * kPfSlots + 1] += gn * gn;
                vmax = fmax(vmax, fabs(gn));
            }
            if (!grid_dots(v, vmax)) {
            bail();
            return;
        }
            if (tid == 0) {
                const double *t = G.red;
                for (int i = 0; i <= np; i++) {
                    G.SY[i][np] = t[4 * i + 0];
                    G.YY[i][np] = t[4 * i + 1];
                    G.Sg[i] = t[4 * i + 2];
                    G.Yg[i] = t[4 * i + 3];
                }
                const double sy = t[4 * np + 0], yy = t[4 * np + 1], ss = t[4 * kPfSlots + 0];
                G.gg = t[4 * kPfSlots + 1];
                G.gmax = t[kPfDots - 2];
                G.floor_reached = Pp.tol > 0.0 && G.f - ft <= Pp.tol * G.f;
                G.f = ft;
                if (sy > 1e-10 * sqrt(ss) * sqrt(yy) && sy > 0.0) {
                    G.rD[np] = 1.0 / sy;
                    G.np = np + 1;
                    if (G.np > m) {  // drop the oldest pair; its slot becomes the free one
                        const int s0 = G.slot[0];
                        for (int i = 0; i < m; i++) {
                            for (int j = i; j < m; j++) {
                                G.SY[i][j] = G.SY[i + 1][j + 1];
                                G.YY[i][j] = G.YY[i + 1][j + 1];
                            }
                            G.Sg[i] = G.Sg[i + 1];
                            G.Yg[i] = G.Yg[i + 1];
                            G.rD[i] = G.rD[i + 1];
                            G.slot[i] = G.slot[i + 1];
                        }
                        G.slot[m] = s0;
                        G.np = m;
                    }
                }
                pf_coefficients(G);
            }
            __syncthreads();
        }
        done = it + 1;
        if (G.floor_reached) break;
    }

    // ---- remove the free constant: arg(sum_k w_k e^{i phi_k}) = 0 ----
    {
        double v[kPfDots] = {0.0};
        for (int k = k0 + tid; k < k1; k += nt) {
            double s, c;
            sincos(W.phi[k], &s, &c);
            const double wk = Pp.wts ? (double)Pp.wts[k] : 1.0;
            v[0] += wk * c;
            v[1] += wk * s;
        }
        if (!grid_dots(v, 0.0)) {
            bail();
            return;
        }
        const double shift = atan2(G.red[1], G.red[0]);
        for (int k = k0 + tid; k < k1; k += nt) Pp.phi[k] = W.phi[k] - shift;
        if (blockIdx.x == 0 && tid == 0) {
            if (Pp.iters_done) *Pp.iters_done = done;
            if (Pp.loss_out) *Pp.loss_out = G.f;
        }
    }
}

// dynamic shared memory of k_phase_fit: 1 grid (kind 0) or 3 (kind 1), the
// twiddles, the ramps and the reduction scratch
static size_t phase_fit_smem(int ny, int nx, int kind)
{
    const int ngrid = kind == 1 ? 3 : 1;
    return sizeof(float2) * ((size_t)ngrid * ny * (nx + 1) + ny / 2 + nx / 2 + ny + nx + 1) +
           sizeof(double) * (32 * kPfDots + kPfDots + 8) + 64;
}

bool phase_fit2x_fits(int ny, int nx) { return phase_fit_smem(ny, nx, 1) + sizeof(PFGram) + 1024 <= 227 * 1024; }

cudaError_t launch_phase_fit(const PhaseFitParams &p, cudaStream_t s)
{
    const int grid = phase_fit_grid(p.ny, p.nx, p.Nd);
    const int P = p.ny * p.nx;
    const size_t sm = phase_fit_smem(p.ny, p.nx, p.kind);
    (void)P;
    cudaError_t e = cudaFuncSetAttribute(k_phase_fit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_phase_fit, 512, sm);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    PhaseFitParams pp = p;
    void *args[] = {&pp};
    return cudaLaunchCooperativeKernel((const void *)k_phase_fit, dim3(grid), dim3(512), args, sm, s);
}

}  // namespace tmr
