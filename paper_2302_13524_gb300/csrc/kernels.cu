// kernels.cu -- fused forward-model and gradient kernels, defocus fields,
// phase application, and the host-side FFT twiddle tables.
//
// Forward model (Eq. optTMsmall2): one CTA per (row, mask) computes
// z = F(d_j .* t) in registers and writes |z|^2.  Gradient (Eq. derivative,
// App. A): one CTA per row loops over the J masks, keeping the accumulated
// Q^H(z .* r) in registers: forward FFT, residual r = y - |z|^2 and its square
// sum, inverse FFT of z .* r, multiply by conj(d_j), accumulate; g = -4 * acc.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"

namespace tmr {

#define TMR_DISPATCH_N(NVAR, ...)                \
    switch (NVAR) {                              \
    case 64: { constexpr int NN = 64; __VA_ARGS__; } break;     \
    case 128: { constexpr int NN = 128; __VA_ARGS__; } break;   \
    case 256: { constexpr int NN = 256; __VA_ARGS__; } break;   \
    case 512: { constexpr int NN = 512; __VA_ARGS__; } break;   \
    case 1024: { constexpr int NN = 1024; __VA_ARGS__; } break; \
    case 2048: { constexpr int NN = 2048; __VA_ARGS__; } break; \
    case 4096: { constexpr int NN = 4096; __VA_ARGS__; } break; \
    default: return cudaErrorInvalidValue;       \
    }

bool fft_supported(int N) { return N >= 64 && N <= 4096 && (N & (N - 1)) == 0; }

template <int N>
static int fft_table_t(float2 *out)
{
    using Pl = FftPlan<N, N / fft_threads(N)>;
    if (out) {
        for (int p = 1; p < Pl::P; p++) {
            const int R = Pl::radix(p), Ns = Pl::ns(p), off = Pl::tw_off(p);
            for (int r = 1; r < R; r++)
                for (int j = 0; j < Ns; j++) {
                    const double a = -2.0 * M_PI * (double)r * (double)j / ((double)Ns * R);
                    out[off + (r - 1) * Ns + j] = make_float2((float)std::cos(a), (float)std::sin(a));
                }
        }
    }
    return Pl::TW_SIZE;
}

static int fft_table_dispatch(int N, float2 *out)
{
    switch (N) {
    case 64: return fft_table_t<64>(out);
    case 128: return fft_table_t<128>(out);
    case 256: return fft_table_t<256>(out);
    case 512: return fft_table_t<512>(out);
    case 1024: return fft_table_t<1024>(out);
    case 2048: return fft_table_t<2048>(out);
    case 4096: return fft_table_t<4096>(out);
    default: return -1;
    }
}

int fft_table(int N, float2 *out) { return fft_table_dispatch(N, out); }
int fft_table_len(int N) { return fft_table_dispatch(N, nullptr); }

// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(fft_threads(N)) k_forward(const float2 *__restrict__ T,
                                                          const float2 *__restrict__ masks,
                                                          const float2 *__restrict__ twg,
                                                          float *__restrict__ Y, int J)
{
    constexpr int NT = fft_threads(N), E = N / NT, TWN = FftPlan<N, E>::TW_SIZE;
    extern __shared__ float2 smem[];
    float2 *buf = smem, *tw = smem + fft_buf_len(N);
    const int tid = threadIdx.x, row = blockIdx.x, j = blockIdx.y;
    for (int i = tid; i < TWN; i += NT) tw[i] = twg[i];
    float2 v[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        const int n = tid + e * NT;
        v[e] = cmul(T[(size_t)row * N + n], masks[(size_t)j * N + n]);
    }
    __syncthreads();
    block_fft<N, NT, -1>(v, buf, tw, tid);
    float *yr = Y + ((size_t)row * J + j) * N;
#pragma unroll
    for (int e = 0; e < E; e++) yr[tid + e * NT] = cabs2(v[e]);
}

template <int N>
__global__ void __launch_bounds__(fft_threads(N)) k_grad(const float2 *__restrict__ T,
                                                       const float2 *__restrict__ masks,
                                                       const float2 *__restrict__ twg,
                                                       const float *__restrict__ Y,
                                                       float *__restrict__ loss,
                                                       float2 *__restrict__ G, int J)
{
    constexpr int NT = fft_threads(N), E = N / NT, TWN = FftPlan<N, E>::TW_SIZE;
    extern __shared__ float2 smem[];
    float2 *buf = smem, *tw = smem + fft_buf_len(N);
    __shared__ float red[NT / 32], fsum[1];
    const int tid = threadIdx.x, row = blockIdx.x;
    for (int i = tid; i < TWN; i += NT) tw[i] = twg[i];
    float2 t[E], acc[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        t[e] = T[(size_t)row * N + tid + e * NT];
        acc[e] = make_float2(0.f, 0.f);
    }
    float f = 0.f;
    __syncthreads();
    for (int j = 0; j < J; j++) {
        const float2 *d = masks + (size_t)j * N;
        const float *y = Y + ((size_t)row * J + j) * N;
        float2 v[E];
#pragma unroll
        for (int e = 0; e < E; e++) v[e] = cmul(t[e], d[tid + e * NT]);
        block_fft<N, NT, -1>(v, buf, tw, tid);
#pragma unroll
        for (int e = 0; e < E; e++) {
            const float r = y[tid + e * NT] - cabs2(v[e]);
            f = fmaf(r, r, f);
            v[e] = cscale(v[e], r);
        }
        block_fft<N, NT, +1>(v, buf, tw, tid);
#pragma unroll
        for (int e = 0; e < E; e++) acc[e] = cadd(acc[e], cmulc(v[e], d[tid + e * NT]));
    }
    if (G) {
#pragma unroll
        for (int e = 0; e < E; e++) G[(size_t)row * N + tid + e * NT] = cscale(acc[e], -4.f);
    }
    float fv[1] = {f};
    block_sum<1>(fv, red, fsum);
    if (loss && tid == 0) loss[row] = fsum[0];
}

// Defocus fields: CTA (row, j) computes z_j = F(d_j .* t) and keeps the
// entries whose pattern index j*N + k is below Nd.
template <int N>
__global__ void __launch_bounds__(fft_threads(N)) k_fields(const float2 *__restrict__ T,
                                                         const float2 *__restrict__ masks,
                                                         const float2 *__restrict__ twg,
                                                         float2 *__restrict__ Zd, int M, int Nd)
{
    constexpr int NT = fft_threads(N), E = N / NT, TWN = FftPlan<N, E>::TW_SIZE;
    extern __shared__ float2 smem[];
    float2 *buf = smem, *tw = smem + fft_buf_len(N);
    const int tid = threadIdx.x, row = blockIdx.x, j = blockIdx.y;
    for (int i = tid; i < TWN; i += NT) tw[i] = twg[i];
    float2 v[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        const int n = tid + e * NT;
        v[e] = cmul(T[(size_t)row * N + n], masks[(size_t)j * N + n]);
    }
    __syncthreads();
    block_fft<N, NT, -1>(v, buf, tw, tid);
#pragma unroll
    for (int e = 0; e < E; e++) {
        const int pat = j * N + tid + e * NT;
        if (pat < Nd) Zd[(size_t)pat * M + row] = v[e];
    }
}

// T[r] *= e^{i phi[r]}: one CTA per row (strided), the phase factor made once per row.
__global__ void k_apply_phase(int N, int M, const double *__restrict__ phi,
                              const float2 *__restrict__ Tin, float2 *__restrict__ Tout)
{
    __shared__ float2 u;
    for (int r = blockIdx.x; r < M; r += gridDim.x) {
        if (threadIdx.x == 0) {
            double s, c;
            sincos(phi[r], &s, &c);
            u = make_float2((float)c, (float)s);
        }
        __syncthreads();
        const float2 ur = u;
        for (int n = threadIdx.x; n < N; n += blockDim.x)
            Tout[(size_t)r * N + n] = cmul(Tin[(size_t)r * N + n], ur);
        __syncthreads();
    }
}

__global__ void k_row_energy(int N, int M, const float2 *__restrict__ T, float *__restrict__ w)
{
    const int r = blockIdx.x;
    float s = 0.f;
    for (int n = threadIdx.x; n < N; n += blockDim.x) s += cabs2(T[(size_t)r * N + n]);
    __shared__ float red[32], out[1];
    float v[1] = {s};
    block_sum<1>(v, red, out);
    if (threadIdx.x == 0) w[r] = out[0];
}

// ---------------------------------------------------------------------------
template <int N>
static size_t fft_kernel_smem() { return sizeof(float2) * (fft_buf_len(N) + FftPlan<N, N / fft_threads(N)>::TW_SIZE); }

cudaError_t launch_forward(int N, int M, int J, const float2 *T, const float2 *masks,
                           const float2 *tw, float *Y, cudaStream_t s)
{
    if (M == 0) return cudaSuccess;
    TMR_DISPATCH_N(N, {
        const size_t sm = fft_kernel_smem<NN>();
        cudaFuncSetAttribute(k_forward<NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_forward<NN><<<dim3(M, J), fft_threads(NN), sm, s>>>(T, masks, tw, Y, J);
    });
    return cudaGetLastError();
}

cudaError_t launch_grad(int N, int M, int J, const float2 *T, const float2 *masks,
                        const float2 *tw, const float *Y, float *loss, float2 *G, cudaStream_t s)
{
    if (M == 0) return cudaSuccess;
    TMR_DISPATCH_N(N, {
        const size_t sm = fft_kernel_smem<NN>();
        cudaFuncSetAttribute(k_grad<NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_grad<NN><<<M, fft_threads(NN), sm, s>>>(T, masks, tw, Y, loss, G, J);
    });
    return cudaGetLastError();
}

cudaError_t launch_fields(int N, int M, int J, int Nd, const float2 *T, const float2 *masks,
                          const float2 *tw, float2 *Zd, cudaStream_t s)
{
    if (M == 0 || Nd == 0) return cudaSuccess;
    const int Jn = (Nd + N - 1) / N < J ? (Nd + N - 1) / N : J;
    TMR_DISPATCH_N(N, {
        const size_t sm = fft_kernel_smem<NN>();
        cudaFuncSetAttribute(k_fields<NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_fields<NN><<<dim3(M, Jn), fft_threads(NN), sm, s>>>(T, masks, tw, Zd, M, Nd);
    });
    return cudaGetLastError();
}

cudaError_t launch_apply_phase(int N, int M, const double *phi, const float2 *Tin, float2 *Tout,
                               cudaStream_t s)
{
    if (M == 0) return cudaSuccess;
    const int blocks = M < 152 * 16 ? M : 152 * 16;
    k_apply_phase<<<blocks, 256, 0, s>>>(N, M, phi, Tin, Tout);
    return cudaGetLastError();
}

// y[i] = -ln(u) with u uniform in (0, 1] from a counter hash: exponential
// intensities with mean 1, like fully developed speckle.
__global__ void k_fill_synthetic(float *y, size_t n, unsigned seed)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const uint4 o = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), seed, 7u), make_uint2(seed, 11u));
        const float u = fmaf((float)o.x, 0x1p-32f, 0x1p-33f);
        y[i] = -logf(u);
    }
}

cudaError_t launch_fill_synthetic(float *y, size_t n, unsigned seed, cudaStream_t s)
{
    k_fill_synthetic<<<512, 256, 0, s>>>(y, n, seed);
    return cudaGetLastError();
}

cudaError_t launch_row_energy(int N, int M, const float2 *T, float *w, cudaStream_t s)
{
    if (M == 0) return cudaSuccess;
    k_row_energy<<<M, 256, 0, s>>>(N, M, T, w);
    return cudaGetLastError();
}

}  // namespace tmr
