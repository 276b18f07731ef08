// kernels.cu -- fused forward-model and gradient kernels, defocus fields,
// phase application, and the host-side FFT twiddle tables.
//
// Forward model (Eq. optTMsmall2): one CTA per (row, mask) computes
// z = F(d_j .* t) in registers and writes |z|^2.  Gradient (Eq. derivative,
// App. A): one CTA per row loops over the J masks, keeping the accumulated
// Q^H(z .* r) in registers: forward FFT, residual r = y - |z|^2 and its square
// sum, inverse FFT of z .* r, multiply by conj(d_j), accumulate; g = -4 * acc.
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include <cuda_fp16.h>

#include "common.cuh"
#include "cost.cuh"
#include "fft.cuh"
#include "internal.h"
#include "xform.cuh"

namespace tmr {

bool fft_supported(int N) { return N >= 64 && N <= 4096 && (N & (N - 1)) == 0; }

bool xform_blue_shape(int N, int *L, int *ne)
{
    if (N < 16 || N > 4096 || fft_supported(N)) return false;
    if (N > 2048 && N <= kBlueSplitMaxN) {  // split outputs at L = 4096 (XfBlueSplit)
        *L = 4096;
        *ne = (N + 511) / 512;
        return true;
    }
    int l = 512;
    while (l < 2 * N - 1) l *= 2;
    if (l > 8192) return false;
    const int nt = l / 16;
    const int need = (N + nt - 1) / nt;
    *L = l;
    *ne = l == 8192 ? need : 8;  // exact register count where it matters (largest L)
    return need <= *ne;
}

bool xform_supported(int N)
{
    int L, ne;
    return fft_supported(N) || xform_blue_shape(N, &L, &ne);
}

// Twiddles of passes 1 .. P-1 (npass = P) or 1 .. P-2 (npass = P - 1) of a plan.
template <class Pl>
static int plan_table(float2 *out, int npass)
{
    if (out) {
        for (int p = 1; p < npass; p++) {
            const int R = Pl::radix(p), Ns = Pl::ns(p), off = Pl::tw_off(p);
            for (int r = 1; r < R; r++)
                for (int j = 0; j < Ns; j++) {
                    const double a = -2.0 * M_PI * (double)r * (double)j / ((double)Ns * R);
                    out[off + (r - 1) * Ns + j] = make_float2((float)std::cos(a), (float)std::sin(a));
                }
        }
    }
    return Pl::tw_off(npass);
}

template <int N>
static int fft_table_t(float2 *out)
{
    using Pl = FftPlan<N, N / fft_threads(N)>;
    return plan_table<Pl>(out, Pl::P);
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

// In-place FP64 radix-2 DFT X_k = sum_m x_m exp(-2 pi i k m / n), n a power of two.
static void host_fft(std::vector<std::complex<double>> &x)
{
    const size_t n = x.size();
    for (size_t i = 1, j = 0; i < n; i++) {  // bit reversal
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(x[i], x[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        for (size_t k = 0; k < len / 2; k++) {
            const double a = -2.0 * M_PI * (double)k / (double)len;
            const std::complex<double> w(std::cos(a), std::sin(a));
            for (size_t i = 0; i < n; i += len) {
                const std::complex<double> u = x[i + k], v = x[i + k + len / 2] * w;
                x[i + k] = u + v;
                x[i + k + len / 2] = u - v;
            }
        }
    }
}

template <int L, int NE>
static int blue_table(int N, float2 *out)
{
    using X = XfBlue<L, NE>;
    const int len = X::NCONST + N;
    if (!out) return len;
    plan_table<typename X::Plan>(out, X::Plan::P - 1);
    // exp(i pi s m^2 / N) with m^2 reduced mod 2N (exact)
    auto chirp = [N](long long m, double s) {
        const double a = s * M_PI * (double)((m * m) % (2LL * N)) / (double)N;
        return std::complex<double>(std::cos(a), std::sin(a));
    };
    std::vector<std::complex<double>> b(L, 0.0);
    for (int m = 0; m < N; m++) {
        b[m] = chirp(m, +1.0);
        if (m > 0) b[L - m] = b[m];
    }
    host_fft(b);
    for (int k = 0; k <= L / 2; k++) {
        const std::complex<double> v = b[k] / (double)L;
        out[X::NCONST_TW + k] = make_float2((float)v.real(), (float)v.imag());
    }
    for (int n = 0; n < N; n++) {
        const std::complex<double> c = chirp(n, -1.0);
        out[X::NCONST + n] = make_float2((float)c.real(), (float)c.imag());
    }
    return len;
}

// [twiddles | B_1 | B_2 | chirp] of the split-output transform (XfBlueSplit)
template <int NE>
static int blue_split_table(int N, float2 *out)
{
    using X = XfBlueSplit<NE>;
    constexpr int L = X::L;
    const int len = X::NCONST + N;
    if (!out) return len;
    std::vector<float2> full(fft_table_len(L));
    fft_table(L, full.data());
    for (int i = 0; i < X::NCONST_TW; i++) out[i] = full[i];
    auto chirp = [N](long long m, double sgn) {
        const long long q = (m * m) % (2LL * N);
        const double a = sgn * M_PI * (double)q / (double)N;
        return std::complex<double>(std::cos(a), std::sin(a));
    };
    const int H = (N + 1) / 2;
    for (int half = 0; half < 2; half++) {
        // b_m = exp(i pi m^2 / N) on the half's range of k - n
        const int m0 = half == 0 ? -(N - 1) : H - (N - 1), m1 = half == 0 ? H - 1 : N - 1;
        std::vector<std::complex<double>> b(L, 0.0);
        for (int m = m0; m <= m1; m++) b[((m % L) + L) % L] = chirp(m < 0 ? -m : m, +1.0);
        host_fft(b);
        for (int k = 0; k < L; k++) {
            const std::complex<double> v = b[k] / (double)L;
            out[X::NCONST_TW + half * L + k] = make_float2((float)v.real(), (float)v.imag());
        }
    }
    for (int n = 0; n < N; n++) {
        const std::complex<double> c = chirp(n, -1.0);
        out[X::NCONST + n] = make_float2((float)c.real(), (float)c.imag());
    }
    return len;
}

int xform_table(int N, float2 *out)
{
    if (fft_supported(N)) return fft_table(N, out);
    int L, ne;
    if (!xform_blue_shape(N, &L, &ne)) return -1;
    if (N > 2048 && L == 4096) return ne == 5 ? blue_split_table<5>(N, out) : blue_split_table<6>(N, out);
    switch (L) {
    case 512: return blue_table<512, 8>(N, out);
    case 1024: return blue_table<1024, 8>(N, out);
    case 2048: return blue_table<2048, 8>(N, out);
    case 4096: return blue_table<4096, 8>(N, out);
    default: break;
    }
    switch (ne) {  // the constants do not depend on the register count
    case 6: return blue_table<8192, 6>(N, out);
    case 7: return blue_table<8192, 7>(N, out);
    default: return blue_table<8192, 8>(N, out);
    }
}

// Tables of XfPow2D<N> (the 2D probing DFT, xform.cuh): the twiddles of
// passes 1 .. P-2 with boundary B = n1 (forward) and B = N / n1 (adjoint):
// W_{Ns R}^{r j} for passes with Ns < B, W_{(Ns/B) R}^{r (j div B)} for the
// others; then the entry (n1, N / n1).
template <int N>
static int fft_table_2d_t(int n1, float2 *out)
{
    using Pl = FftPlan<N, N / fft_threads(N)>;
    const int tws = Pl::tw_off(Pl::P - 1);
    if (out) {
        for (int half = 0; half < 2; half++) {
            const int B = half == 0 ? n1 : N / n1;
            for (int p = 1; p < Pl::P - 1; p++) {
                const int R = Pl::radix(p), Ns = Pl::ns(p), off = Pl::tw_off(p);
                for (int r = 1; r < R; r++)
                    for (int j = 0; j < Ns; j++) {
                        const double a = Ns >= B ? -2.0 * M_PI * (double)r * (double)(j / B) / ((double)(Ns / B) * R)
                                                 : -2.0 * M_PI * (double)r * (double)j / ((double)Ns * R);
                        out[half * tws + off + (r - 1) * Ns + j] = make_float2((float)std::cos(a), (float)std::sin(a));
                    }
            }
        }
        out[2 * tws] = make_float2((float)n1, (float)(N / n1));
    }
    return 2 * tws + 1;
}

int fft_table_2d(int N, int n1, float2 *out)
{
    if (!probe_2d_boundary(N, n1) || !probe_2d_boundary(N, N / n1)) return -1;
    return N == 512 ? fft_table_2d_t<512>(n1, out) : fft_table_2d_t<4096>(n1, out);
}

int xform_table_blue_full(int N, float2 *out)
{
    if (N <= 2048 || N > kBlueSplitMaxN) return -1;
    return blue_table<8192, 6>(N, out);  // the constants do not depend on the register count
}

bool mixed_supported(int N) { return N == 256 || N == 1024 || N == 2048 || N == 4096; }

// Round to the nearest BF16 (ties to even); returns the bits.
static uint16_t host_bf16(float v)
{
    uint32_t u;
    std::memcpy(&u, &v, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

static float host_bf16_value(uint16_t b)
{
    const uint32_t u = (uint32_t)b << 16;
    float v;
    std::memcpy(&v, &u, 4);
    return v;
}

// m16n8k16 A fragments of a 16 x 16 tile given element by element: word w of
// lane (g, t) holds rows g + 8 (w & 1), columns 2t + 8 (w >> 1) + {0, 1}, the
// lower column in the low half; part 0 = hi, 1 = lo of the BF16 split.
template <class F>
static void write_frag(uint32_t *dst, int part, F &&elem)
{
    for (int lane = 0; lane < 32; lane++) {
        const int g = lane >> 2, t = lane & 3;
        for (int w = 0; w < 4; w++) {
            uint32_t word = 0;
            for (int h = 0; h < 2; h++) {
                const double v = elem(g + 8 * (w & 1), 2 * t + 8 * (w >> 1) + h);
                const uint16_t hi = host_bf16((float)v);
                const uint16_t lo = host_bf16((float)(v - (double)host_bf16_value(hi)));
                word |= (uint32_t)(part == 0 ? hi : lo) << (16 * h);
            }
            dst[lane * 4 + w] = word;
        }
    }
}

template <int N>
static int mixed_table(float2 *out)
{
    using X = XfMixed<N>;
    if (!out) return X::NCONST;
    std::vector<float2> full(fft_table_len(N));
    fft_table(N, full.data());
    for (int i = 0; i < X::OFF_FRAG16; i++) out[i] = full[i];
    auto cs = [](int q, int r, int R, bool sine) {
        const double a = 2.0 * M_PI * (double)((q * r) % R) / (double)R;
        return sine ? std::sin(a) : std::cos(a);
    };
    // radix 16: blocks C, S, -S of the 16-point DFT (row q = output, column r = input)
    uint32_t *f16 = reinterpret_cast<uint32_t *>(out + X::OFF_FRAG16);
    for (int tile = 0; tile < kTcTiles16; tile++) {
        const int kind = tile / 2;  // 0 C, 1 S, 2 -S
        write_frag(f16 + tile * 128, tile % 2, [&](int q, int r) {
            return kind == 0 ? cs(q, r, 16, false) : (kind == 1 ? cs(q, r, 16, true) : -cs(q, r, 16, true));
        });
    }
    // radix 8: the whole real form [[C, sS], [-sS, C]] (s = +1 forward, -1 inverse),
    // rows 0-7 Re y_q, 8-15 Im y_q; columns 0-7 Re x_r, 8-15 Im x_r
    uint32_t *f8 = reinterpret_cast<uint32_t *>(out + X::OFF_FRAG8);
    for (int tile = 0; tile < kTcTiles8; tile++) {
        const double sgn = tile / 2 == 0 ? 1.0 : -1.0;
        write_frag(f8 + tile * 128, tile % 2, [&](int row, int col) {
            const int q = row & 7, r = col & 7;
            const bool re_out = row < 8, re_in = col < 8;
            if (re_out == re_in) return cs(q, r, 8, false);
            return (re_out ? sgn : -sgn) * cs(q, r, 8, true);
        });
    }
    for (int k = 0; k < N; k++) {
        const double a = -2.0 * M_PI * (double)k / (double)N;
        out[X::OFF_ROOT + k] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    return X::NCONST;
}

int xform_table_prec(int N, int prec, float2 *out)
{
    if (prec == 0) return xform_table(N, out);
    switch (N) {
    case 256: return mixed_table<256>(out);
    case 1024: return mixed_table<1024>(out);
    case 2048: return mixed_table<2048>(out);
    case 4096: return mixed_table<4096>(out);
    default: return -1;
    }
}

// Calls f(Xf{}) with the transform policy of length N and kind prec (0: FP32
// with the 1D probing DFT, 1: mixed precision, 2: FP32 with the 2D probing DFT).
template <class F>
static cudaError_t dispatch_xf(int N, int prec, F &&f)
{
    if (prec == 2) {  // the 2D probing DFT
        switch (N) {
        case 512: return f(XfPow2D<512>{});
        case 4096: return f(XfPow2D<4096>{});
        default: return cudaErrorInvalidValue;
        }
    }
    if (prec != 0) {
        switch (N) {
        case 256: return f(XfMixed<256>{});
        case 1024: return f(XfMixed<1024>{});
        case 2048: return f(XfMixed<2048>{});
        case 4096: return f(XfMixed<4096>{});
        default: return cudaErrorInvalidValue;
        }
    }
    switch (N) {
    case 64: return f(XfPow2<64>{});
    case 128: return f(XfPow2<128>{});
    case 256: return f(XfPow2<256>{});
    case 512: return f(XfPow2<512>{});
    case 1024: return f(XfPow2<1024>{});
    case 2048: return f(XfPow2<2048>{});
    case 4096: return f(XfPow2<4096>{});
    default: break;
    }
    int L, ne;
    if (!xform_blue_shape(N, &L, &ne)) return cudaErrorInvalidValue;
    if (N > 2048 && L == 4096) return ne == 5 ? f(XfBlueSplit<5>{}) : f(XfBlueSplit<6>{});
    switch (L) {
    case 512: return f(XfBlue<512, 8>{});
    case 1024: return f(XfBlue<1024, 8>{});
    case 2048: return f(XfBlue<2048, 8>{});
    case 4096: return f(XfBlue<4096, 8>{});
    default: break;
    }
    switch (ne) {  // L = 8192: N in (2731, 4096], 6..8 registers
    case 6: return f(XfBlue<8192, 6>{});
    case 7: return f(XfBlue<8192, 7>{});
    default: return f(XfBlue<8192, 8>{});
    }
}

// ---------------------------------------------------------------------------
// Kernels over a transform policy Xf (xform.cuh); shared memory holds the
// exchange buffer (Xf::LBUF) and the transform's shared constants.
template <class Xf>
__global__ void __launch_bounds__(Xf::NT) k_forward(int N, const float2 *__restrict__ T,
                                                    const float2 *__restrict__ masks,
                                                    const float2 *__restrict__ cg,
                                                    float *__restrict__ Y, int J)
{
    constexpr int NT = Xf::NT, E = Xf::NE;
    extern __shared__ float2 smem[];
    float2 *buf = smem, *cst = smem + Xf::BUFS * Xf::LBUF;
    const int tid = threadIdx.x, row = blockIdx.x, j = blockIdx.y;
    for (int i = tid; i < Xf::shared_consts(N); i += NT) cst[i] = cg[i];
    Xf xf;
    xf.setup(masks + (size_t)j * N, cg + Xf::NCONST, N, tid);
    float2 v[E];
#pragma unroll
    for (int e = 0; e < E; e++)
        v[e] = Xf::valid(e, tid, N) ? T[(size_t)row * N + tid + e * NT] : make_float2(0.f, 0.f);
    __syncthreads();
    xf.fwd(v, buf, cst, tid);
    float *yr = Y + ((size_t)row * J + j) * N;
#pragma unroll
    for (int e = 0; e < E; e++)
        if (Xf::valid(e, tid, N)) yr[tid + e * NT] = cabs2(v[e]);
}

template <class Xf>
__global__ void __launch_bounds__(Xf::NT) k_grad(int N, const float2 *__restrict__ T,
                                                 const float2 *__restrict__ masks,
                                                 const float2 *__restrict__ cg,
                                                 const float *__restrict__ Y,
                                                 float *__restrict__ loss,
                                                 float2 *__restrict__ G, int J, int cost)
{
    constexpr int NT = Xf::NT, E = Xf::NE;
    extern __shared__ float2 smem[];
    float2 *buf = smem, *cst = smem + Xf::BUFS * Xf::LBUF;
    __shared__ float red[NT / 32 > 0 ? NT / 32 : 1], fsum[1];
    const int tid = threadIdx.x, row = blockIdx.x;
    for (int i = tid; i < Xf::shared_consts(N); i += NT) cst[i] = cg[i];
    float2 t[E], acc[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        t[e] = Xf::valid(e, tid, N) ? T[(size_t)row * N + tid + e * NT] : make_float2(0.f, 0.f);
        acc[e] = make_float2(0.f, 0.f);
    }
    float f = 0.f;
    __syncthreads();
    for (int j = 0; j < J; j++) {
        Xf xf;
        xf.setup(masks + (size_t)j * N, cg + Xf::NCONST, N, tid);
        __syncthreads();  // a fresh policy restarts the exchange-buffer alternation
        const float *y = Y + ((size_t)row * J + j) * N;
        float2 v[E];
#pragma unroll
        for (int e = 0; e < E; e++) v[e] = t[e];
        xf.fwd(v, buf, cst, tid);
#pragma unroll
        for (int e = 0; e < E; e++) {
            if (cost == COST_AMPLITUDE) {
                const float c = Xf::valid(e, tid, N) ? cost_coef(cost, v[e], y[tid + e * NT], f) : 0.f;
                v[e] = cscale(v[e], c);
            } else {
                const float r = Xf::valid(e, tid, N) ? y[tid + e * NT] - cabs2(v[e]) : 0.f;
                f = fmaf(r, r, f);
                v[e] = cscale(v[e], r);
            }
        }
        xf.adj(v, buf, cst, tid);
#pragma unroll
        for (int e = 0; e < E; e++) acc[e] = cadd(acc[e], v[e]);
    }
    if (G) {
#pragma unroll
        for (int e = 0; e < E; e++)
            if (Xf::valid(e, tid, N)) G[(size_t)row * N + tid + e * NT] = cscale(acc[e], cost_grad_scale(cost));
    }
    float fv[1] = {f};
    block_sum<1>(fv, red, fsum);
    if (loss && tid == 0) loss[row] = fsum[0];
}

// Defocus fields: CTA (row, j) computes z_j = F(d_j .* t) and keeps the
// entries whose pattern index j*N + k is below Nd.
template <class Xf>
__global__ void __launch_bounds__(Xf::NT) k_fields(int N, const float2 *__restrict__ T,
                                                   const float2 *__restrict__ masks,
                                                   const float2 *__restrict__ cg,
                                                   float2 *__restrict__ Zd, int M, int Nd)
{
    constexpr int NT = Xf::NT, E = Xf::NE;
    extern __shared__ float2 smem[];
    float2 *buf = smem, *cst = smem + Xf::BUFS * Xf::LBUF;
    const int tid = threadIdx.x, row = blockIdx.x, j = blockIdx.y;
    for (int i = tid; i < Xf::shared_consts(N); i += NT) cst[i] = cg[i];
    Xf xf;
    xf.setup(masks + (size_t)j * N, cg + Xf::NCONST, N, tid);
    float2 v[E];
#pragma unroll
    for (int e = 0; e < E; e++)
        v[e] = Xf::valid(e, tid, N) ? T[(size_t)row * N + tid + e * NT] : make_float2(0.f, 0.f);
    __syncthreads();
    xf.fwd(v, buf, cst, tid);
#pragma unroll
    for (int e = 0; e < E; e++) {
        const int pat = j * N + tid + e * NT;
        if (Xf::valid(e, tid, N) && pat < Nd) Zd[(size_t)pat * M + row] = v[e];
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
template <class Xf>
static size_t xf_kernel_smem(int N) { return sizeof(float2) * (Xf::BUFS * Xf::LBUF + Xf::shared_consts(N)); }

cudaError_t launch_forward(int N, int M, int J, const float2 *T, const float2 *masks,
                           const float2 *tw, float *Y, cudaStream_t s, int prec)
{
    if (M == 0) return cudaSuccess;
    return dispatch_xf(N, prec, [&](auto xf) {
        using XF = decltype(xf);
        const size_t sm = xf_kernel_smem<XF>(N);
        cudaFuncSetAttribute(k_forward<XF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_forward<XF><<<dim3(M, J), XF::NT, sm, s>>>(N, T, masks, tw, Y, J);
        return cudaGetLastError();
    });
}

cudaError_t launch_grad(int N, int M, int J, const float2 *T, const float2 *masks,
                        const float2 *tw, const float *Y, float *loss, float2 *G, cudaStream_t s,
                        int prec, int cost)
{
    if (M == 0) return cudaSuccess;
    return dispatch_xf(N, prec, [&](auto xf) {
        using XF = decltype(xf);
        const size_t sm = xf_kernel_smem<XF>(N);
        cudaFuncSetAttribute(k_grad<XF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_grad<XF><<<M, XF::NT, sm, s>>>(N, T, masks, tw, Y, loss, G, J, cost);
        return cudaGetLastError();
    });
}

cudaError_t launch_fields(int N, int M, int J, int Nd, const float2 *T, const float2 *masks,
                          const float2 *tw, float2 *Zd, cudaStream_t s, int prec)
{
    if (M == 0 || Nd == 0) return cudaSuccess;
    const int Jn = (Nd + N - 1) / N < J ? (Nd + N - 1) / N : J;
    return dispatch_xf(N, prec, [&](auto xf) {
        using XF = decltype(xf);
        const size_t sm = xf_kernel_smem<XF>(N);
        cudaFuncSetAttribute(k_fields<XF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_fields<XF><<<dim3(M, Jn), XF::NT, sm, s>>>(N, T, masks, tw, Zd, M, Nd);
        return cudaGetLastError();
    });
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

// One CTA per row: the largest |y| of the row, then y / max rounded to FP16
// (rows of zeros keep scale 1; a non-finite value makes the scale non-finite,
// which the solver reports as a numeric row).
__global__ void k_pack_f16(size_t K, const float *__restrict__ y, __half *__restrict__ y16,
                           float *__restrict__ ysc)
{
    const size_t row = blockIdx.x;
    const float *yr = y + row * K;
    float mx = 0.f;
    for (size_t i = threadIdx.x; i < K; i += blockDim.x) {
        const float v = fabsf(yr[i]);
        mx = (v > mx || v != v) ? v : mx;
    }
    __shared__ float red[32], out[1];
    for (int o = 16; o > 0; o >>= 1) {
        const float v = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = (v > mx || v != v) ? v : mx;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) m = (red[w] > m || red[w] != red[w]) ? red[w] : m;
        out[0] = m > 0.f ? m : (m == 0.f ? 1.f : m);
        ysc[row] = out[0];
    }
    __syncthreads();
    const float inv = 1.f / out[0];
    __half *o16 = y16 + row * K;
    for (size_t i = threadIdx.x; i < K; i += blockDim.x) o16[i] = __float2half_rn(yr[i] * inv);
}

cudaError_t launch_pack_f16(int M, size_t K, const float *y, void *y16, float *ysc, cudaStream_t s)
{
    if (M == 0) return cudaSuccess;
    k_pack_f16<<<M, 512, 0, s>>>(K, y, (__half *)y16, ysc);
    return cudaGetLastError();
}

cudaError_t launch_row_energy(int N, int M, const float2 *T, float *w, cudaStream_t s)
{
    if (M == 0) return cudaSuccess;
    k_row_energy<<<M, 256, 0, s>>>(N, M, T, w);
    return cudaGetLastError();
}

}  // namespace tmr
