// fft.cuh -- block-level complex FFT of length N = 2^L held in registers.
//
// A team of T threads computes one length-N transform; thread `tid` holds
// E = N / T elements in the "thread-strided" layout: register e <-> index
// tid + e*T.  Input and output both use this layout, so a forward transform's
// output can be consumed elementwise and fed straight into an inverse
// transform without a shared-memory round trip.
//
// Passes follow the Stockham autosort formulation: N = R_0 * E^(P-1) with the
// small remainder radix first.  In pass p (radix R, stride Ns = product of the
// earlier radices) butterfly b reads x[b + r N/R], multiplies by
// W_{Ns R}^{r (b mod Ns)}, takes an R-point DFT and writes its outputs to
// (b div Ns) Ns R + (b mod Ns) + q Ns.  Every pass but the last exchanges
// through a padded shared buffer (one float2 of padding per 16, which keeps the
// strided writes of the early passes free of bank conflicts); the last pass's
// outputs land in the thread-strided layout directly.
//
// Twiddles come from a table with one block per pass p >= 1:
// tw_p[(r-1) Ns + j] = exp(-2 pi i r j / (Ns R)), r = 1..R-1, j = 0..Ns-1,
// computed in FP64 and rounded to FP32: on the host for a handle
// (tmr::fft_table), on the device for the allocation-free entry point
// (noalloc.cu; the two agree to 1 ulp of FP32) and, for its radix-16 plans,
// by the one-CTA-per-row solver (solver_row.cuh).  A thread reads its row j
// contiguously across the warp.
#pragma once

#include "common.cuh"

namespace tmr {

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x / 2); }
__host__ __device__ constexpr int ipowc(int b, int e) { return e == 0 ? 1 : b * ipowc(b, e - 1); }

// Threads per transform for length N: one warp at least, eight points each
// above that.
__host__ __device__ constexpr int fft_threads(int N) { return N / 8 < 32 ? 32 : N / 8; }

// E points per thread, radix R (a power of two dividing E) in every pass but
// the first; by default R = E (one butterfly per thread and pass).
template <int N, int E, int R = E>
struct FftPlan {
    static constexpr int LN = ilog2c(N), LE = ilog2c(R);
    static constexpr int P = (LN + LE - 1) / LE;  // number of passes
    static constexpr int LR0 = LN - (P - 1) * LE; // log2 of the first radix
    __host__ __device__ static constexpr int radix(int p) { return p == 0 ? (1 << LR0) : R; }
    __host__ __device__ static constexpr int ns(int p) { return p == 0 ? 1 : (1 << LR0) * ipowc(R, p - 1); }
    // offset (in float2) of pass p's twiddle block in the table
    __host__ __device__ static constexpr int tw_off(int p)
    {
        return p <= 1 ? 0 : tw_off(p - 1) + (radix(p - 1) - 1) * ns(p - 1);
    }
    static constexpr int TW_SIZE = tw_off(P);  // total table length
    static constexpr int TW_SMALL = P >= 2 ? tw_off(P - 1) : 0;  // without the last pass
};

__host__ __device__ __forceinline__ constexpr int fft_pad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int fft_buf_len(int N) { return N + N / 16; }

// Multiply by the quarter turn W_4 = exp(SIGN i pi / 2): -i for the forward sign.
template <int SIGN>
__device__ __forceinline__ float2 rot4(float2 a)
{
    return SIGN < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// In-place R-point DFT, X[k] = sum_n x[n] exp(SIGN 2 pi i k n / R), natural order.
template <int R, int SIGN>
__device__ __forceinline__ void dft_small(float2 (&x)[R])
{
    if constexpr (R == 1) {
    } else if constexpr (R == 2) {
        const float2 a = x[0], b = x[1];
        x[0] = cadd(a, b);
        x[1] = csub(a, b);
    } else if constexpr (R == 4) {
        const float2 a0 = cadd(x[0], x[2]), a1 = csub(x[0], x[2]);
        const float2 a2 = cadd(x[1], x[3]), a3 = rot4<SIGN>(csub(x[1], x[3]));
        x[0] = cadd(a0, a2);
        x[2] = csub(a0, a2);
        x[1] = cadd(a1, a3);
        x[3] = csub(a1, a3);
    } else if constexpr (R == 8) {
        // decimation in time: two 4-point DFTs of the even and odd samples
        float2 e[4] = {x[0], x[2], x[4], x[6]};
        float2 o[4] = {x[1], x[3], x[5], x[7]};
        dft_small<4, SIGN>(e);
        dft_small<4, SIGN>(o);
        constexpr float h = 0.70710678118654752440f;
        // W_8^k o_k for k = 1, 2, 3
        const float2 o1 = SIGN < 0 ? make_float2(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x))
                                   : make_float2(h * (o[1].x - o[1].y), h * (o[1].y + o[1].x));
        const float2 o2 = rot4<SIGN>(o[2]);
        const float2 o3 = SIGN < 0 ? make_float2(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y))
                                   : make_float2(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y));
        x[0] = cadd(e[0], o[0]);
        x[4] = csub(e[0], o[0]);
        x[1] = cadd(e[1], o1);
        x[5] = csub(e[1], o1);
        x[2] = cadd(e[2], o2);
        x[6] = csub(e[2], o2);
        x[3] = cadd(e[3], o3);
        x[7] = csub(e[3], o3);
    } else if constexpr (R == 16) {
        // 16 = 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2;
        // X[k1 + 4 k2] = sum_n2 W4^(n2 k2) W16^(n2 k1) sum_n1 x[4 n1 + n2] W4^(n1 k1)
        float2 a[4][4];  // a[n2][k1]
#pragma unroll
        for (int n2 = 0; n2 < 4; n2++) {
            float2 c[4] = {x[n2], x[4 + n2], x[8 + n2], x[12 + n2]};
            dft_small<4, SIGN>(c);
#pragma unroll
            for (int k1 = 0; k1 < 4; k1++) a[n2][k1] = c[k1];
        }
        // W16^k = exp(SIGN i pi k / 8) for the products n2 k1 in {1, 2, 3, 4, 6, 9}
        constexpr float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f;
        constexpr float h = 0.70710678118654752440f;
        constexpr float sg = SIGN < 0 ? -1.f : 1.f;
        const float2 w1 = make_float2(c1, sg * s1), w2 = make_float2(h, sg * h), w3 = make_float2(s1, sg * c1);
        const float2 w6 = make_float2(-h, sg * h), w9 = make_float2(-c1, -sg * s1);
        a[1][1] = cmul(a[1][1], w1);
        a[1][2] = cmul(a[1][2], w2);
        a[1][3] = cmul(a[1][3], w3);
        a[2][1] = cmul(a[2][1], w2);
        a[2][2] = rot4<SIGN>(a[2][2]);
        a[2][3] = cmul(a[2][3], w6);
        a[3][1] = cmul(a[3][1], w3);
        a[3][2] = cmul(a[3][2], w6);
        a[3][3] = cmul(a[3][3], w9);
#pragma unroll
        for (int k1 = 0; k1 < 4; k1++) {
            float2 c[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
            dft_small<4, SIGN>(c);
#pragma unroll
            for (int k2 = 0; k2 < 4; k2++) x[k1 + 4 * k2] = c[k2];
        }
    } else {
        static_assert(R == 1 || R == 2 || R == 4 || R == 8 || R == 16, "unsupported radix");
    }
}

// One Stockham pass (see file comment).  buf: shared, fft_buf_len(N) float2.
// TRAIL = false drops the barrier after the read-back (ping-pong buffers, below).
template <int N, int T, int R, int NS, int TWOFF, int SIGN, bool LAST, bool TRAIL = true>
__device__ __forceinline__ void fft_pass(float2 (&v)[N / T], float2 *buf, const float2 *tw, int tid)
{
    constexpr int E = N / T, BPT = E / R;
    static_assert(BPT * R == E, "radix must divide the points per thread");
#pragma unroll
    for (int i = 0; i < BPT; i++) {
        const int b = tid + i * T;
        const int j = b & (NS - 1);
        float2 x[R];
#pragma unroll
        for (int r = 0; r < R; r++) x[r] = v[i + r * BPT];
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; r++) {
                float2 w = tw[TWOFF + (r - 1) * NS + j];
                if constexpr (SIGN > 0) w.y = -w.y;
                x[r] = cmul(x[r], w);
            }
        }
        dft_small<R, SIGN>(x);
        if constexpr (LAST) {
#pragma unroll
            for (int q = 0; q < R; q++) v[i + q * BPT] = x[q];
        } else {
            const int base = (b - j) * R + j;
#pragma unroll
            for (int q = 0; q < R; q++) buf[fft_pad(base + q * NS)] = x[q];
        }
    }
    if constexpr (!LAST) {
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; e++) v[e] = buf[fft_pad(tid + e * T)];
        if constexpr (TRAIL) __syncthreads();
    }
}

template <int N, int T, int SIGN, int p>
__device__ __forceinline__ void fft_passes(float2 (&v)[N / T], float2 *buf, const float2 *tw, int tid)
{
    using Pl = FftPlan<N, N / T>;
    if constexpr (p < Pl::P) {
        fft_pass<N, T, Pl::radix(p), Pl::ns(p), Pl::tw_off(p), SIGN, p == Pl::P - 1>(v, buf, tw, tid);
        fft_passes<N, T, SIGN, p + 1>(v, buf, tw, tid);
    }
}

// Unnormalised length-N transform of the thread-strided registers v:
// SIGN = -1: X[k] = sum_n x[n] exp(-2 pi i k n / N); SIGN = +1: the conjugate
// kernel (N * ifft).  All T threads of the team must call it (it
// synchronises the block); buf and tw are shared memory.
template <int N, int T, int SIGN>
__device__ __forceinline__ void block_fft(float2 (&v)[N / T], float2 *buf, const float2 *tw, int tid)
{
    fft_passes<N, T, SIGN, 0>(v, buf, tw, tid);
}


// ---------------------------------------------------------------------------
// Variant whose last pass takes its twiddles from a per-thread base instead of
// the table: in the last pass (Ns = N/R, R = E) butterfly b = tid has
// j = tid, so its twiddles are w^r with w = exp(-2 pi i tid / N); the thread
// keeps w in two registers (wb, made once) and forms the powers by complex
// multiplication.  The table then only needs passes 1 .. P-2 (tw_off(P-1)
// entries), which is what lets the solver keep it in shared memory cheaply.
template <int N, int T>
struct FftSmall {
    using Pl = FftPlan<N, N / T>;
    static constexpr int TW_SMALL = Pl::P >= 2 ? Pl::tw_off(Pl::P - 1) : 0;
};

template <int R, int SIGN>
__device__ __forceinline__ void twiddle_powers(float2 (&x)[R], float2 wb)
{
    if constexpr (SIGN > 0) wb.y = -wb.y;
    if constexpr (R >= 2) x[1] = cmul(x[1], wb);
    if constexpr (R >= 4) {
        const float2 w2 = cmul(wb, wb), w3 = cmul(w2, wb);
        x[2] = cmul(x[2], w2);
        x[3] = cmul(x[3], w3);
        if constexpr (R >= 8) {
            const float2 w4 = cmul(w2, w2);
            x[4] = cmul(x[4], w4);
            x[5] = cmul(x[5], cmul(w4, wb));
            x[6] = cmul(x[6], cmul(w4, w2));
            x[7] = cmul(x[7], cmul(w4, w3));
            if constexpr (R >= 16) {
                const float2 w8 = cmul(w4, w4);
                x[8] = cmul(x[8], w8);
                x[9] = cmul(x[9], cmul(w8, wb));
                x[10] = cmul(x[10], cmul(w8, w2));
                x[11] = cmul(x[11], cmul(w8, w3));
                const float2 w12 = cmul(w8, w4);
                x[12] = cmul(x[12], w12);
                x[13] = cmul(x[13], cmul(w12, wb));
                x[14] = cmul(x[14], cmul(w12, w2));
                x[15] = cmul(x[15], cmul(w12, w3));
            }
        }
    }
}

template <int N, int T, int SIGN, int p>
__device__ __forceinline__ void fft_passes_rb(float2 (&v)[N / T], float2 *buf, const float2 *tw, float2 wb,
                                              int tid)
{
    using Pl = FftPlan<N, N / T>;
    if constexpr (p < Pl::P - 1) {
        fft_pass<N, T, Pl::radix(p), Pl::ns(p), Pl::tw_off(p), SIGN, false>(v, buf, tw, tid);
        fft_passes_rb<N, T, SIGN, p + 1>(v, buf, tw, wb, tid);
    } else if constexpr (p == Pl::P - 1) {
        constexpr int R = Pl::radix(p), E = N / T;
        static_assert(R == E, "last pass must use the full radix");
        float2 x[R];
#pragma unroll
        for (int r = 0; r < R; r++) x[r] = v[r];
        if constexpr (Pl::ns(p) > 1) twiddle_powers<R, SIGN>(x, wb);
        dft_small<R, SIGN>(x);
#pragma unroll
        for (int q = 0; q < R; q++) v[q] = x[q];
    }
}

// As block_fft; wb = exp(-2 pi i tid / N) for this thread.
template <int N, int T, int SIGN>
__device__ __forceinline__ void block_fft_rb(float2 (&v)[N / T], float2 *buf, const float2 *tw, float2 wb,
                                             int tid)
{
    fft_passes_rb<N, T, SIGN, 0>(v, buf, tw, wb, tid);
}


// ---------------------------------------------------------------------------
// Several butterflies per thread and pass: E points per thread, radix-R passes
// (BPT = E / R butterflies each).  The last pass takes its twiddles from
// per-thread bases as above, one per butterfly: butterfly i of thread tid is
// b = tid + i T, and wb[i] = exp(-2 pi i b / N).
template <int N, int T, int R, int SIGN, int p>
__device__ __forceinline__ void fft_passes_rbx(float2 (&v)[N / T], float2 *buf, const float2 *tw,
                                               const float2 (&wb)[N / T / R], int tid)
{
    using Pl = FftPlan<N, N / T, R>;
    if constexpr (p < Pl::P - 1) {
        fft_pass<N, T, Pl::radix(p), Pl::ns(p), Pl::tw_off(p), SIGN, false>(v, buf, tw, tid);
        fft_passes_rbx<N, T, R, SIGN, p + 1>(v, buf, tw, wb, tid);
    } else if constexpr (p == Pl::P - 1) {
        constexpr int BPT = N / T / R;
        static_assert(Pl::radix(p) == R, "last pass must use the full radix");
#pragma unroll
        for (int i = 0; i < BPT; i++) {
            float2 x[R];
#pragma unroll
            for (int r = 0; r < R; r++) x[r] = v[i + r * BPT];
            if constexpr (Pl::ns(p) > 1) twiddle_powers<R, SIGN>(x, wb[i]);
            dft_small<R, SIGN>(x);
#pragma unroll
            for (int q = 0; q < R; q++) v[i + q * BPT] = x[q];
        }
    }
}

template <int N, int T, int R, int SIGN>
__device__ __forceinline__ void block_fft_rbx(float2 (&v)[N / T], float2 *buf, const float2 *tw,
                                              const float2 (&wb)[N / T / R], int tid)
{
    fft_passes_rbx<N, T, R, SIGN, 0>(v, buf, tw, wb, tid);
}


// ---------------------------------------------------------------------------
// Ping-pong exchange: exchange k of a transform (k = 0 .. P-2) goes through
// buffer (ph + k) & 1 of a pair, and the barrier after each read-back is
// dropped: the next exchange writes the other buffer, and its own barrier
// orders every read of this one before any later write to it.  ph carries the
// alternation from one transform to the next (it flips when a transform has
// an odd number of exchanges), so a transform's first write never lands in the
// buffer that the previous transform read last.  Every thread of the block
// must run the same sequence of transforms.  Last pass and twiddle bases as
// in fft_passes_rbx.
template <int N, int T, int R, int SIGN, int p>
__device__ __forceinline__ void fft_passes_pp(float2 (&v)[N / T], float2 *b0, float2 *b1, const float2 *tw,
                                              const float2 (&wb)[N / T / R], int tid)
{
    using Pl = FftPlan<N, N / T, R>;
    if constexpr (p < Pl::P - 1) {
        fft_pass<N, T, Pl::radix(p), Pl::ns(p), Pl::tw_off(p), SIGN, false, false>(v, (p & 1) ? b1 : b0, tw,
                                                                                 tid);
        fft_passes_pp<N, T, R, SIGN, p + 1>(v, b0, b1, tw, wb, tid);
    } else if constexpr (p == Pl::P - 1) {
        fft_passes_rbx<N, T, R, SIGN, p>(v, b0, tw, wb, tid);
    }
}

// buf: two fft_buf_len(N) buffers back to back; ph: the pair's parity (0 or 1)
template <int N, int T, int R, int SIGN>
__device__ __forceinline__ void block_fft_pp(float2 (&v)[N / T], float2 *buf, const float2 *tw,
                                             const float2 (&wb)[N / T / R], int tid, int &ph)
{
    using Pl = FftPlan<N, N / T, R>;
    float2 *b0 = buf + (ph ? fft_buf_len(N) : 0), *b1 = buf + (ph ? 0 : fft_buf_len(N));
    fft_passes_pp<N, T, R, SIGN, 0>(v, b0, b1, tw, wb, tid);
    ph ^= (Pl::P - 1) & 1;
}

}  // namespace tmr
