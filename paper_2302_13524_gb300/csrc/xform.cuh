// xform.cuh -- the masked probing transforms of one team of threads.
//
// A team of NT threads holds a length-N vector in the thread-strided layout
// (register e of thread tid <-> index tid + e NT, NE registers, indices >= N
// unused and kept at zero) and applies
//   fwd:  x <- F(d .* x)           (one block of Q, Eq. probingmatrix)
//   adj:  x <- conj(d) .* F^H x    (its adjoint, Eq. derivative)
// with the unnormalised length-N DFT F.
//
// XfPow2<N>: N a power of two; one register Stockham FFT of length N.
//
// XfBlue<L, NE>: any other N with 2N - 1 <= L (L a power of two), by
// Bluestein's chirp-z identity kn = (k^2 + n^2 - (k - n)^2) / 2:
//   (F x)_k = c_k sum_n (x_n c_n) conj(c_{k-n}),   c_n = exp(-i pi n^2 / N),
// a linear convolution of a_n = x_n c_n (n < N) with b_m = conj(c_m)
// (|m| < N), evaluated as a cyclic one of length L >= 2N - 1:
//   F x = c .* F_L^{+}( F_L^{-}(a) .* B ),   B = F_L(b) / L.
// b is even (b_{-m} = b_m), so B is even too and half of it (B_k, k <= L/2)
// is stored.  The adjoint uses F^H x = conj(F conj(x)).  With the mask folded
// into the chirp (dc = d .* c):
//   fwd: a = x .* dc,         x <- c .* conv(a)
//   adj: a = conj(x) .* c,    x <- conj(dc .* conv(a))
// Four length-L FFTs per forward/adjoint pair instead of two length-N ones.
//
// Constants (host-made in FP64, rounded to FP32), one table per N:
//   [ FFT twiddles (NCONST_TW) | B half (L/2 + 1) | chirp c (N) ]
// Every CTA copies the first shared_consts(N) entries (all of it for
// Bluestein, the twiddles of the non-final passes for powers of two) to shared
// memory; dc is made once per thread in registers.
#pragma once

#include "common.cuh"
#include "fft.cuh"

namespace tmr {

template <int N_>
struct XfPow2 {
    static constexpr bool kBlue = false;
    static constexpr int kN = N_;              // length fixed at compile time
    static constexpr int NT = fft_threads(N_);  // threads per team
    static constexpr int NE = N_ / NT;          // registers per length-N vector
    static constexpr int LBUF = fft_buf_len(N_);  // exchange buffer per team (float2)
    static constexpr int NCONST = FftSmall<N_, NT>::TW_SMALL;  // constants before the chirp (float2)
    __host__ __device__ static constexpr int shared_consts(int n) { return NCONST; }

    float2 dm[NE];
    float2 wb;

    __device__ __forceinline__ static bool valid(int e, int tid, int n) { return true; }

    __device__ __forceinline__ void setup(const float2 *__restrict__ mask, const float2 *__restrict__ chirp,
                                          int n, int tid)
    {
#pragma unroll
        for (int e = 0; e < NE; e++) dm[e] = mask[tid + e * NT];
        double s, c;
        sincospi(-2.0 * (double)tid / (double)N_, &s, &c);
        wb = make_float2((float)c, (float)s);
    }
    __device__ __forceinline__ void fwd(float2 (&x)[NE], float2 *buf, const float2 *cst, int tid) const
    {
#pragma unroll
        for (int e = 0; e < NE; e++) x[e] = cmul(x[e], dm[e]);
        block_fft_rb<N_, NT, -1>(x, buf, cst, wb, tid);
    }
    __device__ __forceinline__ void adj(float2 (&x)[NE], float2 *buf, const float2 *cst, int tid) const
    {
        block_fft_rb<N_, NT, +1>(x, buf, cst, wb, tid);
#pragma unroll
        for (int e = 0; e < NE; e++) x[e] = cmulc(x[e], dm[e]);
    }
};

template <int L_, int NE_>
struct XfBlue {
    static constexpr bool kBlue = true;
    static constexpr int kN = 0;  // length given at run time
    static constexpr int L = L_, EL = 16, R = 8, BPT = EL / R;
    static constexpr int NT = L_ / EL;
    static constexpr int NE = NE_;
    static_assert(NE <= EL / 2, "N <= L / 2");
    using Plan = FftPlan<L_, EL, R>;
    static constexpr int LBUF = fft_buf_len(L_);
    static constexpr int NCONST_TW = Plan::TW_SMALL;
    static constexpr int NCONST = NCONST_TW + L_ / 2 + 1;
    __host__ __device__ static constexpr int shared_consts(int n) { return NCONST + n; }

    float2 dc[NE];
    float2 wb[BPT];
    int n;

    __device__ __forceinline__ static bool valid(int e, int tid, int n) { return tid + e * NT < n; }

    __device__ __forceinline__ void setup(const float2 *__restrict__ mask, const float2 *__restrict__ chirp,
                                          int n_, int tid)
    {
        n = n_;
#pragma unroll
        for (int e = 0; e < NE; e++) {
            const int i = tid + e * NT;
            dc[e] = i < n ? cmul(mask[i], chirp[i]) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < BPT; i++) {
            double s, co;
            sincospi(-2.0 * (double)(tid + i * NT) / (double)L_, &s, &co);
            wb[i] = make_float2((float)co, (float)s);
        }
    }
    // v <- F_L^{+}(F_L^{-}(v) .* B)
    __device__ __forceinline__ void conv(float2 (&v)[EL], float2 *buf, const float2 *cst, int tid) const
    {
        block_fft_rbx<L_, NT, R, -1>(v, buf, cst, wb, tid);
        const float2 *B = cst + NCONST_TW;
#pragma unroll
        for (int e = 0; e < EL; e++) {
            const int k = tid + e * NT;
            v[e] = cmul(v[e], B[e < EL / 2 ? k : L_ - k]);
        }
        block_fft_rbx<L_, NT, R, +1>(v, buf, cst, wb, tid);
    }
    __device__ __forceinline__ void fwd(float2 (&x)[NE], float2 *buf, const float2 *cst, int tid) const
    {
        float2 v[EL];
#pragma unroll
        for (int e = 0; e < EL; e++)
            v[e] = (e < NE && valid(e, tid, n)) ? cmul(x[e < NE ? e : 0], dc[e < NE ? e : 0]) : make_float2(0.f, 0.f);
        conv(v, buf, cst, tid);
        const float2 *c = cst + NCONST;
#pragma unroll
        for (int e = 0; e < NE; e++) x[e] = valid(e, tid, n) ? cmul(v[e], c[tid + e * NT]) : make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ void adj(float2 (&x)[NE], float2 *buf, const float2 *cst, int tid) const
    {
        float2 v[EL];
        const float2 *c = cst + NCONST;
#pragma unroll
        for (int e = 0; e < EL; e++)
            v[e] = (e < NE && valid(e, tid, n)) ? cmul(cconj(x[e < NE ? e : 0]), c[tid + e * NT])
                                                : make_float2(0.f, 0.f);
        conv(v, buf, cst, tid);
#pragma unroll
        for (int e = 0; e < NE; e++) x[e] = valid(e, tid, n) ? cconj(cmul(v[e], dc[e])) : make_float2(0.f, 0.f);
    }
};

}  // namespace tmr
