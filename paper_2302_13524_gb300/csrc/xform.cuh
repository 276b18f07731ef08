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

#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"
#include "fft.cuh"

namespace tmr {

template <int N_>
struct XfPow2 {
    static constexpr bool kBlue = false;
    static constexpr int kN = N_;              // length fixed at compile time
    static constexpr int NT = fft_threads(N_);  // threads per team
    static constexpr int NE = N_ / NT;          // registers per length-N vector
    static constexpr int LBUF = fft_buf_len(N_);  // one exchange buffer (float2)
    // exchange buffers per team: two (ping-pong, one barrier per exchange)
    // where shared memory allows, else one (two barriers per exchange)
    static constexpr int BUFS = N_ <= 2048 ? 2 : 1;
    static constexpr int NCONST = FftSmall<N_, NT>::TW_SMALL;  // constants before the chirp (float2)
    __host__ __device__ static constexpr int shared_consts(int n) { return NCONST; }

    float2 dm[NE];
    float2 wb[1];
    int ph;  // ping-pong parity

    __device__ __forceinline__ static bool valid(int e, int tid, int n) { return true; }

    __device__ __forceinline__ void setup(const float2 *__restrict__ mask, const float2 *__restrict__ chirp,
                                          int n, int tid)
    {
#pragma unroll
        for (int e = 0; e < NE; e++) dm[e] = mask[tid + e * NT];
        double s, c;
        sincospi(-2.0 * (double)tid / (double)N_, &s, &c);
        wb[0] = make_float2((float)c, (float)s);
        ph = 0;
    }
    template <int SIGN>
    __device__ __forceinline__ void fft(float2 (&x)[NE], float2 *buf, const float2 *cst, int tid)
    {
        if constexpr (BUFS == 2) block_fft_pp<N_, NT, NE, SIGN>(x, buf, cst, wb, tid, ph);
        else block_fft_rb<N_, NT, SIGN>(x, buf, cst, wb[0], tid);
    }
    // buf: BUFS * LBUF float2 of this team
    __device__ __forceinline__ void fwd(float2 (&x)[NE], float2 *buf, const float2 *cst, int tid)
    {
#pragma unroll
        for (int e = 0; e < NE; e++) x[e] = cmul(x[e], dm[e]);
        fft<-1>(x, buf, cst, tid);
    }
    __device__ __forceinline__ void adj(float2 (&x)[NE], float2 *buf, const float2 *cst, int tid)
    {
        fft<+1>(x, buf, cst, tid);
#pragma unroll
        for (int e = 0; e < NE; e++) x[e] = cmulc(x[e], dm[e]);
    }
};

// XfDenseMV<N>: the probing DFT as an explicit matrix-vector product, the
// paper's "TM retrieval without FFT" (Sec. 3, Table 1: Algorithm 1 with the
// FFTs replaced by matrix-vector multiplication).  The team writes its masked
// vector to shared memory in natural order and every thread forms its
// outputs z[k] = sum_n W_N^{kn} x[n] from the table W_N^m, m < N (made in
// FP64 on the host): N complex multiply-adds per output, N^2 per transform.
template <int N_>
struct XfDenseMV {
    static constexpr bool kBlue = false;
    static constexpr int kN = N_;
    static constexpr int NT = fft_threads(N_);
    static constexpr int NE = N_ / NT;
    static constexpr int LBUF = N_;
    static constexpr int BUFS = 1;
    static constexpr int NCONST = N_;
    __host__ __device__ static constexpr int shared_consts(int n) { return NCONST; }

    float2 dm[NE];

    __device__ __forceinline__ static bool valid(int e, int tid, int n) { return true; }

    __device__ __forceinline__ void setup(const float2 *__restrict__ mask, const float2 *__restrict__ chirp,
                                          int n, int tid)
    {
#pragma unroll
        for (int e = 0; e < NE; e++) dm[e] = mask[tid + e * NT];
    }
    template <int SIGN>
    __device__ __forceinline__ void mv(float2 (&x)[NE], float2 *buf, const float2 *cst, int tid)
    {
#pragma unroll
        for (int e = 0; e < NE; e++) buf[tid + e * NT] = x[e];
        __syncthreads();
        float2 acc[NE];
#pragma unroll
        for (int e = 0; e < NE; e++) acc[e] = make_float2(0.f, 0.f);
        for (int n = 0; n < N_; n++) {
            const float2 v = buf[n];
#pragma unroll
            for (int e = 0; e < NE; e++) {
                float2 w = cst[((tid + e * NT) * n) & (N_ - 1)];
                if (SIGN > 0) w.y = -w.y;
                acc[e].x = fmaf(w.x, v.x, fmaf(-w.y, v.y, acc[e].x));
                acc[e].y = fmaf(w.x, v.y, fmaf(w.y, v.x, acc[e].y));
            }
        }
        __syncthreads();  // buf is read before the caller reuses it
#pragma unroll
        for (int e = 0; e < NE; e++) x[e] = acc[e];
    }
    __device__ __forceinline__ void fwd(float2 (&x)[NE], float2 *buf, const float2 *cst, int tid)
    {
#pragma unroll
        for (int e = 0; e < NE; e++) x[e] = cmul(x[e], dm[e]);
        mv<-1>(x, buf, cst, tid);
    }
    __device__ __forceinline__ void adj(float2 (&x)[NE], float2 *buf, const float2 *cst, int tid)
    {
        mv<+1>(x, buf, cst, tid);
#pragma unroll
        for (int e = 0; e < NE; e++) x[e] = cmulc(x[e], dm[e]);
    }
};

// XfPow2D<N>: the paper's 2D probing DFT (Eq. probingmatrix: K the 2D Fourier
// transform of the row read as an n1 x n2 array, n1 n2 = N) through the same
// register Stockham passes.  The Stockham passes whose stride Ns reaches n1
// combine the length-n1 DFTs along the first index; with the twiddle of such
// a pass taken as W_{(Ns/n1) R}^{r (j div n1)} instead of W_{Ns R}^{r j}
// (the factors that couple the two indices dropped) the passes compute the 2D
// DFT, spectrum X[k1][k2] at index k1 + n1 k2.  The adjoint reads its input in
// that order, i.e. as an n2 x n1 array, so it runs the same passes with n2 in
// place of n1.  n1 and n2 must both be strides at which a pass starts (the
// products of the leading radices: 8 and 64 for N = 512; 8, 64, 512 for
// N = 4096).  Constants: [ forward table (n1) | adjoint table (n2) | (n1, n2) ].
template <int N_>
struct XfPow2D {
    static constexpr bool kBlue = false;
    static constexpr int kN = N_;
    static constexpr int NT = fft_threads(N_);
    static constexpr int NE = N_ / NT;
    static constexpr int LBUF = fft_buf_len(N_);
    static constexpr int BUFS = N_ <= 2048 ? 2 : 1;
    static constexpr int TWS = FftSmall<N_, NT>::TW_SMALL;  // one table
    static constexpr int NCONST = 2 * TWS;
    __host__ __device__ static constexpr int shared_consts(int n) { return NCONST; }

    float2 dm[NE];
    float2 wbf[1], wba[1];  // last-pass bases of the forward and the adjoint passes
    int ph;

    __device__ __forceinline__ static bool valid(int e, int tid, int n) { return true; }

    // chirp: the (n1, n2) entry after the two tables
    __device__ __forceinline__ void setup(const float2 *__restrict__ mask, const float2 *__restrict__ chirp,
                                          int n, int tid)
    {
#pragma unroll
        for (int e = 0; e < NE; e++) dm[e] = mask[tid + e * NT];
        const int n1 = (int)chirp[0].x, n2 = (int)chirp[0].y;
        // the last pass has stride N / NE >= n1, n2: twiddle base W_{N/B}^{tid div B}
        double s, c;
        sincospi(-2.0 * (double)(tid / n1) / (double)(N_ / n1), &s, &c);
        wbf[0] = make_float2((float)c, (float)s);
        sincospi(-2.0 * (double)(tid / n2) / (double)(N_ / n2), &s, &c);
        wba[0] = make_float2((float)c, (float)s);
        ph = 0;
    }
    __device__ __forceinline__ void fwd(float2 (&x)[NE], float2 *buf, const float2 *cst, int tid)
    {
#pragma unroll
        for (int e = 0; e < NE; e++) x[e] = cmul(x[e], dm[e]);
        if constexpr (BUFS == 2) block_fft_pp<N_, NT, NE, -1>(x, buf, cst, wbf, tid, ph);
        else block_fft_rb<N_, NT, -1>(x, buf, cst, wbf[0], tid);
    }
    __device__ __forceinline__ void adj(float2 (&x)[NE], float2 *buf, const float2 *cst, int tid)
    {
        if constexpr (BUFS == 2) block_fft_pp<N_, NT, NE, +1>(x, buf, cst + TWS, wba, tid, ph);
        else block_fft_rb<N_, NT, +1>(x, buf, cst + TWS, wba[0], tid);
#pragma unroll
        for (int e = 0; e < NE; e++) x[e] = cmulc(x[e], dm[e]);
    }
};

// The strides at which a pass of the XfPow2 plan of length N starts
// (products of the leading radices), excluding 1 and N.
__host__ __device__ inline bool probe_2d_boundary(int N, int b)
{
    if (N != 512 && N != 4096) return false;  // plans with radix 8 in every pass
    for (int s = 8; s < N; s *= 8)
        if (s == b) return true;
    return false;
}

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
    static constexpr int BUFS = 1;
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
    __device__ __forceinline__ void fwd(float2 (&x)[NE], float2 *buf, const float2 *cst, int tid)
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
    __device__ __forceinline__ void adj(float2 (&x)[NE], float2 *buf, const float2 *cst, int tid)
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

// XfBlueSplit<NE>: N in (2048, 2731] by Bluestein at L = 4096 < 2N - 1, with
// the outputs split in two halves [0, H) and [H, N), H = ceil(N / 2).  Output
// k needs b_{k-n} for n < N only; for the first half the indices run over
// [-(N-1), H-1], for the second over [H-(N-1), N-1], each of length at most
// N + H - 1 <= L, so each half is an exact cyclic convolution with its own
// filter b~_h (b_m placed at m mod L on the half's range, zero elsewhere):
//   F x = c .* F_L^{+}( A .* B_h ) on half h,   A = F_L^{-}(x .* d .* c),
//   B_h = F_L(b~_h) / L.
// One forward and two inverse length-4096 FFTs per transform (three, against
// two of length 8192 above), 8 points per thread; the filters are not even,
// so both are stored whole.
// Constants: [ FFT twiddles | B_1 (L) | B_2 (L) | chirp c (N) ].
constexpr int kBlueSplitMaxN = 2731;  // N + ceil(N / 2) - 1 <= 4096

template <int NE_>
struct XfBlueSplit {
    static constexpr bool kBlue = true;
    static constexpr int kN = 0;
    static constexpr int L = 4096;
    static constexpr int NT = L / 8, EL = 8;
    static constexpr int NE = NE_;
    static_assert(NE * NT <= 2 * L, "registers");
    static constexpr int LBUF = fft_buf_len(L);
    static constexpr int BUFS = 1;
    static constexpr int NCONST_TW = FftSmall<L, NT>::TW_SMALL;
    static constexpr int NCONST = NCONST_TW + 2 * L;
    __host__ __device__ static constexpr int shared_consts(int n) { return NCONST + n; }

    float2 dc[NE];
    float2 wb;
    int n, h;

    __device__ __forceinline__ static bool valid(int e, int tid, int n) { return tid + e * NT < n; }

    __device__ __forceinline__ void setup(const float2 *__restrict__ mask, const float2 *__restrict__ chirp,
                                          int n_, int tid)
    {
        n = n_;
        h = (n_ + 1) / 2;
#pragma unroll
        for (int e = 0; e < NE; e++) {
            const int i = tid + e * NT;
            dc[e] = i < n ? cmul(mask[i], chirp[i]) : make_float2(0.f, 0.f);
        }
        double s, co;
        sincospi(-2.0 * (double)tid / (double)L, &s, &co);
        wb = make_float2((float)co, (float)s);
    }
    // out[e] (index k = tid + e NT < n) <- (c .* conv_h(a))_k, a given in v
    __device__ __forceinline__ void conv2(float2 (&v)[EL], float2 (&out)[NE], float2 *buf, const float2 *cst,
                                          int tid, bool conj_out) const
    {
        block_fft_rb<L, NT, -1>(v, buf, cst, wb, tid);
        const float2 *c = cst + NCONST;
#pragma unroll
        for (int half = 0; half < 2; half++) {
            const float2 *B = cst + NCONST_TW + half * L;
            float2 w[EL];
#pragma unroll
            for (int e = 0; e < EL; e++) w[e] = cmul(v[e], B[tid + e * NT]);
            block_fft_rb<L, NT, +1>(w, buf, cst, wb, tid);
#pragma unroll
            for (int e = 0; e < NE; e++) {
                const int k = tid + e * NT;
                const bool mine = half == 0 ? k < h : (k >= h && k < n);
                if (mine) out[e] = conj_out ? w[e] : cmul(w[e], c[k]);
            }
        }
    }
    __device__ __forceinline__ void fwd(float2 (&x)[NE], float2 *buf, const float2 *cst, int tid)
    {
        float2 v[EL];
#pragma unroll
        for (int e = 0; e < EL; e++)
            v[e] = (e < NE && valid(e, tid, n)) ? cmul(x[e < NE ? e : 0], dc[e < NE ? e : 0]) : make_float2(0.f, 0.f);
#pragma unroll
        for (int e = 0; e < NE; e++) x[e] = make_float2(0.f, 0.f);
        conv2(v, x, buf, cst, tid, false);
    }
    __device__ __forceinline__ void adj(float2 (&x)[NE], float2 *buf, const float2 *cst, int tid)
    {
        const float2 *c = cst + NCONST;
        float2 v[EL];
#pragma unroll
        for (int e = 0; e < EL; e++)
            v[e] = (e < NE && valid(e, tid, n)) ? cmul(cconj(x[e < NE ? e : 0]), c[tid + e * NT])
                                                : make_float2(0.f, 0.f);
#pragma unroll
        for (int e = 0; e < NE; e++) x[e] = make_float2(0.f, 0.f);
        conv2(v, x, buf, cst, tid, true);  // x <- conv(a) on [0, n), unmultiplied
#pragma unroll
        for (int e = 0; e < NE; e++) x[e] = valid(e, tid, n) ? cconj(cmul(x[e], dc[e])) : make_float2(0.f, 0.f);
    }
};

// ---------------------------------------------------------------------------
// XfMixed<N>: N a power of two, 64 <= N <= 4096, written N = 16^A 8^B with A
// as large as possible.  The FP32 transforms of XfPow2<N>, plus a tensor-core
// form of the same DFT (tc = true): A radix-16 then B radix-8 Stockham passes
// (the butterfly, twiddle and output placement of fft_pass), each R-point DFT
// of a pass evaluated as a real GEMM on the tensor cores,
//   [Re y; Im y] = [[C, sS]; [-sS, C]] [Re x; Im x],  C = cos(2 pi q r / R),
//   S = sin(2 pi q r / R), s = +1 forward, -1 inverse,
// with mma.sync m16n8k16 (BF16 operands, FP32 accumulation) on 8 butterflies
// per instruction group: for R = 16 the 32 x 32 block takes 2 x 2 tiles
// (12 instructions with the split below), for R = 8 the 16 x 16 block is one
// tile (3 instructions).  Operands are split hi + lo (hi = bf16(v),
// lo = bf16(v - hi)) and each product is A_hi B_lo + A_lo B_hi + A_hi B_hi
// (the lo*lo term dropped): about 16 significant bits per product.
// Twiddles are FP32 roots W_N^k from a table in shared memory.
// Constants: [FP32 small twiddles | radix-16 fragments (C, S, -S; hi, lo) |
// radix-8 fragments (forward and inverse blocks; hi, lo) | roots W_N^k].
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint4 &a, uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t *>(&v); }

// (lo, hi) pair of values -> hi and lo split words
__device__ __forceinline__ void split_bf16x2(float a, float b, uint32_t &hi, uint32_t &lo)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - __low2float(h), b - __high2float(h));
    hi = bf16x2_bits(h);
    lo = bf16x2_bits(l);
}

// fragment tiles: radix 16: C, S, -S (hi at even, lo at odd index); radix 8:
// forward block then inverse block (hi, lo)
enum { kTcC = 0, kTcS = 2, kTcNS = 4, kTcTiles16 = 6, kTc8Fwd = 0, kTc8Inv = 2, kTcTiles8 = 4 };

// radix-16 passes of N = 2^lg written 16^A 8^B with A largest
__host__ __device__ constexpr int mixed_a16(int lg) { return lg % 3 == 0 ? (lg >= 12 ? 3 : 0) : (lg % 3 == 1 ? 1 : 2); }

// Element i of a tensor-core transform's buffer lives at tc_addr(i): bits 2-3
// of i are XORed with a hash of bits 4, 6, 8 and 10, a bijection inside each
// 16-element block.  The passes read a butterfly's inputs at strides of N/16
// (N/8) and write outputs at strides of 16 or 256; with a plain (or per-16
// padded) layout those land on the same banks, and the swizzle spreads them
// (for N = 2048 the 64-bit accesses of a transform take 1.29 times the
// minimum number of shared-memory wavefronts instead of 3.0).
__device__ __forceinline__ int tc_addr(int i)
{
    return i ^ ((((i >> 4) ^ (i >> 6) ^ (i >> 8) ^ (i >> 10)) & 3) << 2);
}

template <int N_>
struct XfMixed {
    static constexpr bool kBlue = false;
    static constexpr bool kMixed = true;
    static constexpr int kN = N_;
    using F32 = XfPow2<N_>;
    static constexpr int NT = F32::NT, NE = F32::NE;
    static constexpr int LBUF = F32::LBUF;
    static constexpr int BUFS = F32::BUFS;
    static constexpr int LG = ilog2c(N_);
    static constexpr int A16 = mixed_a16(LG);     // radix-16 passes
    static constexpr int B8 = (LG - 4 * A16) / 3;  // radix-8 passes
    static_assert(4 * A16 + 3 * B8 == LG && A16 >= 0 && B8 >= 0, "N = 16^A 8^B");
    static constexpr int P = A16 + B8;
    static constexpr int NWT = NT / 32;  // warps per team
    static constexpr int OFF_FRAG16 = F32::NCONST;
    static constexpr int OFF_FRAG8 = OFF_FRAG16 + kTcTiles16 * 32 * 4 / 2;  // in float2 units
    static constexpr int OFF_ROOT = OFF_FRAG8 + kTcTiles8 * 32 * 4 / 2;
    static constexpr int NCONST = OFF_ROOT + N_;
    __host__ __device__ static constexpr int shared_consts(int n) { return NCONST; }
    __host__ __device__ static constexpr int radix(int p) { return p < A16 ? 16 : 8; }
    __host__ __device__ static constexpr int ns(int p) { return p <= 0 ? 1 : ns(p - 1) * radix(p - 1); }

    F32 f32;
    bool tc;

    __device__ __forceinline__ static bool valid(int e, int tid, int n) { return true; }

    __device__ __forceinline__ void setup(const float2 *__restrict__ mask, const float2 *__restrict__ chirp,
                                          int n, int tid)
    {
        f32.setup(mask, chirp, n, tid);
        tc = true;
    }

    // one radix-16 pass: 8-butterfly groups, lane (g, t) loads inputs
    // r = 2t, 2t+1, 2t+8, 2t+9 of butterfly g and ends with outputs
    // q = g, g+8 of butterflies 2t, 2t+1
    template <int SIGN, int p>
    __device__ __forceinline__ void tc_pass16(const float2 *src, float2 *dst, const float2 *cst, int tid) const
    {
        constexpr int Ns = ns(p), NB = N_ / 16, GPW = NB / 8 / NWT;
        static_assert(GPW * 8 * NWT == NB && GPW >= 1, "group split");
        const int lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
        const uint4 *frag = reinterpret_cast<const uint4 *>(cst + OFF_FRAG16);
        const float2 *root = cst + OFF_ROOT;
        const uint4 Ch = frag[(kTcC + 0) * 32 + lane], Cl = frag[(kTcC + 1) * 32 + lane];
        // forward: Re y = C Re x + S Im x, Im y = C Im x - S Re x; inverse: S -> -S
        const uint4 Ph = frag[((SIGN < 0 ? kTcS : kTcNS) + 0) * 32 + lane];
        const uint4 Pl = frag[((SIGN < 0 ? kTcS : kTcNS) + 1) * 32 + lane];
        const uint4 Qh = frag[((SIGN < 0 ? kTcNS : kTcS) + 0) * 32 + lane];
        const uint4 Ql = frag[((SIGN < 0 ? kTcNS : kTcS) + 1) * 32 + lane];
        float2 out[GPW][4];
#pragma unroll
        for (int gi = 0; gi < GPW; gi++) {
            const int grp = warp * GPW + gi;
            const int b = grp * 8 + g;
            const int j = b & (Ns - 1);
            float2 xin[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int r = 2 * t + (u & 1) + 8 * (u >> 1);
                float2 v = src[tc_addr(b + r * NB)];
                if constexpr (Ns > 1) {
                    float2 w = root[(r * j) * (N_ / (16 * Ns))];
                    if constexpr (SIGN > 0) w.y = -w.y;
                    v = cmul(v, w);
                }
                xin[u] = v;
            }
            uint32_t reh0, rel0, reh1, rel1, imh0, iml0, imh1, iml1;
            split_bf16x2(xin[0].x, xin[1].x, reh0, rel0);
            split_bf16x2(xin[2].x, xin[3].x, reh1, rel1);
            split_bf16x2(xin[0].y, xin[1].y, imh0, iml0);
            split_bf16x2(xin[2].y, xin[3].y, imh1, iml1);
            float cre[4] = {0.f, 0.f, 0.f, 0.f}, cim[4] = {0.f, 0.f, 0.f, 0.f};
            // small terms first, then the hi x hi products
            mma_bf16_16816(cre, Ch, rel0, rel1);
            mma_bf16_16816(cre, Cl, reh0, reh1);
            mma_bf16_16816(cre, Ph, iml0, iml1);
            mma_bf16_16816(cre, Pl, imh0, imh1);
            mma_bf16_16816(cim, Ch, iml0, iml1);
            mma_bf16_16816(cim, Cl, imh0, imh1);
            mma_bf16_16816(cim, Qh, rel0, rel1);
            mma_bf16_16816(cim, Ql, reh0, reh1);
            mma_bf16_16816(cre, Ch, reh0, reh1);
            mma_bf16_16816(cre, Ph, imh0, imh1);
            mma_bf16_16816(cim, Ch, imh0, imh1);
            mma_bf16_16816(cim, Qh, reh0, reh1);
#pragma unroll
            for (int u = 0; u < 4; u++) out[gi][u] = make_float2(cre[u], cim[u]);
        }
        if (src == dst) __syncthreads();  // in place: every input is read before any write
#pragma unroll
        for (int gi = 0; gi < GPW; gi++) {
            const int grp = warp * GPW + gi;
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int bb = grp * 8 + 2 * t + (u & 1);
                const int q = g + 8 * (u >> 1);
                const int jj = bb & (Ns - 1);
                dst[tc_addr((bb - jj) * 16 + jj + q * Ns)] = out[gi][u];
            }
        }
        __syncthreads();
    }
    // one radix-8 pass: lane (g, t) loads inputs r = 2t, 2t+1 of butterfly g
    // and ends with output q = g of butterflies 2t, 2t+1
    template <int SIGN, int p>
    __device__ __forceinline__ void tc_pass8(const float2 *src, float2 *dst, const float2 *cst, int tid) const
    {
        constexpr int Ns = ns(p), NB = N_ / 8, GPW = NB / 8 / NWT;
        static_assert(GPW * 8 * NWT == NB && GPW >= 1, "group split");
        const int lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
        const uint4 *frag = reinterpret_cast<const uint4 *>(cst + OFF_FRAG8);
        const float2 *root = cst + OFF_ROOT;
        constexpr int base = SIGN < 0 ? kTc8Fwd : kTc8Inv;
        const uint4 Ah = frag[(base + 0) * 32 + lane], Al = frag[(base + 1) * 32 + lane];
        float2 out[GPW][2];
#pragma unroll
        for (int gi = 0; gi < GPW; gi++) {
            const int grp = warp * GPW + gi;
            const int b = grp * 8 + g;
            const int j = b & (Ns - 1);
            float2 xin[2];
#pragma unroll
            for (int u = 0; u < 2; u++) {
                const int r = 2 * t + u;
                float2 v = src[tc_addr(b + r * NB)];
                if constexpr (Ns > 1) {
                    float2 w = root[(r * j) * (N_ / (8 * Ns))];
                    if constexpr (SIGN > 0) w.y = -w.y;
                    v = cmul(v, w);
                }
                xin[u] = v;
            }
            uint32_t reh, rel, imh, iml;
            split_bf16x2(xin[0].x, xin[1].x, reh, rel);  // rows 2t, 2t+1: Re of inputs 2t, 2t+1
            split_bf16x2(xin[0].y, xin[1].y, imh, iml);  // rows 2t+8, 2t+9: their Im
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            mma_bf16_16816(d, Ah, rel, iml);
            mma_bf16_16816(d, Al, reh, imh);
            mma_bf16_16816(d, Ah, reh, imh);
            // rows g (Re y_g) and g + 8 (Im y_g), columns 2t, 2t+1
            out[gi][0] = make_float2(d[0], d[2]);
            out[gi][1] = make_float2(d[1], d[3]);
        }
        if (src == dst) __syncthreads();  // in place: every input is read before any write
#pragma unroll
        for (int gi = 0; gi < GPW; gi++) {
            const int grp = warp * GPW + gi;
#pragma unroll
            for (int u = 0; u < 2; u++) {
                const int bb = grp * 8 + 2 * t + u;
                const int jj = bb & (Ns - 1);
                dst[tc_addr((bb - jj) * 8 + jj + g * Ns)] = out[gi][u];
            }
        }
        __syncthreads();
    }
    template <int SIGN, int p>
    // pass p reads b0 (p even) or b1 (p odd) and writes the other one; with a
    // single buffer (b0 == b1) the passes work in place
    __device__ __forceinline__ void tc_passes(float2 *b0, float2 *b1, const float2 *cst, int tid) const
    {
        if constexpr (p < P) {
            const float2 *src = (p & 1) ? b1 : b0;
            float2 *dst = (p & 1) ? b0 : b1;
            if constexpr (radix(p) == 16) tc_pass16<SIGN, p>(src, dst, cst, tid);
            else tc_pass8<SIGN, p>(src, dst, cst, tid);
            tc_passes<SIGN, p + 1>(b0, b1, cst, tid);
        }
    }
    // x (thread-strided) <- DFT_N^SIGN x through the tensor-core passes.  With
    // two buffers the passes alternate between them (one barrier per pass),
    // starting in the buffer the FP32 transforms would write next, and the
    // ping-pong parity is left pointing at the buffer not read last, so the
    // next transform's first write cannot race the final read-back; with one
    // buffer every pass works in place and the transform ends with a barrier.
    template <int SIGN>
    __device__ __forceinline__ void tc_transform(float2 (&x)[NE], float2 *buf0, const float2 *cst, int tid)
    {
        float2 *cur = buf0 + (BUFS == 2 && f32.ph ? LBUF : 0);
        float2 *oth = BUFS == 2 ? buf0 + (f32.ph ? 0 : LBUF) : cur;
#pragma unroll
        for (int e = 0; e < NE; e++) cur[tc_addr(tid + e * NT)] = x[e];
        __syncthreads();
        tc_passes<SIGN, 0>(cur, oth, cst, tid);
        const float2 *last = (P & 1) ? oth : cur;
#pragma unroll
        for (int e = 0; e < NE; e++) x[e] = last[tc_addr(tid + e * NT)];
        if constexpr (BUFS == 2) f32.ph ^= (P & 1) ? 0 : 1;
        else __syncthreads();
    }
    __device__ __forceinline__ void fwd(float2 (&x)[NE], float2 *buf, const float2 *cst, int tid)
    {
        if (!tc) {
            f32.fwd(x, buf, cst, tid);
            return;
        }
#pragma unroll
        for (int e = 0; e < NE; e++) x[e] = cmul(x[e], f32.dm[e]);
        tc_transform<-1>(x, buf, cst, tid);
    }
    __device__ __forceinline__ void adj(float2 (&x)[NE], float2 *buf, const float2 *cst, int tid)
    {
        if (!tc) {
            f32.adj(x, buf, cst, tid);
            return;
        }
        tc_transform<+1>(x, buf, cst, tid);
#pragma unroll
        for (int e = 0; e < NE; e++) x[e] = cmulc(x[e], f32.dm[e]);
    }
};

}  // namespace tmr
