// lanczos.cuh -- the spectral start's leading eigenvector by the Lanczos
// method, shared by the per-row solvers.
//
// The spectral start wants the leading eigenvector of
// A = Q^H diag(tau) Q / (J N) (tau = min(y / mean y, clip)).  The power
// iteration needs about a hundred products with A on the mode-model rows; k
// Lanczos steps (k <= 16) reach the same vector in k products: from
// v_0 = t / ||t||, step j forms w = A v_j and orthogonalises it against every
// v_0 .. v_j by two passes of classical Gram-Schmidt (coefficients
// h_l = <v_l, w>); alpha_j is the real part of v_j's two coefficients,
// beta_j = ||w||, and v_{j+1} = w / beta_j, until j = k - 1 or
// beta_j <= 1e-6 alpha_0 (an invariant subspace).  The start is
// t = sum_l s_l v_l with s the eigenvector of the largest eigenvalue of the
// tridiagonal T (alpha on the diagonal, beta beside it), signed so that
// s_0 >= 0.  The Lanczos vectors live in a global workspace region of the CTA
// (or cluster), or, for the one-CTA-per-row solver where they fit, in the
// SM's tensor memory (lanczos_start_tmem); each thread reads back only the
// elements it wrote.
#pragma once

#include "common.cuh"
#include "internal.h"
#include "tmem.cuh"

namespace tmr {

// Eigenvalues of T below x (Sturm sequence of the LDL^T pivots).
static __device__ __forceinline__ int sturm_below(const float *a, const float *b, int n, float x)
{
    int c = 0;
    float d = 1.f;
    for (int i = 0; i < n; i++) {
        d = (a[i] - x) - (i > 0 ? b[i - 1] * b[i - 1] / d : 0.f);
        if (d == 0.f) d = -1e-30f;
        c += d < 0.f;
    }
    return c;
}

// s <- unit eigenvector of the largest eigenvalue of the symmetric tridiagonal
// T (a[0..n) diagonal, b[i] = T[i][i+1]), s[0] >= 0.  Called by all 32 lanes
// of one warp: the eigenvalue by multisection (each lane counts the
// eigenvalues below one of 32 points of the Gershgorin interval, six rounds),
// then two steps of inverse iteration with (T - lambda I) factored by Gaussian
// elimination with partial pivoting on lane 0.
static __device__ void tridiag_top_eigvec(const float *a, const float *b, int n, float *s)
{
    const int lane = threadIdx.x & 31;
    if (n == 1) {
        if (lane == 0) s[0] = 1.f;
        __syncwarp();
        return;
    }
    float lo = 3.4e38f, hi = -3.4e38f, scale = 0.f;
    for (int i = 0; i < n; i++) {
        const float r = (i > 0 ? fabsf(b[i - 1]) : 0.f) + (i < n - 1 ? fabsf(b[i]) : 0.f);
        lo = fminf(lo, a[i] - r);
        hi = fmaxf(hi, a[i] + r);
        scale = fmaxf(scale, fabsf(a[i]) + r);
    }
    for (int round = 0; round < 6; round++) {
        const float w = (hi - lo) / 33.f;
        const float x = lo + w * (float)(lane + 1);
        // lambda_max >= x exactly when fewer than n eigenvalues lie below x
        const unsigned above = __ballot_sync(0xffffffffu, sturm_below(a, b, n, x) <= n - 1);
        const int last = above ? 31 - __clz(above) : -1;  // the highest point still below lambda_max
        const float nlo = last >= 0 ? lo + w * (float)(last + 1) : lo;
        const float nhi = last < 31 ? lo + w * (float)(last + 2) : hi;
        lo = nlo;
        hi = nhi;
    }
    if (lane == 0) {
        const float lam = 0.5f * (lo + hi), tiny = 1e-7f * (scale > 0.f ? scale : 1.f);
        float x[kMaxLanczos], d[kMaxLanczos], du[kMaxLanczos], dl[kMaxLanczos], du2[kMaxLanczos];
        for (int i = 0; i < n; i++) x[i] = 1.f;
        for (int step = 0; step < 2; step++) {
            for (int i = 0; i < n; i++) {
                d[i] = a[i] - lam;
                du[i] = i < n - 1 ? b[i] : 0.f;
                dl[i] = i < n - 1 ? b[i] : 0.f;
                du2[i] = 0.f;
            }
            // eliminate below the diagonal; a row swap brings the fill-in du2
            for (int i = 0; i < n - 1; i++) {
                if (fabsf(d[i]) >= fabsf(dl[i])) {
                    if (d[i] == 0.f) d[i] = tiny;
                    const float f = dl[i] / d[i];
                    d[i + 1] -= f * du[i];
                    x[i + 1] -= f * x[i];
                } else {
                    const float f = d[i] / dl[i];
                    d[i] = dl[i];
                    const float t = d[i + 1];
                    d[i + 1] = du[i] - f * t;
                    if (i < n - 2) {
                        du2[i] = du[i + 1];
                        du[i + 1] = -f * du[i + 1];
                    }
                    du[i] = t;
                    const float r = x[i];
                    x[i] = x[i + 1];
                    x[i + 1] = r - f * x[i + 1];
                }
            }
            if (d[n - 1] == 0.f) d[n - 1] = tiny;
            x[n - 1] /= d[n - 1];
            x[n - 2] = (x[n - 2] - du[n - 2] * x[n - 1]) / d[n - 2];
            for (int i = n - 3; i >= 0; i--) x[i] = (x[i] - du[i] * x[i + 1] - du2[i] * x[i + 2]) / d[i];
            float nrm = 0.f;
            for (int i = 0; i < n; i++) nrm = fmaf(x[i], x[i], nrm);
            const float inv = nrm > 0.f && isfinite(nrm) ? rsqrtf(nrm) : 0.f;
            for (int i = 0; i < n; i++) x[i] *= inv;
        }
        const float sg = x[0] < 0.f ? -1.f : 1.f;
        for (int i = 0; i < n; i++) s[i] = sg * x[i];
    }
    __syncwarp();
}

// Step j's update coefficients from the sweep's partial sums (all threads):
// pv holds <v_l, w> for l <= j and pg <v_l, v_j> for l < j (re, im pairs);
// the new Gram column goes to Gw, the coefficients c (see lanczos_start) to
// hc and alpha_j to la[j].  Ends with a block barrier.
template <class Reduce>
__device__ __forceinline__ void lanczos_coefficients(int j, float (&pv)[32], float (&pg)[32], float2 *Gw,
                                                     const float *red, float *la, float *hc, Reduce &&reduce)
{
    const int tid = threadIdx.x, lane = tid & 31;
    reduce(pv, 2 * (j + 1));
    if (tid < 2 * (j + 1)) hc[tid] = red[tid];
    if (j > 0) {
        reduce(pg, 2 * j);
        if (tid < 32) {
            if (lane < j) Gw[lane * kMaxLanczos + j] = make_float2(red[2 * lane], red[2 * lane + 1]);
            if (lane == j) {
#pragma unroll
                for (int l = 0; l < kMaxLanczos; l++)
                    if (l < j) Gw[j * kMaxLanczos + l] = make_float2(red[2 * l], -red[2 * l + 1]);
            }
        }
    }
    __syncwarp();
    if (tid < 32) {
        float2 c = make_float2(0.f, 0.f);
        if (lane <= j) {
            c = make_float2(hc[2 * lane], hc[2 * lane + 1]);
#pragma unroll
            for (int m = 0; m < kMaxLanczos; m++) {
                if (m <= j && m != lane) {
                    const float2 g = Gw[lane * kMaxLanczos + m], hm = make_float2(hc[2 * m], hc[2 * m + 1]);
                    c.x -= g.x * hm.x - g.y * hm.y;
                    c.y -= g.x * hm.y + g.y * hm.x;
                }
            }
        }
        __syncwarp();
        if (lane <= j) {
            hc[2 * lane] = c.x;
            hc[2 * lane + 1] = c.y;
        }
        if (lane == j) la[j] = c.x;
    }
    __syncthreads();
}

// The Lanczos start on this CTA's nloc elements (thread-strided by blockDim.x).
//   ts   in: the seed vector; out: the Ritz vector (unit norm)
//   gs   scratch, nloc elements
//   V    Lanczos vectors: vector l's element i at V[l vs + i] (global)
//   Gw   kMaxLanczos^2 complex64 of global scratch: the Gram matrix of the
//        stored Lanczos vectors (row l at Gw + l kMaxLanczos)
//   red  the row's reduction results (reduce writes its sums there)
//   lz   48 floats of shared scratch (alpha, beta, s); hc 32 floats (h, then c)
//   applyA()      gs <- A ts on the whole row (synchronises before and after)
//   reduce(v, n)  sums v[0..n) over the row into red[0..n), then synchronises
// All threads call.
//
// The second Gram-Schmidt pass is taken from the Gram matrix G = V^H V of the
// stored vectors instead of a second sweep over them: with h = V^H w the
// first pass's coefficients, the second pass's would be
// V^H (w - V h) = h - G h, so w is updated once by c = h + (h - G h), which
// with G_ll = 1 is c_l = h_l - sum_{m != l} G_lm h_m.  G's new column,
// <v_l, v_j>, comes from the same sweep that forms h (each v_l is loaded once
// for both dots), so each step reads the stored vectors twice (the h sweep
// and the update) instead of four times.  In exact arithmetic this is the
// two-pass update; in FP32 it keeps the Ritz vector as close to the FP64
// two-pass result as the explicit second pass does (about 1e-6 relative on
// the mode-model rows), where one pass alone drifts by up to 1e-2 at k = 16.
// (Forming G's column in the update sweep instead, with the v_l held in
// registers, saves a reduction but spills registers of the L-BFGS loop that
// shares the kernel, which then runs 16 % slower.)
template <class ApplyA, class Reduce>
__device__ void lanczos_start(int k, int nloc, float2 *ts, float2 *gs, float2 *V, size_t vs, float2 *Gw,
                              const float *red, float *lz, float *hc, ApplyA &&applyA, Reduce &&reduce)
{
    const int tid = threadIdx.x, BT = blockDim.x;
    float *la = lz, *lb = lz + kMaxLanczos, *ls = lz + 2 * kMaxLanczos;
    {
        float pv[32] = {0.f};
        for (int i = tid; i < nloc; i += BT) pv[0] += cabs2(ts[i]);
        reduce(pv, 1);
        const float nr = red[0];
        const float inv = nr > 0.f ? rsqrtf(nr) : 0.f;
        for (int i = tid; i < nloc; i += BT) {
            const float2 v = cscale(ts[i], inv);
            ts[i] = v;
            V[i] = v;
        }
    }
    int kk = k;
    float alpha0 = 0.f;
    for (int j = 0; j < k; j++) {
        applyA();
        float pv[32], pg[32];
#pragma unroll
        for (int q = 0; q < 32; q++) pv[q] = pg[q] = 0.f;
#pragma unroll 2
        for (int i = tid; i < nloc; i += BT) {
            const float2 w = gs[i], vj = ts[i];
#pragma unroll
            for (int l = 0; l < kMaxLanczos; l++) {
                if (l <= j) {
                    const float2 v = V[(size_t)l * vs + i];
                    pv[2 * l] = fmaf(v.x, w.x, fmaf(v.y, w.y, pv[2 * l]));
                    pv[2 * l + 1] = fmaf(v.x, w.y, fmaf(-v.y, w.x, pv[2 * l + 1]));
                    if (l < j) {
                        pg[2 * l] = fmaf(v.x, vj.x, fmaf(v.y, vj.y, pg[2 * l]));
                        pg[2 * l + 1] = fmaf(v.x, vj.y, fmaf(-v.y, vj.x, pg[2 * l + 1]));
                    }
                }
            }
        }
        lanczos_coefficients(j, pv, pg, Gw, red, la, hc, reduce);
        const float alpha = la[j];
        if (j == 0) alpha0 = alpha;
#pragma unroll
        for (int q = 0; q < 32; q++) pv[q] = 0.f;
#pragma unroll 2
        for (int i = tid; i < nloc; i += BT) {
            float2 w = gs[i];
#pragma unroll
            for (int l = 0; l < kMaxLanczos; l++) {
                if (l <= j) {
                    const float2 v = V[(size_t)l * vs + i];
                    const float cr = hc[2 * l], ci = hc[2 * l + 1];
                    w.x -= cr * v.x - ci * v.y;
                    w.y -= cr * v.y + ci * v.x;
                }
            }
            gs[i] = w;
            pv[0] = fmaf(w.x, w.x, fmaf(w.y, w.y, pv[0]));
        }
        reduce(pv, 1);
        const float beta = sqrtf(red[0]);
        if (tid == 0) lb[j] = beta;
        if (j == k - 1 || !(beta > 1e-6f * alpha0)) {
            kk = j + 1;
            break;
        }
        const float inv = 1.f / beta;
        for (int i = tid; i < nloc; i += BT) {
            const float2 v = cscale(gs[i], inv);
            ts[i] = v;
            V[(size_t)(j + 1) * vs + i] = v;
        }
    }
    __syncthreads();
    if (tid < 32) tridiag_top_eigvec(la, lb, kk, ls);
    __syncthreads();
    for (int i = tid; i < nloc; i += BT) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < kMaxLanczos; l++) {
            if (l < kk) {
                const float2 v = V[(size_t)l * vs + i];
                acc.x = fmaf(ls[l], v.x, acc.x);
                acc.y = fmaf(ls[l], v.y, acc.y);
            }
        }
        ts[i] = acc;
    }
    __syncthreads();
}

// The same start with the Lanczos vectors in tensor memory (one CTA per row,
// nloc = N).  Thread tid keeps elements i = tid + e BT, e < ept, of every
// vector in its own lane; vectors l .. l + 3 of element e sit in 8
// consecutive columns from tv + 2 (e KM + l), KM = k rounded up to a multiple
// of 4, so one 8-column load brings four of them.  Every thread runs all ept
// steps of each sweep (the tensor-memory loads and stores are warp-wide);
// steps past nloc move zeros.  The arithmetic and its order are those of
// lanczos_start.
template <class ApplyA, class Reduce>
__device__ void lanczos_start_tmem(int k, int nloc, int ept, uint32_t tv, float2 *ts, float2 *gs, float2 *Gw,
                                   const float *red, float *lz, float *hc, ApplyA &&applyA, Reduce &&reduce)
{
    const int tid = threadIdx.x, BT = blockDim.x;
    const int KM = (k + 3) & ~3;
    float *la = lz, *lb = lz + kMaxLanczos, *ls = lz + 2 * kMaxLanczos;
    auto col = [&](int l, int e) { return tv + (uint32_t)(2 * (e * KM + l)); };
    tmem_fence_after_sync();
    {
        float pv[32] = {0.f};
        for (int i = tid; i < nloc; i += BT) pv[0] += cabs2(ts[i]);
        reduce(pv, 1);
        const float nr = red[0];
        const float inv = nr > 0.f ? rsqrtf(nr) : 0.f;
        for (int e = 0; e < ept; e++) {
            const int i = tid + e * BT;
            float2 v = make_float2(0.f, 0.f);
            if (i < nloc) {
                v = cscale(ts[i], inv);
                ts[i] = v;
            }
            tmem_st2(col(0, e), v.x, v.y);
        }
        tmem_wait_st();
    }
    int kk = k;
    float alpha0 = 0.f;
    for (int j = 0; j < k; j++) {
        applyA();
        float pv[32], pg[32];
#pragma unroll
        for (int q = 0; q < 32; q++) pv[q] = pg[q] = 0.f;
        for (int e = 0; e < ept; e++) {
            const int i = tid + e * BT;
            const bool in = i < nloc;
            const float2 w = in ? gs[i] : make_float2(0.f, 0.f), vj = in ? ts[i] : make_float2(0.f, 0.f);
#pragma unroll
            for (int g = 0; g < kMaxLanczos / 4; g++) {
                if (4 * g <= j) {
                    uint32_t r[8];
                    tmem_ld8(col(4 * g, e), r);
                    tmem_wait_ld();
                    tmem_reg_ready(r);
                    if (in) {
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            const int l = 4 * g + q;
                            if (l <= j) {
                                const float2 v = make_float2(__uint_as_float(r[2 * q]), __uint_as_float(r[2 * q + 1]));
                                pv[2 * l] = fmaf(v.x, w.x, fmaf(v.y, w.y, pv[2 * l]));
                                pv[2 * l + 1] = fmaf(v.x, w.y, fmaf(-v.y, w.x, pv[2 * l + 1]));
                                if (l < j) {
                                    pg[2 * l] = fmaf(v.x, vj.x, fmaf(v.y, vj.y, pg[2 * l]));
                                    pg[2 * l + 1] = fmaf(v.x, vj.y, fmaf(-v.y, vj.x, pg[2 * l + 1]));
                                }
                            }
                        }
                    }
                }
            }
        }
        lanczos_coefficients(j, pv, pg, Gw, red, la, hc, reduce);
        const float alpha = la[j];
        if (j == 0) alpha0 = alpha;
#pragma unroll
        for (int q = 0; q < 32; q++) pv[q] = 0.f;
        for (int e = 0; e < ept; e++) {
            const int i = tid + e * BT;
            const bool in = i < nloc;
            float2 w = in ? gs[i] : make_float2(0.f, 0.f);
#pragma unroll
            for (int g = 0; g < kMaxLanczos / 4; g++) {
                if (4 * g <= j) {
                    uint32_t r[8];
                    tmem_ld8(col(4 * g, e), r);
                    tmem_wait_ld();
                    tmem_reg_ready(r);
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const int l = 4 * g + q;
                        if (l <= j) {
                            const float2 v = make_float2(__uint_as_float(r[2 * q]), __uint_as_float(r[2 * q + 1]));
                            const float cr = hc[2 * l], ci = hc[2 * l + 1];
                            w.x -= cr * v.x - ci * v.y;
                            w.y -= cr * v.y + ci * v.x;
                        }
                    }
                }
            }
            if (in) {
                gs[i] = w;
                pv[0] = fmaf(w.x, w.x, fmaf(w.y, w.y, pv[0]));
            }
        }
        reduce(pv, 1);
        const float beta = sqrtf(red[0]);
        if (tid == 0) lb[j] = beta;
        if (j == k - 1 || !(beta > 1e-6f * alpha0)) {
            kk = j + 1;
            break;
        }
        const float inv = 1.f / beta;
        for (int e = 0; e < ept; e++) {
            const int i = tid + e * BT;
            float2 v = make_float2(0.f, 0.f);
            if (i < nloc) {
                v = cscale(gs[i], inv);
                ts[i] = v;
            }
            tmem_st2(col(j + 1, e), v.x, v.y);
        }
        tmem_wait_st();
    }
    __syncthreads();
    if (tid < 32) tridiag_top_eigvec(la, lb, kk, ls);
    __syncthreads();
    for (int e = 0; e < ept; e++) {
        const int i = tid + e * BT;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int g = 0; g < kMaxLanczos / 4; g++) {
            if (4 * g < kk) {
                uint32_t r[8];
                tmem_ld8(col(4 * g, e), r);
                tmem_wait_ld();
                tmem_reg_ready(r);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int l = 4 * g + q;
                    if (l < kk) {
                        acc.x = fmaf(ls[l], __uint_as_float(r[2 * q]), acc.x);
                        acc.y = fmaf(ls[l], __uint_as_float(r[2 * q + 1]), acc.y);
                    }
                }
            }
        }
        if (i < nloc) ts[i] = acc;
    }
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
}

}  // namespace tmr
