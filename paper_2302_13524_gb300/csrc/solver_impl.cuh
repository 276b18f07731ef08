// solver_impl.cuh -- persistent per-row retrieval (Algorithm 1) on thread-block
// clusters.  The kernel is a template over the transform policy (xform.cuh);
// solver.cu instantiates it for powers of two, solver_bs.cu for the other
// lengths (Bluestein).
//
// One cluster of J/G CTAs solves one TM row at a time; rows come from an
// atomic work counter, so a launch of (clusters x J/G) CTAs walks the whole
// matrix.  Each CTA runs G teams, team g of CTA c owning mask j = c G + g:
//   registers: the mask constants of the transform, z_j = F(d_j .* t) (the
//              current fields), y_j and w_j = F(d_j .* p), all in the
//              transform's thread-strided layout;
//   shared:    the FFT exchange buffers and the transform's constants, a
//              1/(J/G) slice of every length-N vector (t, g and the L-BFGS
//              pairs), and two receive areas.
// Exchanges between the CTAs of a cluster are pushes: a CTA stores its data
// into its peers' shared memory (distributed shared memory) and then arrives at
// the cluster barrier, so that after the barrier every read is local.
//   X[N]      full direction p (or t), assembled from the owners' slices; once
//             a CTA has read X into registers, X serves as its FFT exchange
//             buffer until the next gather;
//   Y[J][SL]  the J masks' adjoint outputs for my slice (summed into g);
//   part[2][J][32]  reduction partials (two buffers used alternately).
//
// One iteration (Algorithm 1: f and its gradient by FFT, then the L-BFGS step):
//   A  p = -H g on my slice from the compact L-BFGS form
//      H = gamma I + [S gamma Y] M [S^T; gamma Y^T] (Byrd, Nocedal & Schnabel
//      1994), coefficients from the Gram scalars; push the slice into X.  B1.
//   C  w_j = F(d_j .* p)                                     (J FFTs per row)
//   D  sums of the quartic phi(a) = f(t + a p) = sum_i (r_i - 2 a Re(conj z_i w_i)
//      - a^2 |w_i|^2)^2; push.  B2.  Exact minimiser from phi'(a) = 0.
//   E  t += a p, z += a w, r = y - |z|^2, u = z .* r (registers)
//   F  v_j = conj(d_j) .* F^H u_j; push each slice to its owner.  B3.
//   G  g = -4 sum_j v_j on my slice (Eq. derivative), pair s = a p,
//      y = g_new - g_old, every Gram dot product in one batched reduction.  B4.
// Four cluster barriers and two FFT batches per iteration.
//
// Buffer reuse across barriers: X is read (step C) before its reader arrives at
// B2 and written again only after B4; Y is written after B2 and read before
// B4; a part buffer is read right after the barrier that completes it and
// rewritten two reductions later.  No CTA touches a peer's shared memory after
// the barrier that hands out the final (past-the-end) row, so CTAs may exit.
#pragma once

#include <cooperative_groups.h>

#include <cuda_fp16.h>

#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "fft.cuh"
#include "cost.cuh"
#include "internal.h"
#include "lanczos.cuh"
#include "xform.cuh"

namespace cg = cooperative_groups;

namespace tmr {

enum { ROW_MAXITER = 0, ROW_CONVERGED = 1, ROW_ZERO = 2, ROW_NUMERIC = 3 };
enum { INIT_RANDOM = 0, INIT_BP = 1, INIT_SPECTRAL = 2 };

constexpr int kSlots = kMaxMem + 1;  // m+1 slots: the new pair never overwrites a live one
constexpr int kParts = 32;           // values per reduction: one per lane of a warp
// the Lanczos start keeps alpha, beta and s in Gram::SY, unused before the first pair
static_assert(kSlots * kSlots >= 3 * kMaxLanczos && kSlots * kSlots >= 2 * kMaxLanczos,
              "Lanczos scratch in Gram::SY and Gram::YY");
static_assert(4 * kSlots + 3 <= kParts, "reduction width");
// layout of the per-iteration dot products: 4 per age k (s_k.y, y_k.y, s_k.g,
// y_k.g with the new y and g), then these three
constexpr int kIdxSS = 4 * kSlots, kIdxGG = 4 * kSlots + 1, kIdxF = 4 * kSlots + 2;

// L-BFGS scalars, replicated in every CTA of the cluster: each CTA computes
// them from identical sums added in the same order, so they agree bit for bit
// and every CTA takes the same branches.  FP32 like the rest of the path (the
// FP64 pipe of this part is a small fraction of its FP32 rate, and these
// scalars sit on the critical path of every iteration).  Pairs are indexed by
// age (0 = oldest); slot[] maps an age to its physical vector slot, and
// slot[np] is the free slot that receives the next pair.
struct Gram {
    float SY[kSlots][kSlots];  // s_i^T y_j, ages i <= j
    float YY[kSlots][kSlots];  // y_i^T y_j, ages i <= j
    float rD[kSlots];          // 1 / s_i^T y_i
    float Sg[kSlots], Yg[kSlots];
    float c1[kSlots], c2[kSlots];  // direction coefficients by age (c2 includes gamma)
    float gamma, gg, f, sumy, alpha;
    float yscale, tsc;  // the row's intensity scale 4^-j and its t scale 2^j
    float red[kParts];  // the last cluster-wide sums
    int slot[kSlots];
    int np;
    int status, done, stop, early, row;
};

// Global minimiser of phi(a) = c0 + c1 a + c2 a^2 + c3 a^3 + c4 a^4 (c4 > 0)
// over the real line.  phi' = g(a) = c1 + 2 c2 a + 3 c3 a^2 + 4 c4 a^3 rises at
// both ends; with three real roots the middle one is a local maximum of phi,
// so the minimiser is the leftmost or the rightmost root.  The critical
// points r1 < r2 of g (roots of a quadratic) say which case holds; each
// needed root is bracketed (expanding outwards from a point of known sign)
// and found by Newton steps kept inside the bracket.  Ties go to the smallest
// positive root.  c4 == 0 means w == 0: no step.
static __device__ float quartic_argmin_safe(const float *c)
{
    const float c1 = c[1], c2 = c[2], c3 = c[3], c4 = c[4];
    if (!(c4 > 0.f)) {
        if (c2 > 0.f && c3 == 0.f) return -c1 / (2.f * c2);
        return 0.f;
    }
    auto g = [&](float a) { return fmaf(fmaf(fmaf(4.f * c4, a, 3.f * c3), a, 2.f * c2), a, c1); };
    auto dg = [&](float a) { return fmaf(fmaf(12.f * c4, a, 6.f * c3), a, 2.f * c2); };
    auto phi = [&](float a) { return a * fmaf(fmaf(fmaf(c4, a, c3), a, c2), a, c1); };
    // a root in [lo, hi] with g(lo) <= 0 <= g(hi)
    auto solve = [&](float lo, float hi, float glo, float ghi) {
        float a = (ghi != glo) ? lo - glo * (hi - lo) / (ghi - glo) : 0.5f * (lo + hi);
        if (!(a >= lo && a <= hi)) a = 0.5f * (lo + hi);
        for (int it = 0; it < 60; it++) {
            const float ga = g(a);
            if (ga == 0.f) break;
            if (ga < 0.f) lo = a;
            else hi = a;
            const float d = dg(a);
            float na = (d != 0.f) ? a - ga / d : 0.5f * (lo + hi);
            if (!(na > lo && na < hi)) na = 0.5f * (lo + hi);
            if (na == a || hi - lo <= 4e-7f * fmaxf(fabsf(lo), fabsf(hi))) {
                a = na;
                break;
            }
            a = na;
        }
        return a;
    };
    // walk from x0 (sign of g known) in direction dir until g changes sign
    auto bracket = [&](float x0, float dir, float &lo, float &hi, float &glo, float &ghi) {
        const float g0 = g(x0);
        float step = fmaxf(1.f, fabsf(x0));
        float x = x0, gx = g0;
        for (int it = 0; it < 80; it++) {
            const float xn = x + dir * step;
            const float gn = g(xn);
            if ((dir > 0.f && gn >= 0.f) || (dir < 0.f && gn <= 0.f)) {
                if (dir > 0.f) { lo = x; glo = gx; hi = xn; ghi = gn; }
                else { lo = xn; glo = gn; hi = x; ghi = gx; }
                return;
            }
            x = xn;
            gx = gn;
            step *= 2.f;
        }
        lo = hi = x;
        glo = ghi = gx;
    };
    float cand[2];
    int nc = 0;
    const float qa = 12.f * c4, qb = 6.f * c3, qc = 2.f * c2;
    const float disc = qb * qb - 4.f * qa * qc;
    bool three = false;
    float r1 = 0.f, r2 = 0.f;
    if (disc > 0.f) {
        const float sq = sqrtf(disc);
        const float q = -0.5f * (qb + (qb >= 0.f ? sq : -sq));
        r1 = q / qa;
        r2 = (q != 0.f) ? qc / q : r1;
        if (r1 > r2) {
            const float t = r1;
            r1 = r2;
            r2 = t;
        }
        three = g(r1) >= 0.f && g(r2) <= 0.f;
    }
    float lo, hi, glo, ghi;
    if (three) {
        bracket(r1, -1.f, lo, hi, glo, ghi);
        cand[nc++] = solve(lo, hi, glo, ghi);
        bracket(r2, +1.f, lo, hi, glo, ghi);
        cand[nc++] = solve(lo, hi, glo, ghi);
    } else {
        const float g0 = g(0.f);
        if (g0 == 0.f) return 0.f;
        bracket(0.f, g0 < 0.f ? +1.f : -1.f, lo, hi, glo, ghi);
        cand[nc++] = solve(lo, hi, glo, ghi);
    }
    float best = cand[0], bestv = phi(cand[0]);
    for (int k = 1; k < nc; k++) {
        const float v = phi(cand[k]);
        if (v < bestv || (v == bestv && cand[k] > 0.f && (best <= 0.f || cand[k] < best))) {
            best = cand[k];
            bestv = v;
        }
    }
    return best;
}

// The same minimiser from the closed-form roots of the cubic phi'(a) = 0
// (Cardano's formula for one real root, the trigonometric form for three),
// each polished by Newton steps on phi' in FP32, the up to three polishings on
// lanes 0..2 of a warp (every lane of the warp calls it and gets the same
// result); among the real roots the one with the smallest phi wins (ties: the
// smallest positive root).  The roots are found for the variable b = 2^-k a,
// with k such that 2^(4k) c4 lies in [1/2, 8): an exact power-of-two
// substitution that keeps the coefficients near 1 when the step's fields are
// tiny (late iterations), where 1 / c4 and the cubic's coefficients would
// leave FP32 range.  Falls back to the bracketing search when c4 <= 0 or a
// root comes out non-finite.
static __device__ float quartic_argmin_warp(const float *c, int lane)
{
    if (!(c[4] > 0.f)) return quartic_argmin_safe(c);
    int e;
    frexpf(c[4], &e);  // c4 = f 2^e, f in [1/2, 1)
    const int ks = -(e >> 2);  // -floor(e / 4)
    const float c1 = ldexpf(c[1], ks), c2 = ldexpf(c[2], 2 * ks), c3 = ldexpf(c[3], 3 * ks),
                c4 = ldexpf(c[4], 4 * ks);
    auto g = [&](float a) { return fmaf(fmaf(fmaf(4.f * c4, a, 3.f * c3), a, 2.f * c2), a, c1); };
    auto dg = [&](float a) { return fmaf(fmaf(12.f * c4, a, 6.f * c3), a, 2.f * c2); };
    auto phi = [&](float a) { return a * fmaf(fmaf(fmaf(c4, a, c3), a, c2), a, c1); };
    const float inv = 1.f / c4;
    const float B3 = 0.25f * c3 * inv;
    const float C = 0.5f * c2 * inv, D = 0.25f * c1 * inv;
    const float p = fmaf(-3.f * B3, B3, C);
    const float q = fmaf(B3, fmaf(2.f * B3, B3, -C), D);
    const float hp = p * (1.f / 3.f), hq = 0.5f * q;
    const float disc = fmaf(hq, hq, hp * hp * hp);
    float a = 0.f;
    int nc;
    if (disc > 0.f) {
        nc = 1;
        if (lane == 0) {
            const float u = cbrtf(-hq - copysignf(sqrtf(disc), hq));
            a = (u != 0.f ? u - hp / u : 0.f) - B3;
        }
    } else {
        nc = 3;
        if (lane < 3) {
            const float r = sqrtf(fmaxf(-hp, 0.f));
            const float r3 = r * r * r;
            const float arg = r3 > 0.f ? fminf(fmaxf(-hq / r3, -1.f), 1.f) : 0.f;
            const float th = acosf(arg) * (1.f / 3.f);
            const float tr = 2.0943951023931955f;  // 2 pi / 3
            a = 2.f * r * cosf(lane == 0 ? th : (lane == 1 ? th - tr : th + tr)) - B3;
        }
    }
    if (lane < nc) {
        for (int it = 0; it < 4; it++) {
            const float d = dg(a);
            if (!(d != 0.f)) break;
            const float na = a - g(a) / d;
            if (!isfinite(na) || na == a) break;
            a = na;
        }
    }
    const float v = phi(a);
    float best = 0.f, bestv = 0.f;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float ak = __shfl_sync(0xffffffffu, a, k), vk = __shfl_sync(0xffffffffu, v, k);
        if (k < nc) {
            bad = bad || !isfinite(ak);
            if (k == 0 || vk < bestv || (vk == bestv && ak > 0.f && (best <= 0.f || ak < best))) {
                best = ak;
                bestv = vk;
            }
        }
    }
    if (bad) return quartic_argmin_safe(c);
    return ldexpf(best, ks);
}

// Compact-form coefficients, run by one warp (lane i owns age i):
// p = -(gamma g + sum_i c1_i s_i + sum_i c2_i y_i), c2 already scaled by gamma.
// R c2 = -S^T g is solved by back substitution and R^T c1 =
// -(D + gamma Y^T Y) c2 - gamma Y^T g by forward substitution, each step
// broadcasting the new unknown with a shuffle.  Falls back to p = -g (and
// clears the history) when there is no pair or the result is not a descent
// direction.
// Exponent j of a row's intensity scale: with the mean intensity ybar in
// [2^(e-1), 2^e), j = floor(e / 2), so y 4^-j has a mean in [1/2, 2), rows
// whose mean is already there keep j = 0, and scaling y by 4^k moves j by
// exactly k; 0 for a non-positive or non-finite mean.
static __device__ __forceinline__ int row_scale_exp(float sumy, int K)
{
    const float yb = sumy / (float)K;
    if (!(yb > 0.f) || !isfinite(yb)) return 0;
    int e;
    frexpf(yb, &e);
    return e >> 1;  // floor(e / 2) for either sign
}

static __device__ void lbfgs_coefficients_warp(Gram &G, int lane)
{
    const int np = G.np;
    float c1 = 0.f, c2 = 0.f, gamma = 1.f;
    bool ok = false;
    if (np > 0) {
        gamma = G.SY[np - 1][np - 1] / G.YY[np - 1][np - 1];
        const bool mine = lane < np;
        float acc = mine ? -G.Sg[lane] : 0.f;
        for (int j = np - 1; j >= 0; j--) {
            if (lane == j) c2 = acc * G.rD[j];
            const float cj = __shfl_sync(0xffffffffu, c2, j);
            if (lane < j) acc = fmaf(-G.SY[lane][j], cj, acc);
        }
        float yc = 0.f;
        for (int j = 0; j < np; j++) {
            const float cj = __shfl_sync(0xffffffffu, c2, j);
            if (mine) yc = fmaf(G.YY[lane < j ? lane : j][lane < j ? j : lane], cj, yc);
        }
        float acc1 = mine ? -G.SY[lane][lane] * c2 - gamma * (G.Yg[lane] + yc) : 0.f;
        for (int j = 0; j < np; j++) {
            if (lane == j) c1 = acc1 * G.rD[j];
            const float cj = __shfl_sync(0xffffffffu, c1, j);
            if (mine && lane > j) acc1 = fmaf(-G.SY[j][lane], cj, acc1);
        }
        float t = mine ? fmaf(c1, G.Sg[lane], gamma * c2 * G.Yg[lane]) : 0.f;
        const float pg = gamma * G.gg + warp_sum(t);  // <g, H g> = -<p, g>
        ok = pg > 0.f && isfinite(pg);
    }
    __syncwarp();
    if (lane < kSlots) {
        G.c1[lane] = (ok && lane < np) ? c1 : 0.f;
        G.c2[lane] = (ok && lane < np) ? gamma * c2 : 0.f;
    }
    if (lane == 0) {
        G.gamma = ok ? gamma : 1.f;
        if (!ok) G.np = 0;
    }
    __syncwarp();
}

// Gram bookkeeping after the batched dot products of an iteration, run by one
// warp (lane i owns age i): the new column of S^T Y and Y^T Y and the new
// S^T g, Y^T g from Gm.red, the pair test s^T y > 1e-10 |s| |y|, the shift
// that drops the oldest pair once m are held (its slot becomes the free one),
// the loss and the stopping tests, then the next direction's coefficients.
static __device__ void lbfgs_gram_update(Gram &Gm, int lane, int m, int it, int iters, double tol)
{
    const int np = Gm.np;
    const float *tot = Gm.red;
    if (lane <= np) {
        Gm.SY[lane][np] = tot[4 * lane + 0];
        Gm.YY[lane][np] = tot[4 * lane + 1];
        Gm.Sg[lane] = tot[4 * lane + 2];
        Gm.Yg[lane] = tot[4 * lane + 3];
    }
    const float sy = tot[4 * np + 0], yy = tot[4 * np + 1];
    const float fnew = tot[kIdxF];
    const bool accept = sy > 1e-10f * sqrtf(tot[kIdxSS]) * sqrtf(yy) && sy > 0.f;
    int np2 = np + (accept ? 1 : 0);
    __syncwarp();
    if (accept && lane == 0) Gm.rD[np] = 1.f / sy;
    __syncwarp();
    if (np2 > m) {
        // drop the oldest pair: age i + 1 becomes age i
        float sy_r[kSlots], yy_r[kSlots], sg = 0.f, yg = 0.f, rd = 0.f;
        int sl = 0;
        const bool mine = lane < np2 - 1;
        const int src = lane + 1;
#pragma unroll
        for (int j = 0; j < kSlots; j++) {
            sy_r[j] = (mine && j + 1 < kSlots) ? Gm.SY[src][j + 1 < kSlots ? j + 1 : 0] : 0.f;
            yy_r[j] = (mine && j + 1 < kSlots) ? Gm.YY[src][j + 1 < kSlots ? j + 1 : 0] : 0.f;
        }
        if (mine) {
            sg = Gm.Sg[src];
            yg = Gm.Yg[src];
            rd = Gm.rD[src];
        }
        // the m + 1 allocated slots rotate: the oldest pair's slot
        // becomes the free one at position m
        const int sl_old0 = Gm.slot[0];
        if (lane < m) sl = Gm.slot[lane + 1];
        __syncwarp();
        if (mine) {
#pragma unroll
            for (int j = 0; j < kSlots; j++) {
                Gm.SY[lane][j] = sy_r[j];
                Gm.YY[lane][j] = yy_r[j];
            }
            Gm.Sg[lane] = sg;
            Gm.Yg[lane] = yg;
            Gm.rD[lane] = rd;
        }
        if (lane < m) Gm.slot[lane] = sl;
        if (lane == m) Gm.slot[lane] = sl_old0;
        np2 = m;
    }
    if (lane == 0) {
        Gm.np = np2;
        Gm.gg = tot[kIdxGG];
        const float rel = fabsf(Gm.f - fnew) / fmaxf(Gm.f, 1e-30f);
        Gm.f = fnew;
        Gm.done = it + 1;
        if (!isfinite(fnew) || !isfinite(Gm.gg)) { Gm.status = ROW_NUMERIC; Gm.stop = 1; }
        else if (tol > 0.0 && rel < (float)tol) { Gm.status = ROW_CONVERGED; Gm.stop = 1; }
        else if (it + 1 < iters && (fnew == 0.f || Gm.gg == 0.f)) { Gm.status = ROW_CONVERGED; Gm.stop = 1; }
    }
    __syncwarp();
    if (!Gm.stop && it + 1 < iters) lbfgs_coefficients_warp(Gm, lane);
}

// Sum of up to 32 values over a warp by recursive halving: after the call,
// lane l of the warp holds the warp-wide sum of value l in v[0].
__device__ __forceinline__ void warp_reduce32(float (&v)[32], int lane)
{
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        const bool upper = (lane & h) != 0;
#pragma unroll
        for (int i = 0; i < h; i++) {
            const float send = upper ? v[i] : v[i + h];
            const float keep = upper ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
        }
    }
}

// Storage of the L-BFGS pairs: FP32 pairs, or BF16 pairs for the mixed-precision
// policy (the iterate, gradient and direction stay FP32).
template <class Xf, class = void>
struct MixedTrait : std::false_type {};
template <class Xf>
struct MixedTrait<Xf, std::void_t<decltype(Xf::kMixed)>> : std::integral_constant<bool, Xf::kMixed> {};
template <class Xf>
__host__ __device__ constexpr bool solver_mixed() { return MixedTrait<Xf>::value; }
template <class Xf>
using SolverHist = typename std::conditional<MixedTrait<Xf>::value, __nv_bfloat162, float2>::type;

__device__ __forceinline__ float2 hist_load(float2 v) { return v; }
__device__ __forceinline__ float2 hist_load(__nv_bfloat162 v) { return __bfloat1622float2(v); }
template <class HT>
__device__ __forceinline__ HT hist_store(float2 v)
{
    if constexpr (std::is_same<HT, float2>::value) return v;
    else return __float22bfloat162_rn(v);
}

// FP32 iterations at the end of a mixed-precision run
constexpr int kFinalFp32Iters = 10;

// G masks per CTA (G teams of NT threads, one transform each); the cluster
// has J/G CTAs.  Xf is the transform policy (xform.cuh).
template <class Xf, int G>
struct SolverCfg {
    static constexpr int NT = Xf::NT;   // threads per team (one transform)
    static constexpr int BT = G * NT;   // threads per CTA
    static constexpr int E = Xf::NE;    // registers per length-N vector
    static constexpr int NW = BT / 32;
};

template <class Xf, int G>
__host__ __device__ size_t solver_smem(int N, int J, int m)
{
    using C = SolverCfg<Xf, G>;
    const int JC = J / G;
    const size_t SL = (N + JC - 1) / JC;
    size_t f2 = (size_t)G * Xf::BUFS * Xf::LBUF /*X (team 0's first buffer) and the exchange buffers*/ +
                Xf::shared_consts(N) +
                (size_t)J * SL /*Y*/ + 2 * SL /*t, g*/ + (solver_mixed<Xf>() ? SL : 0) /*p*/;
    size_t bytes = f2 * sizeof(float2) + 2 * (size_t)(m + 1) * SL * sizeof(SolverHist<Xf>) /*pairs*/;
    bytes += sizeof(float) * ((size_t)kParts * C::NW + 2 * (size_t)JC * kParts);
    bytes = (bytes + 15) & ~(size_t)15;
    return bytes + sizeof(Gram);
}

template <class Xf, int G, int COST = COST_INTENSITY>
__global__ void __launch_bounds__(SolverCfg<Xf, G>::BT, (SolverCfg<Xf, G>::BT <= 256 && Xf::kN >= 256) ? 2 : 1)
    k_solver(SolverParams P)
{
    using C = SolverCfg<Xf, G>;
    constexpr int NT = C::NT, BT = C::BT, E = C::E, NW = C::NW;
    constexpr bool kMixed = solver_mixed<Xf>();
    using HT = SolverHist<Xf>;
    const int N = Xf::kN > 0 ? Xf::kN : P.N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cluster = cg::this_cluster();
    const int J = P.J, m = P.m, M = P.M;
    const int JC = J / G;  // CTAs in the cluster
    const int jr = (int)cluster.block_rank();
    const int tid = threadIdx.x;
    const int team = tid / NT, ttid = tid - team * NT;
    const int jm = jr * G + team;  // the mask of this thread's team
    const int SL = (N + JC - 1) / JC;
    const int lo = (jr * N) / JC, hi = ((jr + 1) * N) / JC;  // my slice [lo, hi)
    const int nmine = hi - lo;
    const size_t K = (size_t)J * N;
    const bool even = (N % JC) == 0;  // slices of equal length SL = N / JC

    // ---- shared memory ----
    float2 *X = reinterpret_cast<float2 *>(smem_raw);
    // exchange buffer of this team's FFTs: team 0 reuses X (free once gathered)
    float2 *buf = X + (size_t)team * Xf::BUFS * Xf::LBUF;
    float2 *tws = X + (size_t)G * Xf::BUFS * Xf::LBUF;
    const int NCS = Xf::shared_consts(N);
    float2 *Yr = tws + NCS;  // [J][SL]
    float2 *ts = Yr + (size_t)J * SL;
    float2 *gs = ts + SL;
    // mixed precision: the direction p of my slice in FP32 (the pairs are BF16)
    float2 *Ps = gs + (kMixed ? SL : 0);
    HT *Ss = reinterpret_cast<HT *>(gs + (kMixed ? 2 * SL : SL));  // slot a at Ss + a*SL
    HT *Ys = Ss + (size_t)(m + 1) * SL;
    float *red = reinterpret_cast<float *>(Ys + (size_t)(m + 1) * SL);  // [kParts][NW]
    float *part = red + kParts * NW;                                      // [2][JC][kParts]
    Gram &Gm = *reinterpret_cast<Gram *>(
        smem_raw + ((reinterpret_cast<unsigned char *>(part + 2 * JC * kParts) - smem_raw + 15) &
                    ~(size_t)15));

    for (int i = tid; i < NCS; i += BT) tws[i] = P.tw[i];
    Xf xf;
    xf.setup(P.masks + (size_t)jm * N, P.tw + Xf::NCONST, N, ttid);
    auto valid = [&](int e) { return Xf::valid(e, ttid, N); };
    const float gsc = cost_grad_scale(COST);  // the gradient's scale (-4 intensity, 2 amplitude)
    // x[e] = X[index of register e] (zero past the end)
    auto load_X = [&](float2 (&x)[E]) {
#pragma unroll
        for (int e = 0; e < E; e++) x[e] = valid(e) ? X[ttid + e * NT] : make_float2(0.f, 0.f);
    };
    const int sl_shift = (even && (SL & (SL - 1)) == 0) ? __ffs(SL) - 1 : -1;
    auto owner = [&](int n) {
        if (sl_shift >= 0) return n >> sl_shift;
        if (even) return n / SL;
        int o = (int)(((long long)n * JC) / N);
        while (o + 1 < JC && ((o + 1) * N) / JC <= n) o++;
        while (o > 0 && (o * N) / JC > n) o--;
        return o;
    };
    cluster.sync();  // every CTA of the cluster runs before anyone touches its shared memory

    // Cluster-wide sums of nv <= 32 per-thread values (v padded with zeros):
    // each warp reduces its values (recursive halving for many values, plain
    // shuffle sums for a few), the NW warp sums are added in warp order by
    // thread k, which stores the CTA's sum of value k into part[sel][jr][k]
    // of every CTA (its own copy locally, the peers' by DSMEM stores); one
    // cluster barrier; thread k adds the J partials in rank order into
    // Gm.red[k] and the block synchronises.  The two part buffers alternate: a
    // peer may still read the previous one after this barrier but not the one
    // before.
    const int lane = tid & 31, warp = tid >> 5;
    int sel = 0;
    auto cluster_sum = [&](float (&v)[32], int nv) {
        float *pb = part + (size_t)sel * JC * kParts;
        sel ^= 1;
        if (nv <= 6) {
            // constant indices only: a runtime index would move v to local memory
#pragma unroll
            for (int k = 0; k < 6; k++) {
                if (k < nv) {
                    const float t = warp_sum(v[k]);
                    if (lane == 0) red[k * NW + warp] = t;
                }
            }
        } else {
            warp_reduce32(v, lane);
            if (lane < nv) red[lane * NW + warp] = v[0];
        }
        __syncthreads();
        if (tid < nv) {
            float acc = 0.f;
            for (int w = 0; w < NW; w++) acc += red[tid * NW + w];
            for (int o = 0; o < JC; o++) cluster.map_shared_rank(pb, o)[jr * kParts + tid] = acc;
        }
        cluster.sync();
        if (tid < nv) {
            float acc = 0.f;
            for (int o = 0; o < JC; o++) acc += pb[o * kParts + tid];
            Gm.red[tid] = acc;
        }
        __syncthreads();
    };
    // my slice (length nmine) into X of every CTA
    auto push_slice_to_X = [&](const float2 *src) {
        for (int i = tid; i < nmine; i += BT) {
            const float2 v = src[i];
            for (int o = 0; o < JC; o++) cluster.map_shared_rank(X, o)[lo + i] = v;
        }
    };
    // this team's thread-strided natural-order vector v to the owners' Y[jm][:]
    auto push_to_owners = [&](const float2 (&v)[E]) {
#pragma unroll
        for (int e = 0; e < E; e++) {
            if (!valid(e)) continue;
            const int n = ttid + e * NT;
            const int o = owner(n);
            cluster.map_shared_rank(Yr, o)[(size_t)jm * SL + (n - (o * N) / JC)] = v[e];
        }
    };
    // element i of my slice of sum_j Y[j], times s
    auto slice_sum = [&](int i, float s) {
        float2 acc = Yr[i];
        for (int o = 1; o < J; o++) acc = cadd(acc, Yr[(size_t)o * SL + i]);
        return cscale(acc, s);
    };

    while (true) {
        if (jr == 0 && tid == 0) {
            const int r = (int)atomicAdd(P.queue, 1u);
            for (int o = 0; o < JC; o++) cluster.map_shared_rank(&Gm.row, o)[0] = r;
        }
        cluster.sync();
        const int row = Gm.row;
        if (row >= M) break;  // nobody touches another CTA's shared memory after this barrier

        // ---- intensities of mask jm, their sum and finiteness ----
        float yv[E];
        float2 z[E];
        {
            float pv[32] = {0.f};
            if constexpr (kMixed) xf.tc = P.iters > kFinalFp32Iters;
            const float *yr = P.y + (size_t)row * K + (size_t)jm * N;
            // mixed precision: row-normalised FP16 intensities times the row scale
            const __half *yr16 = reinterpret_cast<const __half *>(P.y16) + (size_t)row * K + (size_t)jm * N;
            const float ysc = kMixed ? P.ysc[row] : 1.f;
#pragma unroll
            for (int e = 0; e < E; e++) {
                if constexpr (kMixed) yv[e] = __half2float(yr16[ttid + e * NT]) * ysc;
                else yv[e] = valid(e) ? yr[ttid + e * NT] : 0.f;
                if (isfinite(yv[e])) pv[0] += yv[e];
                else pv[1] += 1.f;
            }
            cluster_sum(pv, 2);
            if (tid == 0) {
                Gm.status = ROW_MAXITER;
                Gm.done = 0;
                Gm.np = 0;
                Gm.f = 0.0;
                Gm.stop = 0;
                Gm.early = 0;
                Gm.sumy = Gm.red[0];
                const int js = row_scale_exp(Gm.red[0], K);
                Gm.yscale = ldexpf(1.f, -2 * js);
                Gm.tsc = ldexpf(1.f, js);
                if (Gm.red[1] > 0.0 || !isfinite(Gm.red[0])) { Gm.status = ROW_NUMERIC; Gm.stop = 1; Gm.early = 1; }
                else if (Gm.red[0] == 0.0) { Gm.status = ROW_ZERO; Gm.stop = 1; Gm.early = 1; }
            }
            __syncthreads();
        }
        // The row is solved with y 4^-j and t 2^-j, scaled back on output,
        // where 4^j is a power of four near its mean intensity (j = 0 for a
        // mean in [1/2, 2)).  Eq. optTMsmall2 is homogeneous, and a scale by
        // a power of two is exact, so every row takes the same steps as the
        // unscaled problem would in exact-range arithmetic; the quartic
        // line-search coefficients, which grow as the fourth power of the
        // intensity scale, stay inside FP32 range for raw camera counts.  (The
        // scales live in shared memory, not in registers through the loop.)
        {
            const float ysc = Gm.yscale;
#pragma unroll
            for (int e = 0; e < E; e++) yv[e] *= ysc;
        }
        const float sumy = Gm.sumy * Gm.yscale;
        const float JN = (float)J * N;

        if (!Gm.stop) {
            // ---- initialisation ----
            if (P.T_init) {
                const float tinv = 1.f / Gm.tsc;  // t = 2^j (normalised t)
                for (int i = tid; i < nmine; i += BT) ts[i] = cscale(P.T_init[(size_t)row * N + lo + i], tinv);
            } else if (P.init == INIT_BP) {
                float2 u[E];
#pragma unroll
                for (int e = 0; e < E; e++) u[e] = make_float2(sqrtf(fmaxf(yv[e], 0.f)), 0.f);
                xf.adj(u, buf, tws, ttid);
                push_to_owners(u);
                cluster.sync();
                for (int i = tid; i < nmine; i += BT) ts[i] = slice_sum(i, 1.f / JN);
            } else {
                // seed: the proposed start (learned initialiser) where it is
                // finite and nonzero, else the Philox vector
                bool seeded = false;
                if (P.T_cand && P.seed_from_cand) {
                    float pv[32] = {0.f};
                    for (int i = tid; i < nmine; i += BT) {
                        const float2 v = P.T_cand[(size_t)row * N + lo + i];
                        ts[i] = v;
                        pv[0] += cabs2(v);
                    }
                    cluster_sum(pv, 1);
                    seeded = isfinite(Gm.red[0]) && Gm.red[0] > 0.f;
                    if (seeded && jr == 0 && tid == 0 && P.cand_wins) atomicAdd(P.cand_wins, 1u);
                }
                if (!seeded)
                    for (int i = tid; i < nmine; i += BT)
                        ts[i] = philox_cnormal(P.seed, (uint32_t)row, (uint32_t)(lo + i));
                if (P.init == INIT_SPECTRAL) {
                    const float mean = sumy / (float)K;
                    float tau[E];
#pragma unroll
                    for (int e = 0; e < E; e++) {
                        float tv = yv[e] / mean;
                        if (P.clip > 0.f && tv > P.clip) tv = P.clip;
                        tau[e] = tv;
                    }
                    if (P.lanczos) {
                        auto applyA = [&]() {
                            __syncthreads();
                            push_slice_to_X(ts);
                            cluster.sync();
                            float2 x[E];
                            load_X(x);
                            __syncthreads();  // X is read before the FFT reuses it
                            xf.fwd(x, buf, tws, ttid);
#pragma unroll
                            for (int e = 0; e < E; e++) x[e] = cscale(x[e], tau[e]);
                            xf.adj(x, buf, tws, ttid);
                            push_to_owners(x);
                            cluster.sync();
                            for (int i = tid; i < nmine; i += BT) gs[i] = slice_sum(i, 1.f / JN);
                            __syncthreads();
                        };
                        float2 *reg = P.krylov + (size_t)(blockIdx.x / JC) * lanczos_region(N, P.power_iters);
                        float2 *Gw = reg + (size_t)P.power_iters * N + (size_t)jr * kMaxLanczos * kMaxLanczos;
                        lanczos_start(P.power_iters, nmine, ts, gs, reg + lo, (size_t)N, Gw, Gm.red, &Gm.SY[0][0],
                                      &Gm.YY[0][0], applyA, cluster_sum);
                    }
                    for (int it = 0; it < (P.lanczos ? 0 : P.power_iters); it++) {
                        // t <- A t, A = Q^H diag(tau) Q / (J N); the norm is restored
                        // every 8th step and at the end (only the direction matters
                        // to the power iteration, and |A| <= clip bounds the growth)
                        __syncthreads();
                        push_slice_to_X(ts);
                        cluster.sync();
                        float2 x[E];
                        load_X(x);
                        __syncthreads();  // X is read before the FFT reuses it
                        xf.fwd(x, buf, tws, ttid);
#pragma unroll
                        for (int e = 0; e < E; e++) x[e] = cscale(x[e], tau[e]);
                        xf.adj(x, buf, tws, ttid);
                        push_to_owners(x);
                        cluster.sync();
                        const bool renorm = ((it & 7) == 7) || (it == P.power_iters - 1);
                        float pv[32] = {0.f};
                        for (int i = tid; i < nmine; i += BT) {
                            const float2 s = slice_sum(i, 1.f / JN);
                            ts[i] = s;
                            pv[0] = fmaf(s.x, s.x, fmaf(s.y, s.y, pv[0]));
                        }
                        if (renorm) {
                            cluster_sum(pv, 1);
                            const float nrm = Gm.red[0];
                            const float inv = nrm > 0.f ? rsqrtf(nrm) : 0.f;
                            for (int i = tid; i < nmine; i += BT) ts[i] = cscale(ts[i], inv);
                        }
                    }
                }
                // rescale to the Parseval norm ||t||^2 = sum(y) / (J N)
                float pv[32] = {0.f};
                for (int i = tid; i < nmine; i += BT) pv[0] += cabs2(ts[i]);
                cluster_sum(pv, 1);
                const float nrm = Gm.red[0];
                const float sc = nrm > 0.f ? sqrtf(sumy / JN) / sqrtf(nrm) : 0.f;
                for (int i = tid; i < nmine; i += BT) ts[i] = cscale(ts[i], sc);
            }

            // ---- per-row selection: a proposed start (learned initialiser) against this one ----
            if (P.T_cand && P.judge_cand) {
                const float tinv = 1.f / Gm.tsc;
                for (int i = tid; i < nmine; i += BT) gs[i] = cscale(P.T_cand[(size_t)row * N + lo + i], tinv);
                float fv[2];
                for (int c = 0; c < 2; c++) {  // f at the start above, then at the proposal
                    __syncthreads();
                    push_slice_to_X(c == 0 ? ts : gs);
                    cluster.sync();
                    float2 x[E];
                    load_X(x);
                    __syncthreads();  // X is read before the FFT reuses it
                    xf.fwd(x, buf, tws, ttid);
                    float pv[32] = {0.f};
#pragma unroll
                    for (int e = 0; e < E; e++) {
                        if constexpr (COST == COST_AMPLITUDE) {
                            if (valid(e)) cost_coef(COST, x[e], yv[e], pv[0]);
                        } else {
                            const float r = yv[e] - cabs2(x[e]);
                            pv[0] = fmaf(r, r, pv[0]);
                        }
                    }
                    cluster_sum(pv, 1);
                    fv[c] = Gm.red[0];
                }
                if (fv[1] < fv[0]) {  // NaN proposals lose
                    for (int i = tid; i < nmine; i += BT) ts[i] = gs[i];
                    if (jr == 0 && tid == 0 && P.cand_wins) atomicAdd(P.cand_wins, 1u);
                }
            }

            // ---- f and gradient at t (the start; in a mixed-precision run also the
            // switch to the FP32 transforms, which restarts the history) ----
            auto eval_at_t = [&]() {
                __syncthreads();
                push_slice_to_X(ts);
                cluster.sync();
                load_X(z);
                __syncthreads();  // X is read before the FFT reuses it
                xf.fwd(z, buf, tws, ttid);
                float2 u[E];
                float pv[32] = {0.f};
#pragma unroll
                for (int e = 0; e < E; e++) {
                    if constexpr (COST == COST_AMPLITUDE) {
                        u[e] = valid(e) ? cscale(z[e], cost_coef(COST, z[e], yv[e], pv[0])) : make_float2(0.f, 0.f);
                    } else {
                        const float r = yv[e] - cabs2(z[e]);
                        pv[0] = fmaf(r, r, pv[0]);
                        u[e] = cscale(z[e], r);
                    }
                }
                xf.adj(u, buf, tws, ttid);
                push_to_owners(u);
                cluster.sync();
                for (int i = tid; i < nmine; i += BT) {
                    const float2 g = slice_sum(i, gsc);
                    gs[i] = g;
                    pv[1] += cabs2(g);
                }
                cluster_sum(pv, 2);
                if (warp == 0) {
                    if (lane == 0) {
                        Gm.f = Gm.red[0];
                        Gm.gg = Gm.red[1];
                        Gm.np = 0;
                        if (!isfinite(Gm.f) || !isfinite(Gm.gg)) { Gm.status = ROW_NUMERIC; Gm.stop = 1; }
                        else if (P.iters > 0 && (Gm.f == 0.f || Gm.gg == 0.f)) { Gm.status = ROW_CONVERGED; Gm.stop = 1; }
                    }
                    if (lane < kSlots) Gm.slot[lane] = lane;
                    __syncwarp();
                    if (!Gm.stop) lbfgs_coefficients_warp(Gm, lane);
                }
                __syncthreads();
            };
            eval_at_t();

            // ---- L-BFGS iterations ----
            for (int it = 0; it < P.iters && !Gm.stop; it++) {
                if constexpr (kMixed) {
                    if (xf.tc && it == P.iters - kFinalFp32Iters) {
                        xf.tc = false;  // the last iterations in FP32
                        eval_at_t();
                        if (Gm.stop) break;
                    }
                }
                const int ns = Gm.slot[Gm.np];  // free slot for the new pair
                HT *Sn = Ss + (size_t)ns * SL;
                HT *Yn = Ys + (size_t)ns * SL;
                // A: direction on my slice, parked in the new S slot until the step is known
                {
                    const float gam = Gm.gamma;
                    const int np = Gm.np;
                    float c1r[kSlots], c2r[kSlots];
                    int so[kSlots];  // slot offsets (same for the S and Y halves)
#pragma unroll
                    for (int k = 0; k < kSlots; k++) {
                        const int a = Gm.slot[k < np ? k : 0];
                        c1r[k] = k < np ? Gm.c1[k] : 0.f;
                        c2r[k] = k < np ? Gm.c2[k] : 0.f;
                        so[k] = a * SL;
                    }
                    for (int i = tid; i < nmine; i += BT) {
                        float2 acc = cscale(gs[i], gam);
#pragma unroll
                        for (int k = 0; k < kSlots; k++) {
                            if (k < np) {
                                const float2 sa = hist_load(Ss[so[k] + i]), ya = hist_load(Ys[so[k] + i]);
                                acc.x = fmaf(c1r[k], sa.x, fmaf(c2r[k], ya.x, acc.x));
                                acc.y = fmaf(c1r[k], sa.y, fmaf(c2r[k], ya.y, acc.y));
                            }
                        }
                        const float2 p = make_float2(-acc.x, -acc.y);
                        if constexpr (kMixed) Ps[i] = p;
                        else Sn[i] = p;
                        for (int o = 0; o < JC; o++) cluster.map_shared_rank(X, o)[lo + i] = p;
                    }
                }
                cluster.sync();  // B1
                // C: w = F(d .* p)
                float2 w[E];
                load_X(w);
                __syncthreads();  // X is read before the FFT reuses it
                xf.fwd(w, buf, tws, ttid);
                // D: the step -- the amplitude cost's line search, or the quartic's exact minimiser
                if constexpr (COST == COST_AMPLITUDE) {
                    const float al = amp_line_search(
                        z, w, [&](int e) { return yv[e]; }, valid, cluster_sum, Gm.red, Gm.red + 16);
                    if (tid == 0) {
                        Gm.alpha = al;
                        if (!isfinite(al)) { Gm.status = ROW_NUMERIC; Gm.stop = 1; }
                        else if (al == 0.f) { Gm.status = ROW_CONVERGED; Gm.stop = 1; }
                    }
                    __syncthreads();
                } else {
                    float pv[32] = {0.f};
#pragma unroll
                    for (int e = 0; e < E; e++) {
                        const float a = cdotr(z[e], w[e]);
                        const float b = cabs2(w[e]);
                        const float r = yv[e] - cabs2(z[e]);
                        pv[0] = fmaf(r, r, pv[0]);
                        pv[1] = fmaf(-4.f * r, a, pv[1]);
                        pv[2] += fmaf(4.f * a, a, -2.f * r * b);
                        pv[3] = fmaf(4.f * a, b, pv[3]);
                        pv[4] = fmaf(b, b, pv[4]);
                    }
                    cluster_sum(pv, 5);  // B2
                    if (warp == 0) {
                        const float al = quartic_argmin_warp(Gm.red, lane);
                        if (lane == 0) {
                            Gm.alpha = al;
                            if (!isfinite(al)) { Gm.status = ROW_NUMERIC; Gm.stop = 1; }
                            else if (al == 0.f) { Gm.status = ROW_CONVERGED; Gm.stop = 1; }
                        }
                    }
                    __syncthreads();
                }
                if (Gm.stop) break;
                const float al = Gm.alpha;
                // E: update fields, residual and the step
                float2 u[E];
                float fpart = 0.f;
#pragma unroll
                for (int e = 0; e < E; e++) {
                    z[e] = make_float2(fmaf(al, w[e].x, z[e].x), fmaf(al, w[e].y, z[e].y));
                    if constexpr (COST == COST_AMPLITUDE) {
                        u[e] = valid(e) ? cscale(z[e], cost_coef(COST, z[e], yv[e], fpart)) : make_float2(0.f, 0.f);
                    } else {
                        const float r = yv[e] - cabs2(z[e]);
                        fpart = fmaf(r, r, fpart);
                        u[e] = cscale(z[e], r);
                    }
                }
                for (int i = tid; i < nmine; i += BT) {
                    float2 s;
                    if constexpr (kMixed) {
                        s = cscale(Ps[i], al);
                        Sn[i] = hist_store<HT>(s);
                    } else {
                        s = cscale(Sn[i], al);
                        Sn[i] = s;
                    }
                    ts[i] = cadd(ts[i], s);
                }
                // F: adjoint, pushed to the slice owners
                xf.adj(u, buf, tws, ttid);
                push_to_owners(u);
                cluster.sync();  // B3
                // G: new gradient, new pair, batched dot products
                {
                    const int np = Gm.np;
                    float pv[32];
#pragma unroll
                    for (int k = 0; k < 32; k++) pv[k] = 0.f;
                    int so[kSlots];  // slot offsets (same for the S and Y halves)
#pragma unroll
                    for (int k = 0; k < kSlots; k++) so[k] = Gm.slot[k <= np ? k : 0] * SL;
                    for (int i = tid; i < nmine; i += BT) {
                        const float2 gn = slice_sum(i, gsc);
                        const HT yh = hist_store<HT>(csub(gn, gs[i]));
                        const float2 yn = hist_load(yh);  // the stored pair, as the Gram scalars see it
                        gs[i] = gn;
                        Yn[i] = yh;
                        const float2 sn = hist_load(Sn[i]);
#pragma unroll
                        for (int k = 0; k < kSlots; k++) {
                            if (k <= np) {  // live pairs by age, then the new one (age np)
                                const float2 sa = hist_load(Ss[so[k] + i]);
                                const float2 ya = hist_load(Ys[so[k] + i]);
                                pv[4 * k + 0] += cdotr(sa, yn);
                                pv[4 * k + 1] += cdotr(ya, yn);
                                pv[4 * k + 2] += cdotr(sa, gn);
                                pv[4 * k + 3] += cdotr(ya, gn);
                            }
                        }
                        pv[kIdxSS] += cabs2(sn);
                        pv[kIdxGG] += cabs2(gn);
                    }
                    pv[kIdxF] = fpart;
                    cluster_sum(pv, kParts);  // B4
                    if (warp == 0) lbfgs_gram_update(Gm, lane, m, it, P.iters, P.tol);
                    __syncthreads();
                }
            }
        }

        // ---- outputs (rows decided before initialisation come back as zero) ----
        const bool early = Gm.early != 0;
        const float tsc = Gm.tsc;
        for (int i = tid; i < nmine; i += BT)
            P.T_out[(size_t)row * N + lo + i] = early ? make_float2(0.f, 0.f) : cscale(ts[i], tsc);
        if (jr == 0 && tid == 0) {
            if (P.row_status) P.row_status[row] = Gm.status;
            if (P.row_iters) P.row_iters[row] = Gm.done;
            if (P.row_loss) {
                // the intensity cost scales as y^2 = t^4, the amplitude cost as y = t^2
                const double f2 = COST == COST_AMPLITUDE ? (double)tsc * tsc : (double)tsc * tsc * tsc * tsc;
                P.row_loss[row] = early ? (Gm.status == ROW_ZERO ? 0.f : __int_as_float(0x7fc00000))
                                        : (float)((double)Gm.f * f2);
            }
        }
        if (P.Zd) {
#pragma unroll
            for (int e = 0; e < E; e++) {
                const int pat = jm * N + ttid + e * NT;
                if (valid(e) && pat < P.Nd) P.Zd[(size_t)pat * M + row] = early ? make_float2(0.f, 0.f) : cscale(z[e], tsc);
            }
        }
        __syncthreads();
    }
}

template <class Xf, int G, int COST = COST_INTENSITY>
cudaError_t launch_solver_t(const SolverParams &p, cudaStream_t s, int *clusters_out)
{
    using C = SolverCfg<Xf, G>;
    const int JC = p.J / G;
    const size_t sm = solver_smem<Xf, G>(p.N, p.J, p.m);
    cudaError_t e = cudaFuncSetAttribute(k_solver<Xf, G, COST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = JC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(C::BT);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(JC);
    int maxc = 0;
    e = cudaOccupancyMaxActiveClusters(&maxc, k_solver<Xf, G, COST>, &cfg);
    if (e != cudaSuccess) return e;
    if (maxc < 1) return cudaErrorInvalidConfiguration;
    int nc = maxc < p.M ? maxc : p.M;
    if (p.lanczos && p.init == INIT_SPECTRAL && nc > p.krylov_units) nc = p.krylov_units;  // one region each
    if (nc < 1) nc = 1;
    cfg.gridDim = dim3(nc * JC);
    if (clusters_out) *clusters_out = nc;
    return cudaLaunchKernelEx(&cfg, k_solver<Xf, G, COST>, p);
}

}  // namespace tmr
