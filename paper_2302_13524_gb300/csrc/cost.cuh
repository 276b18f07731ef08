// cost.cuh -- the two costs of the per-row problem and the amplitude cost's
// line search, shared by the gradient kernel and the per-row solvers.
//
// Intensity (Eq. optTMsmall2, the paper's): f = sum (y - |z|^2)^2, real
// gradient -4 Q^H (z r), r = y - |z|^2 (Eq. derivative).  Amplitude (the
// Discussion's alternative for Poisson noise): f = sum (a - |z|)^2 with
// a = sqrt(y), real gradient 2 Q^H ((|z| - a) z / |z|), the term 0 where z = 0.
// Both are written as u = c z and g = s Q^H u with a per-element coefficient c
// and a scale s.
#pragma once

#include "common.cuh"

namespace tmr {

enum { COST_INTENSITY = 0, COST_AMPLITUDE = 1 };

// The coefficient c of element (z, y) and its loss term added to f.
__device__ __forceinline__ float cost_coef(int cost, float2 z, float y, float &f)
{
    if (cost == COST_AMPLITUDE) {
        const float a = sqrtf(fmaxf(y, 0.f)), m = sqrtf(cabs2(z));
        const float d = a - m;
        f = fmaf(d, d, f);
        return m > 0.f ? (m - a) / m : 0.f;
    }
    const float r = y - cabs2(z);
    f = fmaf(r, r, f);
    return r;
}

__host__ __device__ __forceinline__ float cost_grad_scale(int cost) { return cost == COST_AMPLITUDE ? 2.f : -4.f; }

// Half the first and second derivatives of phi(al) = sum (a - |z + al w|)^2
// for one element, added to d1 and d2 (a term with |u| = 0 adds |w|^2 to d2
// only, as in the gradient).
__device__ __forceinline__ void amp_derivs(float2 z, float2 w, float y, float al, float &d1, float &d2)
{
    const float a = sqrtf(fmaxf(y, 0.f));
    const float2 u = make_float2(fmaf(al, w.x, z.x), fmaf(al, w.y, z.y));
    const float m2 = cabs2(u), m = sqrtf(m2);
    const float cr = u.x * w.x + u.y * w.y, ci = u.x * w.y - u.y * w.x;  // conj(u) w
    d2 += cabs2(w);
    if (m > 0.f) {
        d1 = fmaf((m - a) / m, cr, d1);
        d2 -= a * ci * ci / (m2 * m);
    }
}

// The amplitude cost's step along t + al p (fields z + al w), the rule of the
// oracle's line search: bracket the first sign change of phi' at al = 1, 2,
// 4, ... (at most 40 doublings; lower end 0 at first, p being a descent
// direction; if phi' stays negative, the farthest point tried), then Newton
// steps from the lower end kept inside the bracket (the midpoint where a step
// would leave it or phi'' <= 0), the bracket shrunk by the sign of phi' at
// every point, until a step is below 1e-6 al or after 30 steps.  One pass over
// the row's fields and one row reduction per point; thread 0 takes the
// decisions, which every CTA of a cluster takes alike from the same sums.
//   yat(e), valid(e)  the intensity and the validity of this thread's element e
//   reduce(v, n)      row sums of v[0..n) into red[0..n), then synchronises
//   st                4 floats of shared scratch
// All threads call; the step is returned to all.
template <int E, class YAt, class Valid, class Reduce>
__device__ float amp_line_search(const float2 (&z)[E], const float2 (&w)[E], YAt &&yat, Valid &&valid,
                                 Reduce &&reduce, const float *red, float *st)
{
    // st[0] next point, st[1] done, st[2] result
    float pv[32];
#pragma unroll
    for (int q = 0; q < 32; q++) pv[q] = 0.f;
#pragma unroll
    for (int e = 0; e < E; e++)
        if (valid(e)) {
            amp_derivs(z[e], w[e], yat(e), 0.f, pv[0], pv[1]);
            amp_derivs(z[e], w[e], yat(e), 1.f, pv[2], pv[3]);
        }
    reduce(pv, 4);
    // thread 0's state, kept in registers of thread 0 only
    float lo = 0.f, hi = 0.f, x = 1.f, d1lo = red[0], d2lo = red[1], d1 = red[2], d2 = red[3];
    int k = 0, it = 0;
    bool newton = false;
    for (int pass = 0; pass < 72; pass++) {
        if (threadIdx.x == 0) {
            bool done = false;
            float next = x, result = x;
            if (!newton) {
                if (!(d1 < 0.f)) {
                    hi = x;
                    float x0 = d2lo > 0.f ? lo - d1lo / d2lo : __int_as_float(0x7fc00000);
                    if (!(x0 > lo && x0 < hi)) x0 = 0.5f * (lo + hi);
                    newton = true;
                    next = x0;
                } else {
                    lo = x;
                    d1lo = d1;
                    d2lo = d2;
                    if (k == 40) {
                        done = true;
                        result = lo;
                    } else {
                        k++;
                        next = 2.f * x;
                    }
                }
            } else {
                if (d1 == 0.f) {
                    done = true;
                    result = x;
                } else {
                    if (d1 < 0.f) lo = x;
                    else hi = x;
                    float xn = d2 > 0.f ? x - d1 / d2 : __int_as_float(0x7fc00000);
                    if (!(xn > lo && xn < hi)) xn = 0.5f * (lo + hi);
                    if (fabsf(xn - x) <= 1e-6f * x || ++it >= 30) {
                        done = true;
                        result = xn;
                    }
                    next = xn;
                }
            }
            x = next;
            st[0] = next;
            st[1] = done ? 1.f : 0.f;
            st[2] = result;
        }
        __syncthreads();
        if (st[1] != 0.f) break;
        const float al = st[0];
#pragma unroll
        for (int q = 0; q < 2; q++) pv[q] = 0.f;
#pragma unroll
        for (int e = 0; e < E; e++)
            if (valid(e)) amp_derivs(z[e], w[e], yat(e), al, pv[0], pv[1]);
        reduce(pv, 2);
        d1 = red[0];
        d2 = red[1];
    }
    const float res = st[2];
    __syncthreads();  // st is read before the next use rewrites it
    return res;
}

}  // namespace tmr
