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
// transforms their grids in shared memory (in-place radix-2 2D FFTs, FP32);
// loss and gradient partials are written per CTA and reduced in a fixed order
// (deterministic); the L-BFGS state, the Armijo test and every reduction of the
// fit are FP64.  CTAs meet at a grid barrier whose spin is bounded: on timeout
// the kernel raises an error flag and every CTA returns.
#include <cmath>

#include "common.cuh"
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
__device__ __forceinline__ unsigned bitrev(unsigned v, int bits) { return __brev(v) >> (32 - bits); }

// tw[k] = exp(-2 pi i k / n), k < n/2 (twy for ny, twx for nx), made once per CTA.
__device__ void make_tw(float2 *tw, int n)
{
    for (int k = threadIdx.x; k < n / 2; k += blockDim.x) {
        double s, c;
        sincospi(-2.0 * k / n, &s, &c);
        tw[k] = make_float2((float)c, (float)s);
    }
}

__device__ void fft2_inplace(float2 *g, int ny, int nx, int sign, const float2 *twy, const float2 *twx)
{
    const int pitch = nx + 1;
    const int lx = __ffs(nx) - 1, ly = __ffs(ny) - 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    // rows: bit reversal
    for (int i = tid; i < ny * nx; i += nt) {
        const int a = i / nx, b = i % nx;
        const int rb = (int)bitrev((unsigned)b, lx);
        if (rb > b) {
            const float2 t = g[a * pitch + b];
            g[a * pitch + b] = g[a * pitch + rb];
            g[a * pitch + rb] = t;
        }
    }
    __syncthreads();
    for (int half = 1; half < nx; half <<= 1) {
        const int step = nx / (2 * half);
        for (int i = tid; i < ny * (nx / 2); i += nt) {
            const int a = i / (nx / 2), q = i % (nx / 2);
            const int grp = q / half, k = q % half;
            const int b0 = grp * 2 * half + k, b1 = b0 + half;
            float2 w = twx[k * step];
            if (sign > 0) w.y = -w.y;
            const float2 x0 = g[a * pitch + b0], x1 = cmul(g[a * pitch + b1], w);
            g[a * pitch + b0] = cadd(x0, x1);
            g[a * pitch + b1] = csub(x0, x1);
        }
        __syncthreads();
    }
    // columns
    for (int i = tid; i < ny * nx; i += nt) {
        const int a = i / nx, b = i % nx;
        const int ra = (int)bitrev((unsigned)a, ly);
        if (ra > a) {
            const float2 t = g[a * pitch + b];
            g[a * pitch + b] = g[ra * pitch + b];
            g[ra * pitch + b] = t;
        }
    }
    __syncthreads();
    for (int half = 1; half < ny; half <<= 1) {
        const int step = ny / (2 * half);
        for (int i = tid; i < (ny / 2) * nx; i += nt) {
            const int q = i / nx, b = i % nx;
            const int grp = q / half, k = q % half;
            const int a0 = grp * 2 * half + k, a1 = a0 + half;
            float2 w = twy[k * step];
            if (sign > 0) w.y = -w.y;
            const float2 x0 = g[a0 * pitch + b], x1 = cmul(g[a1 * pitch + b], w);
            g[a0 * pitch + b] = cadd(x0, x1);
            g[a1 * pitch + b] = csub(x0, x1);
        }
        __syncthreads();
    }
}

// g <- D g (adjoint: D^H g), including the 1/P of the inverse transform.
__device__ void defocus_apply_smem(float2 *g, int ny, int nx, const float2 *__restrict__ H,
                                   bool adjoint, const float2 *twy, const float2 *twx)
{
    const int pitch = nx + 1, P = ny * nx;
    fft2_inplace(g, ny, nx, -1, twy, twx);
    const float inv = 1.0f / (float)P;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int a = i / nx, b = i % nx;
        float2 h = H[i];
        if (adjoint) h.y = -h.y;
        g[a * pitch + b] = cscale(cmul(g[a * pitch + b], h), inv);
    }
    __syncthreads();
    fft2_inplace(g, ny, nx, +1, twy, twx);
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
// Phase-offset fit.

// bounded grid barrier; bar[0] arrival count, bar[1] generation
__device__ bool grid_sync(unsigned *bar, int *err)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = bar + 1;
        volatile int *verr = err;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u) + 1u;
        if (arrived == gridDim.x) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long spins = 0;
            while (*vgen == gen) {
                if (*verr) break;
                if (++spins > (1LL << 24)) {  // ~1 s at 64 ns a poll, then give up
                    atomicExch(err, 1);
                    break;
                }
                __nanosleep(64);
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

// workspace layout (doubles): phi, p, g, gn, phit, (S, Y)[m], part[grid][P], fpart[grid],
// scal[64], then u[grid][P] as float2 (one e^{i phi} table per CTA)
size_t phase_fit_workspace_doubles(int P, int Nd, int m, int grid)
{
    (void)Nd;
    return (size_t)P * (5 + 2 * m) + 2 * (size_t)grid * P + grid + 64;
}

struct PFWork {
    double *phi, *p, *g, *gn, *phit, *S, *Y, *part, *fpart, *scal;
    float2 *u;
};

__device__ PFWork pf_carve(double *ws, int P, int m, int grid)
{
    PFWork w;
    w.phi = ws;
    w.p = w.phi + P;
    w.g = w.p + P;
    w.gn = w.g + P;
    w.phit = w.gn + P;
    w.S = w.phit + P;
    w.Y = w.S + (size_t)m * P;
    w.part = w.Y + (size_t)m * P;
    w.fpart = w.part + (size_t)grid * P;
    w.scal = w.fpart + grid;
    w.u = reinterpret_cast<float2 *>(w.scal + 64);
    return w;
}

// scal slots
enum { SC_F = 0, SC_GP, SC_A, SC_NP, SC_FT, SC_ACCEPT, SC_STOP, SC_ITERS, SC_HEAD };

template <int NV>
__device__ __forceinline__ void block_sum_d(double (&v)[NV], double *red, double *out)
{
    block_sum<NV, double>(v, red, out);
}

// Loss and gradient partials of this CTA's patterns at phase phi_src into
// part[blockIdx.x][:] and fpart[blockIdx.x].
__device__ void pf_eval(const PhaseFitParams &Pp, const PFWork &W, const double *phi_src, float2 *g,
                        const float2 *twy, const float2 *twx, double *red, double *out)
{
    const int ny = Pp.ny, nx = Pp.nx, P = ny * nx, pitch = nx + 1;
    double *part = W.part + (size_t)blockIdx.x * P;
    float2 *uu = W.u + (size_t)blockIdx.x * P;
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        part[k] = 0.0;
        float s, c;
        sincosf((float)remainder(__ldcg(phi_src + k), 2.0 * M_PI), &s, &c);
        uu[k] = make_float2(c, s);
    }
    __syncthreads();
    double fl = 0.0;
    for (int n = blockIdx.x; n < Pp.Nd; n += gridDim.x) {
        const float2 *cn = Pp.Zd + (size_t)n * P;
        const float *In = Pp.Ydef + (size_t)n * P;
        for (int k = threadIdx.x; k < P; k += blockDim.x) g[(k / nx) * pitch + k % nx] = cmul(cn[k], uu[k]);
        __syncthreads();
        defocus_apply_smem(g, ny, nx, Pp.H, false, twy, twx);
        float fpl = 0.f;
        for (int k = threadIdx.x; k < P; k += blockDim.x) {
            const int gi = (k / nx) * pitch + k % nx;
            const float2 w = g[gi];
            const float G = In[k] - cabs2(w);
            fpl = fmaf(G, G, fpl);
            g[gi] = cscale(w, G);
        }
        fl += (double)fpl;
        __syncthreads();
        defocus_apply_smem(g, ny, nx, Pp.H, true, twy, twx);
        for (int k = threadIdx.x; k < P; k += blockDim.x) {
            const float2 v = cmulc(g[(k / nx) * pitch + k % nx], cn[k]);  // conj(c_n) D^H(w G)
            // -4 Im(conj(u) v)
            const float2 cu = uu[k];
            const float im = fmaf(cu.x, v.y, -cu.y * v.x);
            part[k] += -4.0 * (double)im;
        }
        __syncthreads();
    }
    double fv[1] = {fl};
    block_sum_d<1>(fv, red, out);
    if (threadIdx.x == 0) W.fpart[blockIdx.x] = out[0];
}

__global__ void __launch_bounds__(512) k_phase_fit(PhaseFitParams Pp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ny = Pp.ny, nx = Pp.nx, P = ny * nx, m = Pp.m, nb = gridDim.x;
    float2 *g = reinterpret_cast<float2 *>(smem_raw);
    float2 *twy = g + (size_t)ny * (nx + 1), *twx = twy + ny / 2;
    double *red = reinterpret_cast<double *>(twx + nx / 2 + 1);
    double *out = red + 32 * 4;
    PFWork W = pf_carve(Pp.ws, P, m, nb);
    make_tw(twy, ny);
    make_tw(twx, nx);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int chunk = (P + nb - 1) / nb, k0 = blockIdx.x * chunk, k1 = min(P, k0 + chunk);

    for (int k = k0 + tid; k < k1; k += nt) W.phi[k] = 0.0;
    if (!grid_sync(Pp.sync, Pp.err)) return;
    pf_eval(Pp, W, W.phi, g, twy, twx, red, out);
    if (!grid_sync(Pp.sync, Pp.err)) return;
    for (int k = k0 + tid; k < k1; k += nt) {
        double s = 0.0;
        for (int b = 0; b < nb; b++) s += __ldcg(W.part + (size_t)b * P + k);
        W.g[k] = s;
    }
    if (blockIdx.x == 0 && tid == 0) {
        double f = 0.0;
        for (int b = 0; b < nb; b++) f += __ldcg(W.fpart + b);
        W.scal[SC_F] = f;
        W.scal[SC_NP] = 0;
        W.scal[SC_HEAD] = 0;
        W.scal[SC_ITERS] = 0;
        W.scal[SC_STOP] = 0;
    }
    if (!grid_sync(Pp.sync, Pp.err)) return;

    for (int it = 0; it < Pp.iters; it++) {
        // ---- direction (CTA 0, FP64 two-loop over the ring of pairs) ----
        if (blockIdx.x == 0) {
            const int np = (int)__ldcg(W.scal + SC_NP), head = (int)__ldcg(W.scal + SC_HEAD);  // head: slot of the oldest pair
            __shared__ double alph[kMaxMem];
            for (int k = tid; k < P; k += nt) W.p[k] = __ldcg(W.g + k);
            __syncthreads();
            for (int q = np - 1; q >= 0; q--) {
                const int sl = (head + q) % m;
                const double *s = W.S + (size_t)sl * P, *y = W.Y + (size_t)sl * P;
                double v[2] = {0.0, 0.0};
                for (int k = tid; k < P; k += nt) {
                    v[0] += s[k] * y[k];
                    v[1] += s[k] * W.p[k];
                }
                block_sum_d<2>(v, red, out);
                const double a = out[1] / out[0];
                if (tid == 0) alph[q] = a;
                for (int k = tid; k < P; k += nt) W.p[k] -= a * y[k];
                __syncthreads();
            }
            if (np > 0) {
                const int sl = (head + np - 1) % m;
                const double *s = W.S + (size_t)sl * P, *y = W.Y + (size_t)sl * P;
                double v[2] = {0.0, 0.0};
                for (int k = tid; k < P; k += nt) {
                    v[0] += s[k] * y[k];
                    v[1] += y[k] * y[k];
                }
                block_sum_d<2>(v, red, out);
                const double gam = out[0] / out[1];
                for (int k = tid; k < P; k += nt) W.p[k] *= gam;
                __syncthreads();
            }
            for (int q = 0; q < np; q++) {
                const int sl = (head + q) % m;
                const double *s = W.S + (size_t)sl * P, *y = W.Y + (size_t)sl * P;
                double v[2] = {0.0, 0.0};
                for (int k = tid; k < P; k += nt) {
                    v[0] += s[k] * y[k];
                    v[1] += y[k] * W.p[k];
                }
                block_sum_d<2>(v, red, out);
                const double b = out[1] / out[0];
                const double a = alph[q];
                for (int k = tid; k < P; k += nt) W.p[k] += s[k] * (a - b);
                __syncthreads();
            }
            double v[2] = {0.0, 0.0};
            for (int k = tid; k < P; k += nt) {
                W.p[k] = -W.p[k];
                v[0] += W.g[k] * W.p[k];
                v[1] = fmax(v[1], fabs(W.g[k]));
            }
            // max via a separate pass: reuse block_sum on the sum, max below
            __shared__ double gmaxs[32];
            double mx = v[1];
            for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if ((tid & 31) == 0) gmaxs[tid >> 5] = mx;
            double sv[1] = {v[0]};
            block_sum_d<1>(sv, red, out);
            double gmax = 0.0;
            for (int w = 0; w < nt / 32; w++) gmax = fmax(gmax, gmaxs[w]);
            double gp = out[0];
            __syncthreads();
            if (gmax == 0.0) {
                if (tid == 0) W.scal[SC_STOP] = 1;
            } else if (np == 0 || !(gp < 0.0)) {
                for (int k = tid; k < P; k += nt) W.p[k] = -W.g[k] / gmax;
                double s2[1] = {0.0};
                for (int k = tid; k < P; k += nt) s2[0] += W.g[k] * W.p[k];
                block_sum_d<1>(s2, red, out);
                gp = out[0];
                if (tid == 0) W.scal[SC_NP] = 0;
            }
            if (tid == 0) {
                W.scal[SC_GP] = gp;
                W.scal[SC_A] = 1.0;
            }
        }
        if (!grid_sync(Pp.sync, Pp.err)) return;
        if (__ldcg(W.scal + SC_STOP) != 0.0) break;

        // ---- Armijo backtracking ----
        bool accepted = false;
        for (int h = 0; h <= 30; h++) {
            const double a = __ldcg(W.scal + SC_A);
            // every CTA evaluates at phit = phi + a p; CTA b writes its chunk of phit
            for (int k = k0 + tid; k < k1; k += nt) W.phit[k] = __ldcg(W.phi + k) + a * __ldcg(W.p + k);
            if (!grid_sync(Pp.sync, Pp.err)) return;
            pf_eval(Pp, W, W.phit, g, twy, twx, red, out);
            if (!grid_sync(Pp.sync, Pp.err)) return;
            double ft = 0.0;
            for (int b = 0; b < nb; b++) ft += __ldcg(W.fpart + b);
            const double f = __ldcg(W.scal + SC_F), gp = __ldcg(W.scal + SC_GP);
            if (ft <= f + 1e-4 * a * gp) {
                accepted = true;
                for (int k = k0 + tid; k < k1; k += nt) {
                    double s = 0.0;
                    for (int b = 0; b < nb; b++) s += __ldcg(W.part + (size_t)b * P + k);
                    W.gn[k] = s;
                }
                if (blockIdx.x == 0 && tid == 0) W.scal[SC_FT] = ft;
                break;
            }
            // all CTAs agree on the decision; CTA 0 halves the step after everyone read it
            if (!grid_sync(Pp.sync, Pp.err)) return;
            if (blockIdx.x == 0 && tid == 0) W.scal[SC_A] = 0.5 * a;
            if (!grid_sync(Pp.sync, Pp.err)) return;
        }
        if (!accepted) break;
        if (!grid_sync(Pp.sync, Pp.err)) return;

        // ---- new pair, accept step (CTA 0) ----
        if (blockIdx.x == 0) {
            const int np = (int)__ldcg(W.scal + SC_NP), head = (int)__ldcg(W.scal + SC_HEAD);
            const int sl = (head + np) % m;  // next slot (overwrites the oldest when full)
            double *s = W.S + (size_t)sl * P, *y = W.Y + (size_t)sl * P;
            double v[3] = {0.0, 0.0, 0.0};
            for (int k = tid; k < P; k += nt) {
                const double sv = __ldcg(W.phit + k) - W.phi[k], yv = __ldcg(W.gn + k) - __ldcg(W.g + k);
                v[0] += sv * yv;
                v[1] += sv * sv;
                v[2] += yv * yv;
            }
            block_sum_d<3>(v, red, out);
            const bool ok = out[0] > 1e-10 * sqrt(out[1]) * sqrt(out[2]) && out[0] > 0.0;
            if (ok) {
                for (int k = tid; k < P; k += nt) {
                    s[k] = __ldcg(W.phit + k) - W.phi[k];
                    y[k] = __ldcg(W.gn + k) - __ldcg(W.g + k);
                }
            }
            __syncthreads();
            for (int k = tid; k < P; k += nt) {
                W.phi[k] = __ldcg(W.phit + k);
                W.g[k] = __ldcg(W.gn + k);
            }
            if (tid == 0) {
                if (ok) {
                    if (np == m) W.scal[SC_HEAD] = (head + 1) % m;
                    else W.scal[SC_NP] = np + 1;
                }
                W.scal[SC_F] = __ldcg(W.scal + SC_FT);
                W.scal[SC_ITERS] = it + 1;
            }
        }
        if (!grid_sync(Pp.sync, Pp.err)) return;
    }

    // ---- remove the free constant: arg(sum_k w_k e^{i phi_k}) = 0; write phi ----
    if (blockIdx.x == 0) {
        double v[2] = {0.0, 0.0};
        for (int k = tid; k < P; k += nt) {
            double s, c;
            sincos(W.phi[k], &s, &c);
            const double wk = Pp.wts ? (double)Pp.wts[k] : 1.0;
            v[0] += wk * c;
            v[1] += wk * s;
        }
        block_sum_d<2>(v, red, out);
        const double shift = atan2(out[1], out[0]);
        for (int k = tid; k < P; k += nt) Pp.phi[k] = W.phi[k] - shift;
        if (tid == 0) {
            if (Pp.iters_done) *Pp.iters_done = (int)W.scal[SC_ITERS];
            if (Pp.loss_out) *Pp.loss_out = W.scal[SC_F];
        }
    }
}

cudaError_t launch_phase_fit(const PhaseFitParams &p, cudaStream_t s)
{
    const int grid = phase_fit_grid(p.ny, p.nx, p.Nd);
    const int P = p.ny * p.nx;
    const size_t sm = defocus_smem(p.ny, p.nx) + sizeof(double) * (32 * 4 + 16) + 2 * sizeof(float2);
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
