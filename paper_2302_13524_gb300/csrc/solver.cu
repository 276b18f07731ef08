// solver.cu -- persistent per-row retrieval (Algorithm 1) on thread-block clusters.
//
// One cluster of J CTAs solves one TM row at a time; rows come from an atomic
// work counter, so a launch of (clusters x J) CTAs walks the whole matrix.
// CTA j owns mask j:
//   registers: z_j = F(d_j .* t) (the current fields), y_j, and w_j = F(d_j .* p)
//              in the FFT's thread-strided layout -- never leave the chip;
//   shared:    d_j, the twiddle table, the FFT exchange buffer, and a 1/J
//              slice of every length-N vector: t, g, p and the L-BFGS pairs.
// Length-N vectors are all-gathered and sums over masks are reduced through
// distributed shared memory (DSMEM) between the CTAs of the cluster.
//
// One iteration (Algorithm 1: f and its gradient by FFT, L-BFGS step):
//   A  direction p = -H g on the slice from the compact L-BFGS form
//      H = gamma I + [S gamma Y] M [S^T; gamma Y^T]   (Byrd, Nocedal & Schnabel
//      1994; Nocedal & Wright eq. 7.24), coefficients from FP64 Gram scalars;
//   B1 cluster barrier, gather p;
//   C  w_j = F(d_j .* p)                                   (J FFTs per row)
//   D  quartic line-search sums of phi(a) = f(t + a p) = sum_i (r_i - 2 a Re(conj z_i w_i)
//      - a^2 |w_i|^2)^2; B2; exact minimiser from the cubic phi'(a) = 0 (FP64);
//   E  t += a p, z += a w, r = y - |z|^2, u = z .* r (registers);
//   F  v_j = conj(d_j) .* F^H u_j                          (J inverse FFTs)
//   B3; g = -4 sum_j v_j on the slice (Eq. derivative); new pair s = a p,
//      y = g_new - g_old;
//   G  all Gram dot products of the new vectors with the history in one batched
//      reduction; B4.
// Four cluster barriers and two FFT batches per iteration; the f and gradient
// of Algorithm 1 are those of the iterate produced by the previous step.
#include <cooperative_groups.h>

#include <cmath>

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace tmr {

enum { ROW_MAXITER = 0, ROW_CONVERGED = 1, ROW_ZERO = 2, ROW_NUMERIC = 3 };
enum { INIT_RANDOM = 0, INIT_BP = 1, INIT_SPECTRAL = 2 };

constexpr int kSlots = kMaxMem + 1;  // ring of m+1 slots: the new pair never overwrites a live one
constexpr int kMaxNV = 4 * kSlots + 4;

// FP64 L-BFGS scalars, replicated in every CTA of the cluster (each CTA computes
// them from identical reduced sums, so they agree bit for bit).
struct Gram {
    double SY[kSlots][kSlots];  // s_a^T y_b for slot a no newer than slot b
    double YY[kSlots][kSlots];  // y_a^T y_b, same convention
    double Sg[kSlots], Yg[kSlots];
    double c1[kSlots], c2[kSlots];  // direction coefficients per slot
    double gamma, gg, f, f_prev;
    double alpha;
    int order[kSlots];  // live slots, oldest first
    int np;             // number of live pairs
    int newslot;
    int status, done, stop, early;
};

__device__ __forceinline__ double quartic_val(const double *c, double a)
{
    return (((c[4] * a + c[3]) * a + c[2]) * a + c[1]) * a + c[0];
}

// Global minimiser over the real line of c0 + c1 a + ... + c4 a^4 (c4 > 0),
// among the real roots of the cubic derivative; ties go to the smallest
// positive root.  c4 == 0 means w == 0: no step.
__device__ double quartic_argmin(const double *c)
{
    if (!(c[4] > 0.0)) {
        if (c[2] > 0.0 && c[3] == 0.0) return -c[1] / (2.0 * c[2]);
        return 0.0;
    }
    const double B = 3.0 * c[3] / (4.0 * c[4]), C = 2.0 * c[2] / (4.0 * c[4]), D = c[1] / (4.0 * c[4]);
    const double p = C - B * B / 3.0;
    const double q = 2.0 * B * B * B / 27.0 - B * C / 3.0 + D;
    double roots[3];
    int nr = 0;
    const double disc = q * q / 4.0 + p * p * p / 27.0;
    if (disc > 0.0) {
        const double sq = sqrt(disc);
        const double u = cbrt(-q / 2.0 + (q > 0.0 ? -sq : sq));
        const double x = (u != 0.0) ? u - p / (3.0 * u) : 0.0;
        roots[nr++] = x - B / 3.0;
    } else if (p == 0.0) {
        roots[nr++] = -B / 3.0;
    } else {
        const double m = 2.0 * sqrt(-p / 3.0);
        double arg = 3.0 * q / (p * m);
        arg = arg > 1.0 ? 1.0 : (arg < -1.0 ? -1.0 : arg);
        const double th = acos(arg) / 3.0;
        for (int k = 0; k < 3; k++) roots[nr++] = m * cos(th - 2.0 * M_PI * k / 3.0) - B / 3.0;
    }
    double best = 0.0, bestv = 0.0;
    bool have = false;
    for (int k = 0; k < nr; k++) {
        double a = roots[k];
        for (int it = 0; it < 3; it++) {  // Newton polish on phi'
            const double f1 = ((4.0 * c[4] * a + 3.0 * c[3]) * a + 2.0 * c[2]) * a + c[1];
            const double f2 = (12.0 * c[4] * a + 6.0 * c[3]) * a + 2.0 * c[2];
            if (f2 == 0.0) break;
            const double na = a - f1 / f2;
            if (!isfinite(na)) break;
            a = na;
        }
        const double v = quartic_val(c, a);
        if (!have || v < bestv || (v == bestv && a > 0.0 && (best <= 0.0 || a < best))) {
            best = a;
            bestv = v;
            have = true;
        }
    }
    return best;
}

// Compact-form coefficients (run by one thread): p = -(gamma g + sum c1_i s_i
// + gamma sum c2_i y_i).  Falls back to p = -g (and clears the history) when
// there is no pair or the result is not a descent direction.
__device__ void lbfgs_coefficients(Gram &G)
{
    const int np = G.np;
    for (int a = 0; a < kSlots; a++) G.c1[a] = G.c2[a] = 0.0;
    if (np > 0) {
        const int nw = G.order[np - 1];
        const double gamma = G.SY[nw][nw] / G.YY[nw][nw];
        double av[kSlots], bv[kSlots], c2[kSlots], c1[kSlots];
        for (int i = 0; i < np; i++) {
            av[i] = G.Sg[G.order[i]];
            bv[i] = G.Yg[G.order[i]];
        }
        // R c2 = -a (R upper triangular in age order, R_ij = s_i^T y_j, i <= j)
        for (int i = np - 1; i >= 0; i--) {
            double s = -av[i];
            for (int j = i + 1; j < np; j++) s -= G.SY[G.order[i]][G.order[j]] * c2[j];
            c2[i] = s / G.SY[G.order[i]][G.order[i]];
        }
        // R^T c1 = -(D + gamma Y^T Y) c2 - gamma b
        for (int i = 0; i < np; i++) {
            double rhs = -G.SY[G.order[i]][G.order[i]] * c2[i] - gamma * bv[i];
            for (int j = 0; j < np; j++) {
                const int a = G.order[i < j ? i : j], b = G.order[i < j ? j : i];
                rhs -= gamma * G.YY[a][b] * c2[j];
            }
            for (int j = 0; j < i; j++) rhs -= G.SY[G.order[j]][G.order[i]] * c1[j];
            c1[i] = rhs / G.SY[G.order[i]][G.order[i]];
        }
        double pg = gamma * G.gg;
        for (int i = 0; i < np; i++) pg += c1[i] * av[i] + gamma * c2[i] * bv[i];
        // <p, g> = -pg must be negative
        if (pg > 0.0 && isfinite(pg)) {
            G.gamma = gamma;
            for (int i = 0; i < np; i++) {
                G.c1[G.order[i]] = c1[i];
                G.c2[G.order[i]] = c2[i];
            }
            return;
        }
        G.np = 0;
    }
    G.gamma = 1.0;
}

template <int N>
struct SolverCfg {
    static constexpr int NT = fft_threads(N);
    static constexpr int E = N / NT;
    static constexpr int TWN = FftPlan<N, E>::TW_SIZE;
    static constexpr int NW = NT / 32;
};

// Shared-memory carve-up (dynamic part).  SL = ceil(N / J) slice length.
template <int N>
struct SmemLayout {
    float2 *buf, *tw, *dm, *ps, *ts, *gs, *hs;  // hs: S slots then Y slots, each SL
    float *red, *pub;  // pub: two buffers of kMaxNV, used alternately
    Gram *gram;
    int *rowslot;
};

template <int N>
__host__ __device__ size_t solver_smem(int J, int m)
{
    using C = SolverCfg<N>;
    const int SL = (N + J - 1) / J;
    size_t f2 = (size_t)fft_buf_len(N) + C::TWN + N + 3 * (size_t)SL + 2 * (size_t)(m + 1) * SL;
    size_t bytes = f2 * sizeof(float2);
    bytes += sizeof(float) * (kMaxNV * C::NW + 2 * kMaxNV);
    bytes = (bytes + 15) & ~(size_t)15;
    bytes += sizeof(Gram) + 16;
    return bytes;
}

template <int N>
__device__ __forceinline__ SmemLayout<N> carve(unsigned char *base, int J, int m)
{
    using C = SolverCfg<N>;
    const int SL = (N + J - 1) / J;
    SmemLayout<N> L;
    float2 *f = reinterpret_cast<float2 *>(base);
    L.buf = f;
    f += fft_buf_len(N);
    L.tw = f;
    f += C::TWN;
    L.dm = f;
    f += N;
    L.ps = f;
    f += SL;
    L.ts = f;
    f += SL;
    L.gs = f;
    f += SL;
    L.hs = f;
    f += 2 * (size_t)(m + 1) * SL;
    float *fl = reinterpret_cast<float *>(f);
    L.red = fl;
    fl += kMaxNV * C::NW;
    L.pub = fl;
    fl += 2 * kMaxNV;
    size_t off = (reinterpret_cast<unsigned char *>(fl) - base + 15) & ~(size_t)15;
    L.gram = reinterpret_cast<Gram *>(base + off);
    L.rowslot = reinterpret_cast<int *>(base + off + sizeof(Gram));
    return L;
}

template <int N>
__global__ void __launch_bounds__(SolverCfg<N>::NT) k_solver(SolverParams P)
{
    using C = SolverCfg<N>;
    constexpr int NT = C::NT, E = C::E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cluster = cg::this_cluster();
    const int J = P.J, m = P.m, M = P.M;
    const int jr = (int)cluster.block_rank();
    const int tid = threadIdx.x;
    const int SL = (N + J - 1) / J;
    const int lo = (jr * N) / J, hi = ((jr + 1) * N) / J;  // my slice [lo, hi)
    const size_t K = (size_t)J * N;
    SmemLayout<N> L = carve<N>(smem_raw, J, m);
    float2 *S_slot = L.hs;                                  // S slot a at S_slot + a*SL
    float2 *Y_slot = L.hs + (size_t)(m + 1) * SL;           // Y slot a at Y_slot + a*SL
    Gram &G = *L.gram;

    // slice owner of index n: the largest o with (o N) / J <= n
    auto owner = [&](int n) {
        int o = (int)(((long long)n * J) / N);
        while (o + 1 < J && ((o + 1) * N) / J <= n) o++;
        while (o > 0 && (o * N) / J > n) o--;
        return o;
    };

    for (int i = tid; i < C::TWN; i += NT) L.tw[i] = P.tw[i];
    for (int i = tid; i < N; i += NT) L.dm[i] = P.masks[(size_t)jr * N + i];
    __syncthreads();

    // gather one thread-strided vector x[e] = dm[n] * v[n] from the peers' slices
    auto gather_masked = [&](float2 (&x)[E], float2 *slice_buf) {
#pragma unroll
        for (int e = 0; e < E; e++) {
            const int n = tid + e * NT;
            const int o = owner(n);
            const int olo = (o * N) / J;
            const float2 *rp = cluster.map_shared_rank(slice_buf, o);
            x[e] = cmul(rp[n - olo], L.dm[n]);
        }
    };
    // publish NV block sums in L.pub, barrier, and return the cluster totals in
    // FP64 summed in rank order (identical in every CTA)
    // The two publication buffers alternate: a peer may still be reading the
    // previous reduction's sums when this CTA publishes the next ones, but not
    // the ones before that (each reduction ends in a cluster barrier).
    int pub_sel = 0;
    auto cluster_sum = [&](auto &vals, double *out, int nv) {
        float *pb = L.pub + pub_sel * kMaxNV;
        pub_sel ^= 1;
        block_sum(vals, L.red, pb);
        cluster.sync();
        for (int k = 0; k < nv; k++) out[k] = 0.0;
        for (int o = 0; o < J; o++) {
            const float *rp = cluster.map_shared_rank(pb, o);
            for (int k = 0; k < nv; k++) out[k] += (double)rp[k];
        }
    };
    // v_j = conj(d_j) .* F^H u into L.buf (natural order, unpadded), barrier,
    // and return sum_j v_j on my slice via the callback
    auto adjoint_to_buf = [&](float2 (&u)[E]) {
        block_fft<N, NT, +1>(u, L.buf, L.tw, tid);
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; e++) {
            const int n = tid + e * NT;
            L.buf[n] = cmulc(u[e], L.dm[n]);
        }
        cluster.sync();
    };
    auto slice_sum = [&](int n) {
        float2 s = make_float2(0.f, 0.f);
        for (int o = 0; o < J; o++) {
            const float2 *rp = cluster.map_shared_rank(L.buf, o);
            s = cadd(s, rp[n]);
        }
        return s;
    };

    while (true) {
        if (jr == 0 && tid == 0) *L.rowslot = (int)atomicAdd(P.queue, 1u);
        cluster.sync();
        const int row = *cluster.map_shared_rank(L.rowslot, 0);
        // every peer has read rank 0's slot before rank 0 may rewrite it or any
        // CTA exits (a CTA's shared memory must outlive its peers' accesses)
        cluster.sync();
        if (row >= M) break;

        // ---- intensities of mask jr, their sum and finiteness ----
        float yv[E];
        float2 z[E];
        {
            float part[2] = {0.f, 0.f};
            const float *yr = P.y + (size_t)row * K + (size_t)jr * N;
#pragma unroll
            for (int e = 0; e < E; e++) {
                yv[e] = yr[tid + e * NT];
                if (isfinite(yv[e])) part[0] += yv[e];
                else part[1] += 1.f;
            }
            double tot[2];
            cluster_sum(part, tot, 2);
            if (tid == 0) {
                G.status = ROW_MAXITER;
                G.done = 0;
                G.np = 0;
                G.f = 0.0;
                G.stop = 0;
                G.early = 0;
                if (tot[1] > 0.0) { G.status = ROW_NUMERIC; G.stop = 1; G.early = 1; }
                else if (tot[0] == 0.0) { G.status = ROW_ZERO; G.stop = 1; G.early = 1; }
                G.f_prev = tot[0];  // sum(y), kept for the init scaling
            }
            __syncthreads();
        }
        const double sumy = G.f_prev;

        if (!G.stop) {
            // ---- initialisation ----
            const double JN = (double)J * N;
            if (P.T_init) {
                for (int n = lo + tid; n < hi; n += NT) L.ts[n - lo] = P.T_init[(size_t)row * N + n];
            } else if (P.init == INIT_BP) {
                float2 u[E];
#pragma unroll
                for (int e = 0; e < E; e++) u[e] = make_float2(sqrtf(fmaxf(yv[e], 0.f)), 0.f);
                adjoint_to_buf(u);
                for (int n = lo + tid; n < hi; n += NT) L.ts[n - lo] = cscale(slice_sum(n), (float)(1.0 / JN));
            } else {
                for (int n = lo + tid; n < hi; n += NT)
                    L.ts[n - lo] = philox_cnormal(P.seed, (uint32_t)row, (uint32_t)n);
                if (P.init == INIT_SPECTRAL) {
                    const float mean = (float)(sumy / (double)K);
                    float tau[E];
#pragma unroll
                    for (int e = 0; e < E; e++) {
                        float tv = yv[e] / mean;
                        if (P.clip > 0.f && tv > P.clip) tv = P.clip;
                        tau[e] = tv;
                    }
                    for (int it = 0; it < P.power_iters; it++) {
                        for (int n = lo + tid; n < hi; n += NT) L.ps[n - lo] = L.ts[n - lo];
                        cluster.sync();
                        float2 x[E];
                        gather_masked(x, L.ps);
                        block_fft<N, NT, -1>(x, L.buf, L.tw, tid);
#pragma unroll
                        for (int e = 0; e < E; e++) x[e] = cscale(x[e], tau[e]);
                        adjoint_to_buf(x);
                        float part[1] = {0.f};
                        for (int n = lo + tid; n < hi; n += NT) {
                            const float2 s = cscale(slice_sum(n), (float)(1.0 / JN));
                            L.ts[n - lo] = s;
                            part[0] += cabs2(s);
                        }
                        double nrm;
                        cluster_sum(part, &nrm, 1);
                        const float inv = nrm > 0.0 ? (float)(1.0 / sqrt(nrm)) : 0.f;
                        for (int n = lo + tid; n < hi; n += NT) L.ts[n - lo] = cscale(L.ts[n - lo], inv);
                    }
                }
                // rescale to the Parseval norm ||t||^2 = sum(y) / (J N)
                float part[1] = {0.f};
                for (int n = lo + tid; n < hi; n += NT) part[0] += cabs2(L.ts[n - lo]);
                double nrm;
                cluster_sum(part, &nrm, 1);
                const float sc = nrm > 0.0 ? (float)(sqrt(sumy / JN) / sqrt(nrm)) : 0.f;
                for (int n = lo + tid; n < hi; n += NT) L.ts[n - lo] = cscale(L.ts[n - lo], sc);
            }

            // ---- f and gradient at t0 ----
            {
                for (int n = lo + tid; n < hi; n += NT) L.ps[n - lo] = L.ts[n - lo];
                cluster.sync();
                gather_masked(z, L.ps);
                block_fft<N, NT, -1>(z, L.buf, L.tw, tid);
                float2 u[E];
                float part[2] = {0.f, 0.f};
#pragma unroll
                for (int e = 0; e < E; e++) {
                    const float r = yv[e] - cabs2(z[e]);
                    part[0] = fmaf(r, r, part[0]);
                    u[e] = cscale(z[e], r);
                }
                adjoint_to_buf(u);
                for (int n = lo + tid; n < hi; n += NT) {
                    const float2 g = cscale(slice_sum(n), -4.f);
                    L.gs[n - lo] = g;
                    part[1] += cabs2(g);
                }
                double tot[2];
                cluster_sum(part, tot, 2);
                if (tid == 0) {
                    G.f = tot[0];
                    G.gg = tot[1];
                    G.np = 0;
                    if (!isfinite(tot[0]) || !isfinite(tot[1])) { G.status = ROW_NUMERIC; G.stop = 1; }
                }
                __syncthreads();
            }

            // ---- L-BFGS iterations ----
            for (int it = 0; it < P.iters && !G.stop; it++) {
                // A: direction
                if (tid == 0) {
                    if (G.f == 0.0 || G.gg == 0.0) {
                        G.status = ROW_CONVERGED;
                        G.stop = 1;
                    } else {
                        lbfgs_coefficients(G);
                        // free slot for the new pair
                        bool used[kSlots] = {false};
                        for (int i = 0; i < G.np; i++) used[G.order[i]] = true;
                        int ns = 0;
                        while (used[ns]) ns++;
                        G.newslot = ns;
                    }
                }
                __syncthreads();
                if (G.stop) break;
                {
                    const float gam = (float)G.gamma;
                    const int np = G.np;
                    for (int n = lo + tid; n < hi; n += NT) {
                        const int i = n - lo;
                        float2 acc = cscale(L.gs[i], gam);
                        for (int k = 0; k < np; k++) {
                            const int a = G.order[k];
                            acc = cadd(acc, cscale(S_slot[(size_t)a * SL + i], (float)G.c1[a]));
                            acc = cadd(acc, cscale(Y_slot[(size_t)a * SL + i], (float)(G.gamma * G.c2[a])));
                        }
                        L.ps[i] = cscale(acc, -1.f);
                    }
                }
                cluster.sync();  // B1
                // C: w = F(d .* p)
                float2 w[E];
                gather_masked(w, L.ps);
                block_fft<N, NT, -1>(w, L.buf, L.tw, tid);
                // D: quartic coefficients
                {
                    float part[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int e = 0; e < E; e++) {
                        const float a = cdotr(z[e], w[e]);
                        const float b = cabs2(w[e]);
                        const float r = yv[e] - cabs2(z[e]);
                        part[0] = fmaf(r, r, part[0]);
                        part[1] = fmaf(-4.f * r, a, part[1]);
                        part[2] += fmaf(4.f * a, a, -2.f * r * b);
                        part[3] = fmaf(4.f * a, b, part[3]);
                        part[4] = fmaf(b, b, part[4]);
                    }
                    double c[5];
                    cluster_sum(part, c, 5);  // B2
                    if (tid == 0) {
                        const double al = quartic_argmin(c);
                        G.alpha = al;
                        if (!isfinite(al)) { G.status = ROW_NUMERIC; G.stop = 1; }
                        else if (al == 0.0) { G.status = ROW_CONVERGED; G.stop = 1; }
                    }
                    __syncthreads();
                }
                if (G.stop) break;
                const float al = (float)G.alpha;
                // E: update
                float2 u[E];
                float fpart = 0.f;
#pragma unroll
                for (int e = 0; e < E; e++) {
                    z[e] = make_float2(fmaf(al, w[e].x, z[e].x), fmaf(al, w[e].y, z[e].y));
                    const float r = yv[e] - cabs2(z[e]);
                    fpart = fmaf(r, r, fpart);
                    u[e] = cscale(z[e], r);
                }
                const int ns = G.newslot;
                for (int n = lo + tid; n < hi; n += NT) {
                    const int i = n - lo;
                    const float2 s = cscale(L.ps[i], al);
                    S_slot[(size_t)ns * SL + i] = s;
                    L.ts[i] = cadd(L.ts[i], s);
                }
                // F: adjoint
                adjoint_to_buf(u);  // B3
                // new gradient, new y, and the batched dot products
                {
                    const int np = G.np;
                    float part[kMaxNV];
#pragma unroll
                    for (int k = 0; k < kMaxNV; k++) part[k] = 0.f;
                    for (int n = lo + tid; n < hi; n += NT) {
                        const int i = n - lo;
                        const float2 gn = cscale(slice_sum(n), -4.f);
                        const float2 yn = csub(gn, L.gs[i]);
                        L.gs[i] = gn;
                        Y_slot[(size_t)ns * SL + i] = yn;
                        const float2 sn = S_slot[(size_t)ns * SL + i];
                        // slots: live ones in age order, then the new slot (index np)
#pragma unroll
                        for (int k = 0; k < kSlots; k++) {
                            if (k <= np) {
                                const int a = (k < np) ? G.order[k] : ns;
                                const float2 sa = S_slot[(size_t)a * SL + i];
                                const float2 ya = Y_slot[(size_t)a * SL + i];
                                part[4 * k + 0] += cdotr(sa, yn);
                                part[4 * k + 1] += cdotr(ya, yn);
                                part[4 * k + 2] += cdotr(sa, gn);
                                part[4 * k + 3] += cdotr(ya, gn);
                            }
                        }
                        part[4 * kSlots + 0] += cabs2(sn);
                        part[4 * kSlots + 1] += cabs2(gn);
                    }
                    part[4 * kSlots + 2] = fpart;
                    double tot[kMaxNV];
                    cluster_sum(part, tot, kMaxNV);  // B4
                    if (tid == 0) {
                        // Gram update for the new pair (slot ns)
                        for (int k = 0; k <= np; k++) {
                            const int a = (k < np) ? G.order[k] : ns;
                            G.SY[a][ns] = tot[4 * k + 0];
                            G.YY[a][ns] = tot[4 * k + 1];
                            G.Sg[a] = tot[4 * k + 2];
                            G.Yg[a] = tot[4 * k + 3];
                        }
                        const double sy = tot[4 * np + 0], yy = tot[4 * np + 1];
                        const double ss = tot[4 * kSlots + 0];
                        const double fnew = tot[4 * kSlots + 2];
                        G.gg = tot[4 * kSlots + 1];
                        if (sy > 1e-10 * sqrt(ss) * sqrt(yy) && sy > 0.0) {
                            G.order[G.np++] = ns;
                            if (G.np > m) {
                                for (int k = 0; k + 1 < G.np; k++) G.order[k] = G.order[k + 1];
                                G.np--;
                            }
                        }
                        const double rel = fabs(G.f - fnew) / fmax(G.f, 1e-30);
                        G.f = fnew;
                        G.done = it + 1;
                        if (!isfinite(fnew) || !isfinite(G.gg)) { G.status = ROW_NUMERIC; G.stop = 1; }
                        else if (P.tol > 0.0 && rel < P.tol) { G.status = ROW_CONVERGED; G.stop = 1; }
                    }
                    __syncthreads();
                }
            }
        }

        // ---- outputs (rows decided before initialisation come back as zero) ----
        const bool early = G.early != 0;
        for (int n = lo + tid; n < hi; n += NT)
            P.T_out[(size_t)row * N + n] = early ? make_float2(0.f, 0.f) : L.ts[n - lo];
        if (jr == 0 && tid == 0) {
            if (P.row_status) P.row_status[row] = G.status;
            if (P.row_iters) P.row_iters[row] = G.done;
            if (P.row_loss) P.row_loss[row] = early ? (G.status == ROW_ZERO ? 0.f : __int_as_float(0x7fc00000))
                                                    : (float)G.f;
        }
        if (P.Zd) {
#pragma unroll
            for (int e = 0; e < E; e++) {
                const int pat = jr * N + tid + e * NT;
                if (pat < P.Nd) P.Zd[(size_t)pat * M + row] = early ? make_float2(0.f, 0.f) : z[e];
            }
        }
        cluster.sync();  // all peers done with this row's shared data
    }
}

template <int N>
static cudaError_t launch_solver_t(const SolverParams &p, cudaStream_t s, int *clusters_out)
{
    using C = SolverCfg<N>;
    const size_t sm = solver_smem<N>(p.J, p.m);
    cudaError_t e = cudaFuncSetAttribute(k_solver<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (p.J > 8) {
        e = cudaFuncSetAttribute(k_solver<N>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = p.J;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(C::NT);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(p.J);
    int maxc = 0;
    e = cudaOccupancyMaxActiveClusters(&maxc, k_solver<N>, &cfg);
    if (e != cudaSuccess) return e;
    if (maxc < 1) return cudaErrorInvalidConfiguration;
    int nc = maxc < p.M ? maxc : p.M;
    if (nc < 1) nc = 1;
    cfg.gridDim = dim3(nc * p.J);
    if (clusters_out) *clusters_out = nc;
    return cudaLaunchKernelEx(&cfg, k_solver<N>, p);
}

size_t solver_smem_bytes(int N, int J, int m)
{
    switch (N) {
    case 64: return solver_smem<64>(J, m);
    case 128: return solver_smem<128>(J, m);
    case 256: return solver_smem<256>(J, m);
    case 512: return solver_smem<512>(J, m);
    case 1024: return solver_smem<1024>(J, m);
    case 2048: return solver_smem<2048>(J, m);
    case 4096: return solver_smem<4096>(J, m);
    default: return 0;
    }
}

cudaError_t launch_solver(int N, const SolverParams &p, cudaStream_t s, int *clusters_out)
{
    if (p.M == 0) return cudaSuccess;
    switch (N) {
    case 64: return launch_solver_t<64>(p, s, clusters_out);
    case 128: return launch_solver_t<128>(p, s, clusters_out);
    case 256: return launch_solver_t<256>(p, s, clusters_out);
    case 512: return launch_solver_t<512>(p, s, clusters_out);
    case 1024: return launch_solver_t<1024>(p, s, clusters_out);
    case 2048: return launch_solver_t<2048>(p, s, clusters_out);
    case 4096: return launch_solver_t<4096>(p, s, clusters_out);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tmr
