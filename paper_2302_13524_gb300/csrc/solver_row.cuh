// solver_row.cuh -- the per-row solver (Algorithm 1) with one CTA per row.
//
// The same iteration as k_solver (solver_impl.cuh): initialisation, then
// L-BFGS steps each made of one forward batch w_j = F(d_j .* p), the exact
// minimiser of the quartic phi(a) = f(t + a p), the update t += a p,
// z += a w, one adjoint batch for the new gradient (Eq. derivative) and the
// compact-form direction from the Gram scalars.  What differs is the layout,
// chosen so that a row needs no thread-block cluster:
//   * every mask of the row is a team of NT = N/16 threads in one CTA, each
//     thread holding 16 points of z_j and w_j in registers; the transforms
//     are register Stockham passes of radix 16 after a first pass of the
//     remaining radix (2048 = 8 x 16 x 16: two exchanges through shared
//     memory per transform), the last pass's twiddles formed from per-thread
//     bases and the others' in a small table made on the device (FP64
//     sincospi rounded to FP32);
//   * the masks and the row's intensities live in shared memory (the masks
//     are copied once per CTA and shared by all its rows), next to full-length
//     t, g and the direction p, and one exchange buffer per team;
//   * the L-BFGS pairs (2 (m + 1) vectors of N complex values, 192 KB at
//     N = 2048, m = 5) live in the SM's tensor memory, which the FP32 solver
//     has no other use for: each thread keeps the elements it owns in the
//     A and G phases (i = tid + e BT) in columns of its own lane, so the two
//     passes over the pairs of every iteration read tensor memory instead of
//     L2; before the first pair exists, the same columns hold the vectors of
//     the Lanczos start where they fit (k N complex values: 256 KB, all 512
//     columns, at N = 2048, J = 4, k = 16), else those stay in global memory;
//   * every exchange and every reduction is inside the CTA: block barriers
//     instead of cluster barriers, no distributed shared memory.
// Rows come from the same atomic work counter; a persistent launch of one
// CTA per SM (or two, when shared memory allows) walks the matrix.
#pragma once

#include "solver_impl.cuh"
#include "tmem.cuh"

namespace tmr {

constexpr int kRowPts = 16;

template <int N_>
struct RowCfg {
    static constexpr int N = N_;
    static constexpr int E = kRowPts;  // points per thread of one transform
    static constexpr int NT = N_ / E;  // threads per team (one mask)
    static constexpr int R = 16;       // radix of every pass but the first
    static constexpr int BPT = E / R;  // butterflies per thread in the last pass
    using Plan = FftPlan<N_, E, R>;
    static constexpr int NCONST = Plan::TW_SMALL;  // twiddles of the non-final passes
    static constexpr int LBUF = fft_buf_len(N_);
};

// Variants exist for N = 512 .. 2048 with J * N / 16 <= 512 threads.
__host__ __device__ constexpr bool row_variant_fits(int N, int J) { return J >= 1 && J * (N / kRowPts) <= 512; }

template <int N>
__host__ __device__ size_t row_smem(int J, int m)
{
    using C = RowCfg<N>;
    (void)m;
    const int NW = J * C::NT / 32;
    size_t f2 = ((size_t)C::NCONST + 1) / 2 * 2 /*twiddles, even count*/ + (size_t)J * N /*masks*/ +
                (size_t)J * C::LBUF /*team exchange buffers*/ + 3 * (size_t)N /*p, t, g*/;
    size_t bytes = f2 * sizeof(float2) + sizeof(float) * ((size_t)J * N /*y*/ + (size_t)kParts * (NW > 0 ? NW : 1));
    bytes = (bytes + 15) & ~(size_t)15;
    return bytes + sizeof(Gram);
}

// Tensor-memory columns of one CTA.  Thread tid owns elements tid + e BT,
// e < EPT = ceil(N / BT), of every pair and Lanczos vector.  A warp's block of
// pair columns holds (m + 1) slots x EPT elements x (s re, s im, y re, y im);
// its block of Lanczos columns EPT elements x KM vectors x (re, im), KM = k
// rounded up to a multiple of 4; the up to four warps that share a lane
// quarter take consecutive blocks.  Every row variant with m <= 6 needs at
// most 504 columns for its pairs; the Lanczos vectors go to tensor memory when
// their blocks fit in 512 columns (klz = k steps, else 0).  The allocation is
// the next power of two of the larger need (at least 32).
__host__ __device__ inline int row_ept(int N, int J) { return (N + J * (N / kRowPts) - 1) / (J * (N / kRowPts)); }
__host__ __device__ inline int row_tmem_block(int N, int J, int m) { return 4 * row_ept(N, J) * (m + 1); }
__host__ __device__ inline int row_tmem_lanczos_block(int N, int J, int k) { return 2 * row_ept(N, J) * ((k + 3) & ~3); }
__host__ __device__ inline int row_quarter_warps(int N, int J) { return (J * (N / kRowPts) / 32 + 3) / 4; }
__host__ __device__ inline int row_tmem_klz(int N, int J, bool lanczos_start, int k)
{
    return lanczos_start && k >= 1 && k <= kMaxLanczos && row_quarter_warps(N, J) * row_tmem_lanczos_block(N, J, k) <= 512
               ? k
               : 0;
}
__host__ __device__ inline int row_tmem_cols(int N, int J, int m, int klz)
{
    int need = row_quarter_warps(N, J) * row_tmem_block(N, J, m);
    if (klz > 0) {
        const int lz = row_quarter_warps(N, J) * row_tmem_lanczos_block(N, J, klz);
        if (lz > need) need = lz;
    }
    int c = 32;
    while (c < need) c *= 2;
    return c;
}

// No global pair workspace: the pairs are in tensor memory.
__host__ __device__ inline size_t row_pair_stride(int N, int m)
{
    (void)N;
    (void)m;
    return 0;
}

template <int N, int COST = COST_INTENSITY>
__global__ void __launch_bounds__(512, 1) k_solver_row(SolverParams P)
{
    using C = RowCfg<N>;
    constexpr int NT = C::NT, E = C::E, R = C::R, BPT = C::BPT, NCONST = C::NCONST, LBUF = C::LBUF;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int J = P.J, m = P.m, M = P.M;
    const int BT = J * NT;
    const int NW = BT / 32;
    const int tid = threadIdx.x;
    const int team = tid / NT, ttid = tid - team * NT;
    const int lane = tid & 31, warp = tid >> 5;
    const size_t K = (size_t)J * N;
    const float JN = (float)K;
    const float gsc = cost_grad_scale(COST);  // the gradient's scale (-4 intensity, 2 amplitude)

    // ---- shared memory ----
    float2 *tws = reinterpret_cast<float2 *>(smem_raw);
    float2 *msk = tws + (NCONST + 1) / 2 * 2;     // [J][N]
    float2 *bufs = msk + (size_t)J * N;           // [J][LBUF]
    float2 *buf = bufs + (size_t)team * LBUF;     // this team's exchange buffer
    float2 *X = bufs + (size_t)J * LBUF;          // direction p (or the vector being transformed)
    float2 *ts = X + N;                           // t
    float2 *gs = ts + N;                          // g
    float *ys = reinterpret_cast<float *>(gs + N);  // [J][N] intensities of the row (scaled)
    float *red = ys + (size_t)J * N;                // [kParts][NW]
    Gram &Gm = *reinterpret_cast<Gram *>(
        smem_raw + ((reinterpret_cast<unsigned char *>(red + kParts * NW) - smem_raw + 15) & ~(size_t)15));

    // L-BFGS pairs in tensor memory: element e (i = tid + e BT) of the pair in
    // slot a at columns tcol(a, e) .. + 3 (s, then y)
    __shared__ uint32_t tmem_base;
    const int klz = row_tmem_klz(N, J, P.lanczos && P.init == INIT_SPECTRAL && !P.T_init, P.power_iters);
    const int ncols = row_tmem_cols(N, J, m, klz);
    if (warp == 0) tmem_alloc_warp(&tmem_base, (uint32_t)ncols);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const int EPT = (N + BT - 1) / BT;
    const uint32_t tquarter = tmem_base + ((uint32_t)(32 * (warp & 3)) << 16);
    const uint32_t tlane = tquarter + (uint32_t)((warp >> 2) * row_tmem_block(N, J, m));
    auto tcol = [&](int a, int e) { return tlane + (uint32_t)(4 * (a * EPT + e)); };

    // twiddles of the passes between the first and the last:
    // tw_p[(r - 1) Ns + j] = exp(-2 pi i r j / (Ns R)) at tw_off(p)
    for (int p = 1; p < C::Plan::P - 1; p++) {
        const int Rp = C::Plan::radix(p), Ns = C::Plan::ns(p), off = C::Plan::tw_off(p);
        for (int i = tid; i < (Rp - 1) * Ns; i += BT) {
            const int r = 1 + i / Ns, j = i - (r - 1) * Ns;
            double s, c;
            sincospi(-2.0 * (double)r * (double)j / ((double)Ns * Rp), &s, &c);
            tws[off + i] = make_float2((float)c, (float)s);
        }
    }
    for (int i = tid; i < J * N; i += BT) msk[i] = P.masks[i];
    const float2 *dm = msk + (size_t)team * N;  // this team's mask
    const float *yt = ys + (size_t)team * N;    // this team's intensities
    float2 wb[BPT];  // last-pass twiddle bases exp(-2 pi i b / N), b = ttid + i NT
#pragma unroll
    for (int i = 0; i < BPT; i++) {
        double s, c;
        sincospi(-2.0 * (double)(ttid + i * NT) / (double)N, &s, &c);
        wb[i] = make_float2((float)c, (float)s);
    }
    __syncthreads();

    // x <- F(d .* x) and x <- conj(d) .* F^H x for this team's mask; every team
    // runs the same passes, so the block barriers inside line up
    auto fwd = [&](float2 (&x)[E]) {
#pragma unroll
        for (int e = 0; e < E; e++) x[e] = cmul(x[e], dm[ttid + e * NT]);
        block_fft_rbx<N, NT, R, -1>(x, buf, tws, wb, ttid);
    };
    auto adj = [&](float2 (&x)[E]) {
        block_fft_rbx<N, NT, R, +1>(x, buf, tws, wb, ttid);
#pragma unroll
        for (int e = 0; e < E; e++) x[e] = cmulc(x[e], dm[ttid + e * NT]);
    };
    // after a transform every thread has passed its last exchange, so the team
    // buffer is free: park the natural-order result there (unpadded)
    auto park = [&](const float2 (&x)[E]) {
#pragma unroll
        for (int e = 0; e < E; e++) buf[ttid + e * NT] = x[e];
    };
    // sum over the masks of the parked results, element i, times s
    auto team_sum = [&](int i, float s) {
        float2 acc = bufs[i];
        for (int j = 1; j < J; j++) acc = cadd(acc, bufs[(size_t)j * LBUF + i]);
        return cscale(acc, s);
    };
    auto load_team = [&](const float2 *src, float2 (&x)[E]) {
#pragma unroll
        for (int e = 0; e < E; e++) x[e] = src[ttid + e * NT];
    };
    // Block-wide sums of nv <= 32 per-thread values: warp sums, then thread k
    // adds the NW warp sums of value k in warp order into Gm.red[k].  With
    // all = false only warp 0 (threads 0 .. 31) goes on to read the sums, so
    // a warp barrier replaces the block barrier after them.
    auto block_reduce = [&](float (&v)[32], int nv, bool all = true) {
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
            Gm.red[tid] = acc;
        }
        if (all) __syncthreads();
        else __syncwarp();
    };

    while (true) {
        if (tid == 0) Gm.row = (int)atomicAdd(P.queue, 1u);
        __syncthreads();
        const int row = Gm.row;
        if (row >= M) break;

        // ---- intensities, their sum and finiteness ----
        {
            float pv[32] = {0.f};
            const float *yr = P.y + (size_t)row * K;
            for (size_t i = tid; i < K; i += BT) {
                const float v = yr[i];
                ys[i] = v;
                if (isfinite(v)) pv[0] += v;
                else pv[1] += 1.f;
            }
            block_reduce(pv, 2);
            if (tid == 0) {
                Gm.status = ROW_MAXITER;
                Gm.done = 0;
                Gm.np = 0;
                Gm.f = 0.f;
                Gm.stop = 0;
                Gm.early = 0;
                Gm.sumy = Gm.red[0];
                const int js = row_scale_exp(Gm.red[0], (int)K);
                Gm.yscale = ldexpf(1.f, -2 * js);
                Gm.tsc = ldexpf(1.f, js);
                if (Gm.red[1] > 0.f || !isfinite(Gm.red[0])) { Gm.status = ROW_NUMERIC; Gm.stop = 1; Gm.early = 1; }
                else if (Gm.red[0] == 0.f) { Gm.status = ROW_ZERO; Gm.stop = 1; Gm.early = 1; }
            }
            __syncthreads();
            // the row is solved with y 4^-j and t 2^-j (exact scales; see k_solver)
            const float ysc = Gm.yscale;
            for (size_t i = tid; i < K; i += BT) ys[i] *= ysc;
            __syncthreads();
        }
        const float sumy = Gm.sumy * Gm.yscale;
        float2 z[E];
#pragma unroll
        for (int e = 0; e < E; e++) z[e] = make_float2(0.f, 0.f);

        if (!Gm.stop) {
            // ---- initialisation ----
            if (P.T_init) {
                const float tinv = 1.f / Gm.tsc;
                for (int i = tid; i < N; i += BT) ts[i] = cscale(P.T_init[(size_t)row * N + i], tinv);
            } else if (P.init == INIT_BP) {
                float2 u[E];
#pragma unroll
                for (int e = 0; e < E; e++) u[e] = make_float2(sqrtf(fmaxf(yt[ttid + e * NT], 0.f)), 0.f);
                adj(u);
                park(u);
                __syncthreads();
                for (int i = tid; i < N; i += BT) ts[i] = team_sum(i, 1.f / JN);
            } else {
                // seed: the proposed start (learned initialiser) where it is
                // finite and nonzero, else the Philox vector
                bool seeded = false;
                if (P.T_cand && P.seed_from_cand) {
                    float pv[32] = {0.f};
                    for (int i = tid; i < N; i += BT) {
                        const float2 v = P.T_cand[(size_t)row * N + i];
                        ts[i] = v;
                        pv[0] += cabs2(v);
                    }
                    block_reduce(pv, 1);
                    seeded = isfinite(Gm.red[0]) && Gm.red[0] > 0.f;
                    if (seeded && tid == 0 && P.cand_wins) atomicAdd(P.cand_wins, 1u);
                }
                if (!seeded)
                    for (int i = tid; i < N; i += BT) ts[i] = philox_cnormal(P.seed, (uint32_t)row, (uint32_t)i);
                if (P.init == INIT_SPECTRAL && P.lanczos) {
                    const float mean = sumy / (float)K;
                    auto applyA = [&]() {
                        __syncthreads();
                        float2 x[E];
                        load_team(ts, x);
                        fwd(x);
#pragma unroll
                        for (int e = 0; e < E; e++) {
                            float tv = yt[ttid + e * NT] / mean;
                            if (P.clip > 0.f && tv > P.clip) tv = P.clip;
                            x[e] = cscale(x[e], tv);
                        }
                        adj(x);
                        park(x);
                        __syncthreads();
                        for (int i = tid; i < N; i += BT) gs[i] = team_sum(i, 1.f / JN);
                        __syncthreads();
                    };
                    float2 *V = P.krylov + (size_t)blockIdx.x * lanczos_region(N, P.power_iters);
                    // (the direction p is not in use yet: its buffer X holds
                    // the Gram matrix of the Lanczos vectors)
                    if (klz)
                        lanczos_start_tmem(klz, N, EPT,
                                           tquarter + (uint32_t)((warp >> 2) * row_tmem_lanczos_block(N, J, klz)), ts,
                                           gs, X, Gm.red, &Gm.SY[0][0], &Gm.YY[0][0], applyA, block_reduce);
                    else
                        lanczos_start(P.power_iters, N, ts, gs, V, (size_t)N, V + (size_t)P.power_iters * N, Gm.red,
                                      &Gm.SY[0][0], &Gm.YY[0][0], applyA, block_reduce);
                } else if (P.init == INIT_SPECTRAL) {
                    const float mean = sumy / (float)K;
                    for (int it = 0; it < P.power_iters; it++) {
                        // t <- A t, A = Q^H diag(tau) Q / (J N), tau = min(y / mean, clip);
                        // the norm is restored every 8th step and at the end
                        __syncthreads();
                        float2 x[E];
                        load_team(ts, x);
                        fwd(x);
#pragma unroll
                        for (int e = 0; e < E; e++) {
                            float tv = yt[ttid + e * NT] / mean;
                            if (P.clip > 0.f && tv > P.clip) tv = P.clip;
                            x[e] = cscale(x[e], tv);
                        }
                        adj(x);
                        park(x);
                        __syncthreads();
                        const bool renorm = ((it & 7) == 7) || (it == P.power_iters - 1);
                        float pv[32] = {0.f};
                        for (int i = tid; i < N; i += BT) {
                            const float2 s = team_sum(i, 1.f / JN);
                            ts[i] = s;
                            pv[0] = fmaf(s.x, s.x, fmaf(s.y, s.y, pv[0]));
                        }
                        if (renorm) {
                            block_reduce(pv, 1);
                            const float nrm = Gm.red[0];
                            const float inv = nrm > 0.f ? rsqrtf(nrm) : 0.f;
                            for (int i = tid; i < N; i += BT) ts[i] = cscale(ts[i], inv);
                        }
                    }
                }
                // rescale to the Parseval norm ||t||^2 = sum(y) / (J N)
                float pv[32] = {0.f};
                for (int i = tid; i < N; i += BT) pv[0] += cabs2(ts[i]);
                block_reduce(pv, 1);
                const float nrm = Gm.red[0];
                const float sc = nrm > 0.f ? sqrtf(sumy / JN) / sqrtf(nrm) : 0.f;
                for (int i = tid; i < N; i += BT) ts[i] = cscale(ts[i], sc);
            }

            // ---- per-row selection: a proposed start (learned initialiser) against this one ----
            if (P.T_cand && P.judge_cand) {
                const float tinv = 1.f / Gm.tsc;
                for (int i = tid; i < N; i += BT) gs[i] = cscale(P.T_cand[(size_t)row * N + i], tinv);
                float fv[2];
                for (int c = 0; c < 2; c++) {  // f at the start above, then at the proposal
                    __syncthreads();
                    float2 x[E];
                    load_team(c == 0 ? ts : gs, x);
                    fwd(x);
                    float pv[32] = {0.f};
#pragma unroll
                    for (int e = 0; e < E; e++) {
                        cost_coef(COST, x[e], yt[ttid + e * NT], pv[0]);
                    }
                    block_reduce(pv, 1);
                    fv[c] = Gm.red[0];
                }
                if (fv[1] < fv[0]) {  // NaN proposals lose
                    for (int i = tid; i < N; i += BT) ts[i] = gs[i];
                    if (tid == 0 && P.cand_wins) atomicAdd(P.cand_wins, 1u);
                }
            }

            // ---- f and gradient at the start ----
            {
                __syncthreads();
                load_team(ts, z);
                fwd(z);
                float2 u[E];
                float pv[32] = {0.f};
#pragma unroll
                for (int e = 0; e < E; e++) u[e] = cscale(z[e], cost_coef(COST, z[e], yt[ttid + e * NT], pv[0]));
                adj(u);
                park(u);
                __syncthreads();
                for (int i = tid; i < N; i += BT) {
                    const float2 g = team_sum(i, gsc);
                    gs[i] = g;
                    pv[1] += cabs2(g);
                }
                block_reduce(pv, 2);
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
            }

            // ---- L-BFGS iterations ----
            for (int it = 0; it < P.iters && !Gm.stop; it++) {
                const int np = Gm.np;
                int so[kSlots];  // slots by age
#pragma unroll
                for (int k = 0; k < kSlots; k++) so[k] = Gm.slot[k <= np ? k : 0];
                const int sn_slot = so[np < kSlots ? np : 0];  // the free slot (age np) of the new pair
                // A: direction p = -(gamma g + sum c1 s + sum c2 y) into X
                {
                    const float gam = Gm.gamma;
                    float c1r[kSlots], c2r[kSlots];
#pragma unroll
                    for (int k = 0; k < kSlots; k++) {
                        c1r[k] = k < np ? Gm.c1[k] : 0.f;
                        c2r[k] = k < np ? Gm.c2[k] : 0.f;
                    }
                    // every thread runs all EPT steps (the tensor-memory loads
                    // are warp-wide); steps past N only load
                    tmem_fence_after_sync();
                    for (int e = 0; e < EPT; e++) {
                        const int i = tid + e * BT;
                        const bool in = i < N;
                        float2 acc = in ? cscale(gs[i], gam) : make_float2(0.f, 0.f);
#pragma unroll
                        for (int k = 0; k < kSlots; k++) {
                            if (k < np) {
                                uint32_t r[4];
                                tmem_ld4(tcol(so[k], e), r);
                                tmem_wait_ld();
                                tmem_reg_ready(r);
                                const float2 sa = make_float2(__uint_as_float(r[0]), __uint_as_float(r[1]));
                                const float2 ya = make_float2(__uint_as_float(r[2]), __uint_as_float(r[3]));
                                acc.x = fmaf(c1r[k], sa.x, fmaf(c2r[k], ya.x, acc.x));
                                acc.y = fmaf(c1r[k], sa.y, fmaf(c2r[k], ya.y, acc.y));
                            }
                        }
                        if (in) X[i] = make_float2(-acc.x, -acc.y);
                    }
                }
                __syncthreads();
                // C: w = F(d .* p)
                float2 w[E];
                load_team(X, w);
                fwd(w);
                // D: the step -- the amplitude cost's line search, or the quartic's exact minimiser
                if constexpr (COST == COST_AMPLITUDE) {
                    const float al = amp_line_search(
                        z, w, [&](int e) { return yt[ttid + e * NT]; }, [](int) { return true; }, block_reduce,
                        Gm.red, Gm.red + 16);
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
                        const float r = yt[ttid + e * NT] - cabs2(z[e]);
                        pv[0] = fmaf(r, r, pv[0]);
                        pv[1] = fmaf(-4.f * r, a, pv[1]);
                        pv[2] += fmaf(4.f * a, a, -2.f * r * b);
                        pv[3] = fmaf(4.f * a, b, pv[3]);
                        pv[4] = fmaf(b, b, pv[4]);
                    }
                    block_reduce(pv, 5, false);
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
                // E: fields, residual, t += a p, then the adjoint
                float2 u[E];
                float fpart = 0.f;
#pragma unroll
                for (int e = 0; e < E; e++) {
                    z[e] = make_float2(fmaf(al, w[e].x, z[e].x), fmaf(al, w[e].y, z[e].y));
                    u[e] = cscale(z[e], cost_coef(COST, z[e], yt[ttid + e * NT], fpart));
                }
                adj(u);
                park(u);
                __syncthreads();
                // G: new gradient, new pair, batched dot products
                {
                    float pv[32];
#pragma unroll
                    for (int k = 0; k < 32; k++) pv[k] = 0.f;
                    for (int e = 0; e < EPT; e++) {
                        const int i = tid + e * BT;
                        const bool in = i < N;
                        float2 gn = make_float2(0.f, 0.f), sn = gn, yn = gn;
                        if (in) {
                            gn = team_sum(i, gsc);
                            sn = cscale(X[i], al);
                            yn = csub(gn, gs[i]);
                            ts[i] = cadd(ts[i], sn);
                            gs[i] = gn;
                        }
                        tmem_st4(tcol(sn_slot, e), sn.x, sn.y, yn.x, yn.y);
#pragma unroll
                        for (int k = 0; k < kSlots; k++) {
                            if (k < np) {  // live pairs by age
                                uint32_t r[4];
                                tmem_ld4(tcol(so[k], e), r);
                                tmem_wait_ld();
                                tmem_reg_ready(r);
                                const float2 sa = make_float2(__uint_as_float(r[0]), __uint_as_float(r[1]));
                                const float2 ya = make_float2(__uint_as_float(r[2]), __uint_as_float(r[3]));
                                pv[4 * k + 0] += cdotr(sa, yn);
                                pv[4 * k + 1] += cdotr(ya, yn);
                                pv[4 * k + 2] += cdotr(sa, gn);
                                pv[4 * k + 3] += cdotr(ya, gn);
                            } else if (k == np) {  // the new pair (age np)
                                pv[4 * k + 0] += cdotr(sn, yn);
                                pv[4 * k + 1] += cdotr(yn, yn);
                                pv[4 * k + 2] += cdotr(sn, gn);
                                pv[4 * k + 3] += cdotr(yn, gn);
                            }
                        }
                        pv[kIdxSS] += cabs2(sn);
                        pv[kIdxGG] += cabs2(gn);
                    }
                    tmem_wait_st();  // the new pair is read back from the next iteration on
                    tmem_fence_before_sync();
                    pv[kIdxF] = fpart;
                    block_reduce(pv, kParts, false);
                    if (warp == 0) lbfgs_gram_update(Gm, lane, m, it, P.iters, P.tol);
                    __syncthreads();
                }
            }
        }

        // ---- outputs (rows decided before initialisation come back as zero) ----
        const bool early = Gm.early != 0;
        const float tsc = Gm.tsc;
        for (int i = tid; i < N; i += BT)
            P.T_out[(size_t)row * N + i] = early ? make_float2(0.f, 0.f) : cscale(ts[i], tsc);
        if (tid == 0) {
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
                const int pat = team * N + ttid + e * NT;
                if (pat < P.Nd) P.Zd[(size_t)pat * M + row] = early ? make_float2(0.f, 0.f) : cscale(z[e], tsc);
            }
        }
        __syncthreads();
    }
    tmem_fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tmem_fence_after_sync();
        tmem_dealloc_warp(tmem_base, (uint32_t)ncols);
    }
}

// Shared memory and resident CTAs per SM of a launch.  Every CTA holds
// row_tmem_cols columns of the SM's 512 for its whole life, so at most
// 512 / cols CTAs may share an SM; where registers and shared memory would
// let more in, the shared-memory request is raised until they do not, and no
// allocation has to wait for the columns of another CTA of the same launch.
// (A concurrent launch on another stream that holds tensor memory can delay
// an allocation until its CTAs on that SM exit; they never wait on this one.)
template <int N, int COST>
cudaError_t row_launch_shape(int J, int m, int klz, size_t *smem_out, int *per_sm_out)
{
    const int BT = J * RowCfg<N>::NT;
    const int cap = 512 / row_tmem_cols(N, J, m, klz);
    size_t sm = row_smem<N>(J, m);
    int dev = 0, occ = 0, sm_per_mp = 0, optin = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sm_per_mp, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
        return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    for (int pass = 0; pass < 2; pass++) {
        if (sm > (size_t)optin) return cudaErrorInvalidConfiguration;
        if ((e = cudaFuncSetAttribute(k_solver_row<N, COST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=
            cudaSuccess)
            return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_solver_row<N, COST>, BT, sm)) != cudaSuccess)
            return e;
        if (occ < 1) return cudaErrorInvalidConfiguration;
        if (occ <= cap) break;
        if (pass == 1) return cudaErrorInvalidConfiguration;
        const size_t need = (size_t)sm_per_mp / (size_t)(cap + 1) + 1;
        if (need > sm) sm = (need + 15) & ~(size_t)15;
    }
    *smem_out = sm;
    *per_sm_out = occ;
    return cudaSuccess;
}

template <int N, int COST = COST_INTENSITY>
cudaError_t launch_solver_row_t(const SolverParams &p, cudaStream_t s, int *ctas_out)
{
    if (!row_variant_fits(N, p.J) || p.m < 1 || p.m > kMaxMem) return cudaErrorInvalidValue;
    const int BT = p.J * RowCfg<N>::NT;
    size_t sm = 0;
    int occ = 0, dev = 0, nsm = 0;
    const int klz = row_tmem_klz(N, p.J, p.lanczos && p.init == INIT_SPECTRAL && !p.T_init, p.power_iters);
    cudaError_t e = row_launch_shape<N, COST>(p.J, p.m, klz, &sm, &occ);
    if (e != cudaSuccess) return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    long long grid = (long long)occ * nsm;
    if (grid > p.M) grid = p.M;
    if (grid > p.pair_ctas) grid = p.pair_ctas;  // the resident CTAs the handle sized its workspaces for
    if (p.lanczos && p.init == INIT_SPECTRAL && grid > p.krylov_units) grid = p.krylov_units;
    if (grid < 1) grid = 1;
    if (ctas_out) *ctas_out = (int)grid;
    k_solver_row<N, COST><<<(int)grid, BT, sm, s>>>(p);
    return cudaGetLastError();
}

}  // namespace tmr
