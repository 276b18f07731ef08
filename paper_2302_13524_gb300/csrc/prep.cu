// prep.cu -- camera preprocessing before the per-row solves (Sec. 2.2, the
// procedure that follows Algorithm 1): half-sampling of the K probe images,
// the fiber mask whose one-region holds a given fraction of the summed
// intensity, and the pixel-major rows y[M][K] the solver reads.
//
// Four launches on the caller's stream:
//   k_prep_rows    frames [K][H][W] -> y[M][K] for every kept pixel, plus one
//                  energy partial per (frame chunk, pixel); HBM-bound
//                  (reads the kept camera rows once, writes y once)
//   k_prep_energy  E[p] = the partials of pixel p summed in chunk order
//   k_prep_select  one CTA: the threshold tau = the c-th largest energy, found
//                  by a bitwise search on the energy keys; mask and count
//   k_prep_zero    rows outside the mask set to zero (write-only)
// Every sum runs in a fixed order, so repeated calls agree bitwise; uint16
// frames are summed exactly in 64-bit integers, float32 frames in FP64.
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "tmr.h"

namespace {

constexpr int kTile = 32;    // pixels (and frames) per transpose tile
constexpr int kTy = 8;       // threadIdx.y extent of k_prep_rows
constexpr int kChunk = 256;  // frames per CTA of k_prep_rows (one energy partial each)
constexpr int kSelThreads = 1024;

tmr_status fail(tmr_status st, const char *msg)
{
    tmr::set_last_error(msg);
    return st;
}

bool device_ptr(const void *p) { return tmr::is_device_ptr(p); }

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Pixel types: value as float, and the accumulator of its energy.
template <class PT>
struct Pix;
template <>
struct Pix<uint16_t> {
    using Acc = unsigned long long;  // exact: K * 65535 < 2^64 for any K < 2^31
    static __device__ __forceinline__ float f(uint16_t v) { return (float)v; }
    static __device__ __forceinline__ Acc acc(uint16_t v) { return v; }
    static __device__ __forceinline__ unsigned long long bits(Acc a) { return a; }
};
template <>
struct Pix<float> {
    using Acc = double;
    static __device__ __forceinline__ float f(float v) { return v; }
    static __device__ __forceinline__ Acc acc(float v) { return (double)v; }
    static __device__ __forceinline__ unsigned long long bits(Acc a)
    {
        return (unsigned long long)__double_as_longlong(a);
    }
};

// Grid (ceil(M / 32), ceil(K / kChunk)), block (32, 8).  A CTA moves a tile of
// 32 pixels x kChunk frames through shared memory: warp reads run along a
// kept camera row, warp writes along a row of y (32 consecutive frames).
template <class PT>
__global__ void __launch_bounds__(kTile *kTy) k_prep_rows(const PT *__restrict__ frames, int K, int H,
                                                           int W, int off, int nx, int M,
                                                           float *__restrict__ y,
                                                           unsigned long long *__restrict__ part)
{
    using Acc = typename Pix<PT>::Acc;
    __shared__ float tile[kTile][kTile + 1];
    __shared__ Acc red[kTy][kTile];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int p0 = blockIdx.x * kTile;
    const int c = blockIdx.y;
    const int k_begin = c * kChunk;
    const int k_end = min(K, k_begin + kChunk);
    const int p = p0 + tx;
    const bool live = p < M;
    size_t src = 0;
    if (live) {
        const int a = p / nx, b = p - a * nx;
        src = (size_t)(2 * a + off) * W + (size_t)(2 * b + off);
    }
    const size_t frame = (size_t)H * W;
    constexpr int kPer = kTile / kTy;
    auto load = [&](PT (&r)[kPer], int k0) {
#pragma unroll
        for (int i = 0; i < kPer; i++) {
            const int k = k0 + ty + i * kTy;
            r[i] = (live && k < k_end) ? frames[(size_t)k * frame + src] : PT(0);
        }
    };
    Acc acc = 0;
    PT raw[kPer];
    load(raw, k_begin);
    for (int k0 = k_begin; k0 < k_end; k0 += kTile) {
        PT nxt[kPer];  // the next tile's loads are in flight during this one's stores
        load(nxt, k0 + kTile);
#pragma unroll
        for (int i = 0; i < kPer; i++) {
            acc += Pix<PT>::acc(raw[i]);
            tile[ty + i * kTy][tx] = Pix<PT>::f(raw[i]);
        }
        __syncthreads();
        const int k = k0 + tx;
#pragma unroll
        for (int i = 0; i < kTile / kTy; i++) {
            const int j = ty + i * kTy;
            if (p0 + j < M && k < k_end) y[(size_t)(p0 + j) * K + k] = tile[tx][j];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kPer; i++) raw[i] = nxt[i];
    }
    red[ty][tx] = acc;
    __syncthreads();
    if (ty == 0 && live) {
        Acc s = red[0][tx];
#pragma unroll
        for (int r = 1; r < kTy; r++) s += red[r][tx];
        part[(size_t)c * M + p] = Pix<PT>::bits(s);
    }
}

// E[p] = partials summed in chunk order.  Keys: the uint64 sum (integer
// frames) or the bits of the non-negative FP64 sum (their integer order is
// the numeric order).  A negative or non-finite float sum sets *bad.
template <bool kInt>
__global__ void k_prep_energy(const unsigned long long *__restrict__ part, int C, int M,
                              unsigned long long *__restrict__ key, double *__restrict__ energy,
                              int *__restrict__ bad)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < M; p += gridDim.x * blockDim.x) {
        if constexpr (kInt) {
            unsigned long long s = 0;
            for (int c = 0; c < C; c++) s += part[(size_t)c * M + p];
            key[p] = s;
            if (energy) energy[p] = (double)s;
        } else {
            double s = 0.0;
            for (int c = 0; c < C; c++) s += __longlong_as_double((long long)part[(size_t)c * M + p]);
            s += 0.0;  // -0 -> +0
            if (!(s >= 0.0) || !isfinite(s)) {
                atomicOr(bad, 1);
                s = 0.0;
            }
            key[p] = (unsigned long long)__double_as_longlong(s);
            if (energy) energy[p] = s;
        }
    }
}

// Sum over the block of the energies whose key is >= lo, in a fixed order
// (each thread its strided pixels in turn, then warp and block trees).
// Integer energies are summed exactly and returned converted to FP64.
template <bool kInt>
__device__ double energy_at_or_above(const unsigned long long *__restrict__ key, int M,
                                     unsigned long long lo, double *red_d,
                                     unsigned long long *red_u)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double out;
    if constexpr (kInt) {
        unsigned long long s = 0;
        for (int p = threadIdx.x; p < M; p += blockDim.x) s += key[p] >= lo ? key[p] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red_u[warp] = s;
        __syncthreads();
        unsigned long long t = 0;
        for (int w = 0; w < nw; w++) t += red_u[w];
        out = (double)t;
    } else {
        double s = 0.0;
        for (int p = threadIdx.x; p < M; p += blockDim.x)
            s += key[p] >= lo ? __longlong_as_double((long long)key[p]) : 0.0;
        s = tmr::warp_sum(s);
        if (lane == 0) red_d[warp] = s;
        __syncthreads();
        if (warp == 0) {
            double t = lane < nw ? red_d[lane] : 0.0;
            t = tmr::warp_sum(t);
            if (lane == 0) red_d[32] = t;
        }
        __syncthreads();
        out = red_d[32];
    }
    __syncthreads();  // the scratch is reused by the next call
    return out;
}

// Integer energies: the threshold by 3-bit passes over the keys, from the
// top set bit down.  A pass fixes the next digit of tau: with the bits above
// already fixed (prefix), S(prefix | j << shift) for the eight digits j is
// the sum of the keys whose upper bits exceed the prefix's, plus the keys
// equal to it there whose digit is >= j; each thread accumulates all eight
// sums in registers (no shared-memory atomics, which serialise when most
// keys share their upper bits), the block adds them exactly, and the largest
// j whose S reaches the target is taken (compared in FP64).
__device__ unsigned long long select_tau_int(const unsigned long long *__restrict__ key, int M,
                                             double target, unsigned long long mx,
                                             unsigned long long (*red8)[8], unsigned long long *S8)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long prefix = 0;
    for (int top = 63 - __clzll(mx); top >= 0;) {
        const int shift = top >= 2 ? top - 2 : 0;
        const int nd = 1 << (top - shift + 1);
        const unsigned long long hi_mask = top >= 63 ? 0ull : (~0ull << (top + 1));
        unsigned long long acc[8];
#pragma unroll
        for (int j = 0; j < 8; j++) acc[j] = 0ull;
        for (int p = threadIdx.x; p < M; p += blockDim.x) {
            const unsigned long long k = key[p], kh = k & hi_mask;
            const int d = kh > prefix ? 7 : (kh == prefix ? (int)((k >> shift) & (unsigned long long)(nd - 1)) : -1);
#pragma unroll
            for (int j = 0; j < 8; j++) acc[j] += d >= j ? k : 0ull;
        }
#pragma unroll
        for (int j = 0; j < 8; j++) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < 8; j++) red8[warp][j] = acc[j];
        }
        __syncthreads();
        if (warp < 8) {  // warp j adds sum j over the warps
            unsigned long long v = lane < nw ? red8[lane][warp] : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) S8[warp] = v;
        }
        __syncthreads();
        int best = 0;  // digit 0 always reaches the target (S of the prefix itself)
        for (int j = 1; j < nd; j++)
            if ((double)S8[j] >= target) best = j;
        prefix |= (unsigned long long)best << shift;
        top = shift - 1;
        __syncthreads();  // S8 and red8 are rewritten by the next pass
    }
    return prefix;
}

// One CTA.  S(tau) = sum of the energies >= tau falls as tau grows; the mask
// threshold is the largest key tau with S(tau) >= frac * S(0), built from the
// top bit down (integer keys: 3 bits a pass; FP64 keys: one bit a pass, each
// a fixed-order FP64 block sum).  That tau is the c-th largest energy for the smallest
// brightest-first count c reaching the fraction, and E >= tau includes its ties.
template <bool kInt>
__global__ void __launch_bounds__(kSelThreads) k_prep_select(const unsigned long long *__restrict__ key,
                                                             int M, double frac,
                                                             const int *__restrict__ bad,
                                                             unsigned char *__restrict__ mask_ws,
                                                             unsigned char *__restrict__ mask,
                                                             int *__restrict__ n_inside)
{
    __shared__ double red_d[kSelThreads / 32 + 1];
    __shared__ unsigned long long red_u[kSelThreads / 32];
    __shared__ int cnt[kSelThreads / 32];
    __shared__ unsigned long long red8[kSelThreads / 32][8];
    __shared__ unsigned long long S8[8];
    const bool invalid = *bad != 0;
    unsigned long long tau = ~0ull;  // above every key: empty mask
    if (!invalid) {
        const double total = energy_at_or_above<kInt>(key, M, 0ull, red_d, red_u);
        if (total > 0.0) {
            const double target = frac * total;
            unsigned long long mx = 0;
            for (int p = threadIdx.x; p < M; p += blockDim.x) mx = key[p] > mx ? key[p] : mx;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
                mx = v > mx ? v : mx;
            }
            if ((threadIdx.x & 31) == 0) red_u[threadIdx.x >> 5] = mx;
            __syncthreads();
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) mx = red_u[w] > mx ? red_u[w] : mx;
            __syncthreads();
            if constexpr (kInt) {
                tau = select_tau_int(key, M, target, mx, red8, S8);
            } else {
                unsigned long long t = 0;
                for (int bit = 63 - __clzll(mx); bit >= 0; bit--) {
                    const unsigned long long cand = t | (1ull << bit);
                    if (energy_at_or_above<kInt>(key, M, cand, red_d, red_u) >= target) t = cand;
                }
                tau = t;
            }
        }
    }
    int n = 0;
    for (int p = threadIdx.x; p < M; p += blockDim.x) {
        const unsigned char in = key[p] >= tau ? 1 : 0;
        mask_ws[p] = in;
        if (mask) mask[p] = in;
        n += in;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0) cnt[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0 && n_inside) {
        int s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += cnt[w];
        *n_inside = invalid ? -1 : s;
    }
}

// One CTA per pixel row: zero the rows outside the mask.
__global__ void k_prep_zero(const unsigned char *__restrict__ mask_ws, int K, float *__restrict__ y)
{
    const size_t p = blockIdx.x;
    if (mask_ws[p]) return;
    float *row = y + p * (size_t)K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) row[k] = 0.f;
}

// out[i][p] = frame i at camera pixel (2a + off, 2b + off), p = a * nx + b.
template <class PT>
__global__ void k_half_sample(const PT *__restrict__ frames, int n, int H, int W, int off, int nx,
                              int M, float *__restrict__ out)
{
    const size_t total = (size_t)n * M;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t i = e / M;
        const int p = (int)(e - i * M);
        const int a = p / nx, b = p - a * nx;
        out[e] = Pix<PT>::f(frames[(i * H + (size_t)(2 * a + off)) * W + (size_t)(2 * b + off)]);
    }
}

struct PrepLayout {
    int ny, nx, M, C;
    size_t part, key, mask, bad, total;
};

bool prep_layout(int K, int H, int W, int offset, PrepLayout *L)
{
    if (K < 1 || H < 1 || W < 1 || (offset != 0 && offset != 1)) return false;
    L->ny = (H - offset + 1) / 2;
    L->nx = (W - offset + 1) / 2;
    if (L->ny < 1 || L->nx < 1) return false;
    const long long M = (long long)L->ny * L->nx;
    if (M > 0x7fffffffLL) return false;
    L->M = (int)M;
    L->C = (K + kChunk - 1) / kChunk;
    L->part = 0;
    L->key = align256(L->part + sizeof(unsigned long long) * (size_t)L->C * L->M);
    L->mask = align256(L->key + sizeof(unsigned long long) * (size_t)L->M);
    L->bad = align256(L->mask + (size_t)L->M);
    L->total = align256(L->bad + sizeof(int));
    return true;
}

template <class PT>
cudaError_t launch_prep(const PT *frames, int K, int H, int W, int off, double frac, const PrepLayout &L,
                        char *ws, float *y, unsigned char *mask, double *energy, int *n_inside,
                        cudaStream_t s)
{
    constexpr bool kInt = std::is_same<PT, uint16_t>::value;
    auto *part = (unsigned long long *)(ws + L.part);
    auto *key = (unsigned long long *)(ws + L.key);
    auto *mask_ws = (unsigned char *)(ws + L.mask);
    int *bad = (int *)(ws + L.bad);
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_prep_rows<PT><<<dim3((L.M + kTile - 1) / kTile, L.C), dim3(kTile, kTy), 0, s>>>(
        frames, K, H, W, off, L.nx, L.M, y, part);
    const int eb = 256, eg = (int)std::min<long long>((L.M + eb - 1) / eb, 152LL * 8);
    k_prep_energy<kInt><<<eg, eb, 0, s>>>(part, L.C, L.M, key, energy, bad);
    k_prep_select<kInt><<<1, kSelThreads, 0, s>>>(key, L.M, frac, bad, mask_ws, mask, n_inside);
    k_prep_zero<<<L.M, 256, 0, s>>>(mask_ws, K, y);
    return cudaGetLastError();
}

}  // namespace

extern "C" size_t tmr_preprocess_workspace_bytes(int K, int H, int W, int offset)
{
    PrepLayout L;
    return prep_layout(K, H, W, offset, &L) ? L.total : 0;
}

extern "C" tmr_status tmr_preprocess(const void *frames, int pixel_type, int K, int H, int W,
                                     int offset, double energy_frac, float *y, unsigned char *mask,
                                     double *energy, int *n_inside, void *workspace,
                                     size_t workspace_bytes, void *stream)
{
    PrepLayout L;
    if (!prep_layout(K, H, W, offset, &L))
        return fail(TMR_ERR_INVALID_ARG, "tmr_preprocess: need K, H, W >= 1, offset 0 or 1, a non-empty half grid");
    if (pixel_type != TMR_PIX_U16 && pixel_type != TMR_PIX_F32)
        return fail(TMR_ERR_INVALID_ARG, "tmr_preprocess: pixel_type must be TMR_PIX_U16 or TMR_PIX_F32");
    if (!(energy_frac > 0.0 && energy_frac <= 1.0))
        return fail(TMR_ERR_INVALID_ARG, "tmr_preprocess: energy_frac must be in (0, 1]");
    if (L.C > 65535) return fail(TMR_ERR_INVALID_ARG, "tmr_preprocess: K above 65535 * 256 frames");
    if (!frames || !y || !workspace) return fail(TMR_ERR_INVALID_ARG, "tmr_preprocess: NULL frames, y or workspace");
    if (workspace_bytes < L.total) return fail(TMR_ERR_INVALID_ARG, "tmr_preprocess: workspace smaller than tmr_preprocess_workspace_bytes");
    if (!device_ptr(frames) || !device_ptr(y) || !device_ptr(workspace) || (mask && !device_ptr(mask)) ||
        (energy && !device_ptr(energy)) || (n_inside && !device_ptr(n_inside)))
        return fail(TMR_ERR_INVALID_ARG, "tmr_preprocess: every array must be device memory");
    const cudaStream_t s = (cudaStream_t)stream;
    const cudaError_t e =
        pixel_type == TMR_PIX_U16
            ? launch_prep((const uint16_t *)frames, K, H, W, offset, energy_frac, L, (char *)workspace, y,
                          mask, energy, n_inside, s)
            : launch_prep((const float *)frames, K, H, W, offset, energy_frac, L, (char *)workspace, y, mask,
                          energy, n_inside, s);
    if (e != cudaSuccess) return fail(TMR_ERR_CUDA, cudaGetErrorString(e));
    return TMR_OK;
}

extern "C" tmr_status tmr_half_sample(const void *frames, int pixel_type, int n, int H, int W, int offset,
                                      float *out, void *stream)
{
    PrepLayout L;
    if (!prep_layout(n, H, W, offset, &L))
        return fail(TMR_ERR_INVALID_ARG, "tmr_half_sample: need n, H, W >= 1, offset 0 or 1, a non-empty half grid");
    if (pixel_type != TMR_PIX_U16 && pixel_type != TMR_PIX_F32)
        return fail(TMR_ERR_INVALID_ARG, "tmr_half_sample: pixel_type must be TMR_PIX_U16 or TMR_PIX_F32");
    if (!frames || !out) return fail(TMR_ERR_INVALID_ARG, "tmr_half_sample: NULL frames or out");
    if (!device_ptr(frames) || !device_ptr(out))
        return fail(TMR_ERR_INVALID_ARG, "tmr_half_sample: frames and out must be device memory");
    const cudaStream_t s = (cudaStream_t)stream;
    const size_t total = (size_t)n * L.M;
    const int b = 256;
    const int g = (int)std::min<size_t>((total + b - 1) / b, 152 * 16);
    if (pixel_type == TMR_PIX_U16)
        k_half_sample<<<g, b, 0, s>>>((const uint16_t *)frames, n, H, W, offset, L.nx, L.M, out);
    else
        k_half_sample<<<g, b, 0, s>>>((const float *)frames, n, H, W, offset, L.nx, L.M, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TMR_ERR_CUDA, cudaGetErrorString(e));
    return TMR_OK;
}
