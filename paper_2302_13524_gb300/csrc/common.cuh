// common.cuh -- complex helpers and block reductions shared by the libtmr kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tmr {

constexpr int kMaxMasks = 8;  // J <= 8: one CTA per mask inside a portable cluster
constexpr int kMaxMem = 6;    // L-BFGS memory m <= 6: 4 (m + 1) + 3 reduced values fit one warp

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * b
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }
// Re(conj(a) b)
__host__ __device__ __forceinline__ float cdotr(float2 a, float2 b) { return fmaf(a.x, b.x, a.y * b.y); }

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum NV per-thread values over the block.  red: shared [NV][nwarps] scratch,
// out: shared [NV].  Partials are added warp by warp in a fixed order, so the
// result is deterministic.  Ends with a __syncthreads(); out is then visible
// to every thread.
template <int NV, typename TV>
__device__ __forceinline__ void block_sum(TV (&v)[NV], TV *red, TV *out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        TV s = warp_sum(v[k]);
        if (lane == 0) red[k * nw + warp] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NV; k += blockDim.x) {
        TV s = 0;
        for (int w = 0; w < nw; w++) s += red[k * nw + w];
        out[k] = s;
    }
    __syncthreads();
}

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the multiply/xor
// bijection on a 4-word counter with a 2-word key bumped by the Weyl
// constants between rounds.
__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
#ifdef __CUDA_ARCH__
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
#else
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Standard complex normal for element n of row `row` under `seed`: counter
// (n, row, 0, 0), key (seed lo, seed hi); words 0 and 1 as uniforms
// u = (x + 1/2) 2^-32, Box-Muller rho = sqrt(-2 ln u0), angle 2 pi u1.
__device__ __forceinline__ float2 philox_cnormal(unsigned long long seed, uint32_t row, uint32_t n)
{
    const uint4 o = philox4x32_10(make_uint4(n, row, 0u, 0u),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const float u0 = fmaf((float)o.x, 0x1p-32f, 0x1p-33f);  // (x + 1/2) 2^-32, rounded to FP32
    const float u1 = fmaf((float)o.y, 0x1p-32f, 0x1p-33f);
    const float rho = sqrtf(-2.0f * logf(u0));
    float s, c;
    sincospif(2.0f * u1, &s, &c);
    return make_float2(rho * c, rho * s);
}

}  // namespace tmr
