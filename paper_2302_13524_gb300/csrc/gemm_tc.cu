// gemm_tc.cu -- BF16 x BF16 -> FP32 GEMM on the fifth-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory), fed by TMA.  It computes the
// products of the learned initialiser's network (mlp.cu) where the shapes
// allow (row lengths a multiple of 8 elements, 16-byte aligned rows).
//
//   C[M][N] (FP32, row stride ldc) = A B^T,  A [M][K] and B [N][K] BF16, both
//   K-contiguous (row strides lda, ldb elements).
//
// One CTA computes one 128 x BN tile of C (BN = 128) with 4 warps:
//   warp 0, one lane: TMA producer.  Each k-step of 64 elements loads a
//     128 x 64 tile of A and a BN x 64 tile of B (128-byte rows, 128-byte
//     swizzle) into one of kStages shared-memory stages, arriving on the
//     stage's "full" mbarrier with the transferred byte count;
//   warp 1, one lane: MMA issuer.  Per k-step, four tcgen05.mma of
//     M = 128, N = BN, K = 16 (kind::f16, BF16 operands, FP32 accumulator in
//     BN tensor-memory columns), then tcgen05.commit onto the stage's
//     "empty" mbarrier, which hands the stage back to the producer when the
//     MMAs that read it are done; after the last k-step a commit onto the
//     "done" mbarrier;
//   all 4 warps: epilogue.  Warp w reads tensor-memory lanes 32w .. 32w + 31
//     (rows of the tile) with tcgen05.ld, 32 columns at a time, and stores
//     the FP32 values to C with bounds checks.
// Tensor memory (BN columns) is allocated and freed by warp 0.  Out-of-range
// rows and the K tail are zero-filled by TMA.  Every mbarrier wait is
// bounded: after kSpinLimit polls the waiting thread raises *err and the CTA
// stops issuing work, waits (bounded again) for the MMAs it issued, frees its
// tensor memory and returns; the caller reads the flag.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "internal.h"
#include "tmr.h"

namespace tmr {

namespace {

constexpr int kBM = 128, kBN = 128, kBK = 64, kStages = 4;
constexpr int kTileA = kBM * kBK * 2;  // bytes per stage
constexpr int kTileB = kBN * kBK * 2;
constexpr long long kSpinLimit = 1LL << 22;  // polls of a barrier wait (about 0.1 - 1 s)
constexpr size_t kSmem = 1024 /*alignment slack*/ + (size_t)kStages * (kTileA + kTileB) + 256;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Wait until the phase with parity `parity` of the barrier has completed, at
// most kSpinLimit polls (test_wait does not block; after the first 1024 polls
// each one is followed by a 64 ns sleep); false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (long long i = 0; i < kSpinLimit; i++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (i >= 1024) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte rows in the
// 128-byte swizzle layout: 8-row groups 1024 bytes apart (stride byte offset),
// descriptor version 1, swizzle mode 2 (128 B).  The leading byte offset is
// not used by this layout (set to 16 bytes).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;              // leading byte offset >> 4
    d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset >> 4
    d |= (uint64_t)1 << 46;              // version
    d |= (uint64_t)2 << 61;              // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = kBN, M = kBM.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__global__ void __launch_bounds__(128, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N,
              int K, float *__restrict__ C, int ldc, int *err)
{
    extern __shared__ unsigned char smem_raw[];
    // tiles need 1024-byte alignment for the 128-byte swizzle
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = base;
    unsigned char *sB = base + (size_t)kStages * kTileA;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sB + (size_t)kStages * kTileB);  // full[S], empty[S], done
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * kStages + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int ktiles = (K + kBK - 1) / kBK;
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kStages), done = smem_u32(bars + 2 * kStages);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {  // tensor memory for the accumulator: kBN columns x 128 lanes
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kBN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    int issued_loads = 0;  // producer: k-steps whose loads were issued
    if (warp == 0 && lane == 0) {
        // producer
        for (int kt = 0; kt < ktiles && !*abort_flag; kt++) {
            const int s = kt % kStages;
            if (kt >= kStages && !mbar_wait(empty0 + 8 * s, ((kt / kStages) - 1) & 1)) {
                atomicExch(err, 1);
                *abort_flag = 1;
                break;
            }
            const uint32_t fb = full0 + 8 * s;
            mbar_expect_tx(fb, kTileA + kTileB);
            tma_load_2d(smem_u32(sA + (size_t)s * kTileA), &mapA, kt * kBK, m0, fb);
            tma_load_2d(smem_u32(sB + (size_t)s * kTileB), &mapB, kt * kBK, n0, fb);
            issued_loads = kt + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        for (int kt = 0; kt < ktiles && !*abort_flag; kt++) {
            const int s = kt % kStages;
            if (!mbar_wait(full0 + 8 * s, (kt / kStages) & 1)) {
                atomicExch(err, 1);
                *abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t da = sw128_desc(smem_u32(sA + (size_t)s * kTileA));
            const uint64_t db = sw128_desc(smem_u32(sB + (size_t)s * kTileB));
#pragma unroll
            for (int k = 0; k < kBK / 16; k++)  // K = 16 per MMA: 32 bytes further along the row
                umma_f16(tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), kIdesc, (kt > 0 || k > 0) ? 1u : 0u);
            umma_commit(empty0 + 8 * s);
        }
        umma_commit(done);  // arrives when every MMA issued above has completed
    }
    // epilogue: every warp, its 32 lanes of tensor memory
    __syncwarp();
    const bool ok = mbar_wait(done, 0);
    if (!ok && lane == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && !*abort_flag) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < kBN; c0 += 32) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
                float *crow = C + (size_t)row * ldc + n0 + c0;
                const int nleft = N - (n0 + c0);
                if (nleft >= 32 && (((uintptr_t)crow) & 15) == 0) {
#pragma unroll
                    for (int q = 0; q < 8; q++)
                        reinterpret_cast<float4 *>(crow)[q] =
                            make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                        __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
                } else {
#pragma unroll
                    for (int q = 0; q < 32; q++)
                        if (q < nleft) crow[q] = __uint_as_float(v[q]);
                }
            }
        }
    }
    if (warp == 0 && lane == 0 && *abort_flag) {
        // an aborted tile: let the last loads issued into each stage land
        // (bounded) before the CTA's shared memory goes away
        for (int kt = issued_loads - kStages > 0 ? issued_loads - kStages : 0; kt < issued_loads; kt++)
            mbar_wait(full0 + 8 * (kt % kStages), (kt / kStages) & 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kBN) : "memory");
    }
}

// ---- host: tensor maps through the driver entry point (no -lcuda) ----------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// rows x cols BF16 matrix with row stride ld (elements); box of box_rows x 64
bool make_map(CUtensorMap *map, const __nv_bfloat16 *ptr, int rows, int cols, int ld, int box_rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool gemm_tc_supported(int M, int N, int K, const void *A, int lda, const void *B, int ldb)
{
    // whole boxes inside the matrices in every dimension but the tails
    if (M < kBM || N < kBN || K < kBK) return false;
    if (K % 8 || lda % 8 || ldb % 8 || lda < K || ldb < K) return false;  // 16-byte rows and strides
    if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15)) return false;
    return encode_fn() != nullptr;
}

cudaError_t gemm_tc(int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb,
                    float *C, int ldc, int *err, cudaStream_t s)
{
    if (!gemm_tc_supported(M, N, K, A, lda, B, ldb) || !err) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, M, K, lda, kBM) || !make_map(&mb, B, N, K, ldb, kBN)) return cudaErrorInvalidValue;
    const cudaError_t attr = cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (attr != cudaSuccess) return attr;
    dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM);
    k_gemm_tc<<<grid, 128, kSmem, s>>>(ma, mb, M, N, K, C, ldc, err);
    return cudaGetLastError();
}

}  // namespace tmr

extern "C" tmr_status tmr_gemm_bf16(int M, int N, int K, const void *A, int lda, const void *B, int ldb, float *C,
                                    int ldc, void *stream)
{
    tmr::set_last_error("");
    if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0 || ldc < N) {
        tmr::set_last_error("tmr_gemm_bf16: bad argument");
        return TMR_ERR_INVALID_ARG;
    }
    if (!tmr::is_device_ptr(A) || !tmr::is_device_ptr(B) || !tmr::is_device_ptr(C)) {
        tmr::set_last_error("tmr_gemm_bf16: A, B and C must be device memory of the current device");
        return TMR_ERR_INVALID_ARG;
    }
    if (!tmr::gemm_tc_supported(M, N, K, A, lda, B, ldb)) {
        tmr::set_last_error("tmr_gemm_bf16: needs M, N >= 128, K >= 64, K, lda, ldb multiples of 8, 16-byte alignment");
        return TMR_ERR_UNSUPPORTED;
    }
    int *err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        tmr::set_last_error("tmr_gemm_bf16: error flag");
        return TMR_ERR_OOM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int herr = 0;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess)
        e = tmr::gemm_tc(M, N, K, (const __nv_bfloat16 *)A, lda, (const __nv_bfloat16 *)B, ldb, C, ldc, err, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(err);
    if (e != cudaSuccess) {
        cudaGetLastError();
        tmr::set_last_error(cudaGetErrorString(e));
        return TMR_ERR_CUDA;
    }
    if (herr) {
        tmr::set_last_error("tmr_gemm_bf16: a barrier wait ran out");
        return TMR_ERR_TIMEOUT;
    }
    return TMR_OK;
}
