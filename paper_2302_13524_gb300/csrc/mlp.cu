// mlp.cu -- the learned initialiser's network: a three-layer perceptron
// x -> GELU(W1 x + b1) -> GELU(W2 h1 + b2) -> W3 h2 + b3, trained and run on
// the GPU by the kernels of this file.
//
// Weights are kept as FP32 master copies (updated by Adam) and as BF16 copies
// that feed the products; activations enter the products in BF16; every
// product accumulates in FP32 (mma.sync m16n8k16 BF16 tensor-core steps).  The
// loss is the mean squared error over every output, or its phase-invariant
// form (each target row rotated onto the output row first).  One GEMM kernel serves
// the forward products X W^T, the input gradients dZ W and the weight
// gradients dZ^T H through generic element strides.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "common.cuh"
#include "internal.h"
#include "tmr.h"

namespace tmr {

// C[M][N] (row-major, FP32) = sum_k A(m, k) B(k, n) with A(m, k) = A[m sam + k sak] and
// B(k, n) = B[k sbk + n sbn] in BF16.  64 x 64 tile per CTA, 4 warps of 32 x 32,
// K in steps of 32 through shared memory; out-of-range elements read as zero.
constexpr int GB_M = 64, GB_N = 64, GB_K = 32, GB_PAD = 8;

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__global__ void __launch_bounds__(128) k_gemm_bf16(int M, int N, int K, const __nv_bfloat16 *__restrict__ A,
                                                  long long sam, long long sak,
                                                  const __nv_bfloat16 *__restrict__ B, long long sbk,
                                                  long long sbn, float *__restrict__ C, int ldc)
{
    __shared__ __nv_bfloat16 As[GB_M][GB_K + GB_PAD];
    __shared__ __nv_bfloat16 Bs[GB_N][GB_K + GB_PAD];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int gid = lane >> 2, tig = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[i][j][q] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < K; k0 += GB_K) {
        // A tile: walk along whichever index is contiguous in memory
        for (int e = tid; e < GB_M * GB_K; e += 128) {
            int m, k;
            if (sak == 1) { m = e / GB_K; k = e % GB_K; }
            else { k = e / GB_M; m = e % GB_M; }
            const int gm = m0 + m, gk = k0 + k;
            As[m][k] = (gm < M && gk < K) ? A[gm * sam + gk * sak] : zero;
        }
        for (int e = tid; e < GB_N * GB_K; e += 128) {
            int n, k;
            if (sbk == 1) { n = e / GB_K; k = e % GB_K; }
            else { k = e / GB_N; n = e % GB_N; }
            const int gn = n0 + n, gk = k0 + k;
            Bs[n][k] = (gn < N && gk < K) ? B[gk * sbk + gn * sbn] : zero;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; kk += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; i++) {
                const int r = wm + i * 16 + gid, c = kk + tig * 2;
                af[i][0] = pack_bf16(As[r][c], As[r][c + 1]);
                af[i][1] = pack_bf16(As[r + 8][c], As[r + 8][c + 1]);
                af[i][2] = pack_bf16(As[r][c + 8], As[r][c + 9]);
                af[i][3] = pack_bf16(As[r + 8][c + 8], As[r + 8][c + 9]);
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int n = wn + j * 8 + gid, c = kk + tig * 2;
                bfr[j][0] = pack_bf16(Bs[n][c], Bs[n][c + 1]);
                bfr[j][1] = pack_bf16(Bs[n][c + 8], Bs[n][c + 9]);
            }
#pragma unroll
            for (int i = 0; i < 2; i++)
#pragma unroll
                for (int j = 0; j < 4; j++)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                        "{%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                        : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bfr[j][0]),
                          "r"(bfr[j][1]));
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int r = m0 + wm + i * 16 + gid, c = n0 + wn + j * 8 + tig * 2;
            if (r < M && c < N) C[(size_t)r * ldc + c] = acc[i][j][0];
            if (r < M && c + 1 < N) C[(size_t)r * ldc + c + 1] = acc[i][j][1];
            if (r + 8 < M && c < N) C[(size_t)(r + 8) * ldc + c] = acc[i][j][2];
            if (r + 8 < M && c + 1 < N) C[(size_t)(r + 8) * ldc + c + 1] = acc[i][j][3];
        }
}

static void gemm_sync(int M, int N, int K, const __nv_bfloat16 *A, long long sam, long long sak,
                      const __nv_bfloat16 *B, long long sbk, long long sbn, float *C, cudaStream_t s)
{
    dim3 grid((N + GB_N - 1) / GB_N, (M + GB_M - 1) / GB_M);
    k_gemm_bf16<<<grid, 128, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, N);
}

// out[c][r] = in[r][c] for an rows x cols BF16 matrix (row strides ldi, ldo);
// 32 x 32 tiles through shared memory, block (32, 8)
__global__ void k_transpose_bf16(int rows, int cols, const __nv_bfloat16 *__restrict__ in, long long ldi,
                                 __nv_bfloat16 *__restrict__ out, long long ldo)
{
    __shared__ __nv_bfloat16 t[32][34];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int r = r0 + j, c = c0 + threadIdx.x;
        t[j][threadIdx.x] = (r < rows && c < cols) ? in[(size_t)r * ldi + c] : __float2bfloat16(0.f);
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int c = c0 + j, r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[(size_t)c * ldo + r] = t[threadIdx.x][j];
    }
}

static void transpose_bf16(int rows, int cols, const __nv_bfloat16 *in, long long ldi, __nv_bfloat16 *out,
                           cudaStream_t s)
{
    dim3 grid((cols + 31) / 32, (rows + 31) / 32);
    k_transpose_bf16<<<grid, dim3(32, 8), 0, s>>>(rows, cols, in, ldi, out, rows);
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x)
{
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// Z += b (per column); H = GELU(Z) in BF16 (gelu != 0) or Z itself copied to out.
__global__ void k_bias_act(int B, int N, float *Z, const float *b, __nv_bfloat16 *H, int gelu)
{
    const size_t total = (size_t)B * N;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const float z = Z[i] + b[i % N];
        Z[i] = z;
        if (H) H[i] = __float2bfloat16(gelu ? gelu_f(z) : z);
    }
}

// dY = 2 (Y - T) / (B n); per-block partial sums of (Y - T)^2 into part
__global__ void k_mse(int B, int N, const float *Y, const float *T, __nv_bfloat16 *dY, float *part)
{
    const size_t total = (size_t)B * N;
    const float sc = 2.f / (float)total;
    float acc = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const float e = Y[i] - T[i];
        acc = fmaf(e, e, acc);
        dY[i] = __float2bfloat16(sc * e);
    }
    __shared__ float red[32], out[1];
    float v[1] = {acc};
    block_sum<1>(v, red, out);
    if (threadIdx.x == 0) part[blockIdx.x] = out[0];
}

// Phase-invariant loss: row r of T, read as t = T[:n] + i T[n:], rotated onto
// the output row y = Y[:n] + i Y[n:]: Ta = t conj(c) / |c|, c = sum conj(y) t
// (unrotated where c = 0).  One block per row; the sum in block_sum order.
__global__ void k_align_targets(int n, const float *Y, const float *T, float *Ta)
{
    const size_t o = (size_t)blockIdx.x * 2 * n;
    const float *y = Y + o, *t = T + o;
    float cr = 0.f, ci = 0.f;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const float yr = y[k], yi = y[n + k], tr = t[k], ti = t[n + k];
        cr = fmaf(yr, tr, fmaf(yi, ti, cr));
        ci = fmaf(yr, ti, fmaf(-yi, tr, ci));
    }
    __shared__ float red[64], res[2];
    float v[2] = {cr, ci};
    block_sum<2>(v, red, res);
    const float ac = sqrtf(res[0] * res[0] + res[1] * res[1]);
    const float rr = ac > 0.f ? res[0] / ac : 1.f, ri = ac > 0.f ? -res[1] / ac : 0.f;  // conj(c) / |c|
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const float tr = t[k], ti = t[n + k];
        Ta[o + k] = tr * rr - ti * ri;
        Ta[o + n + k] = tr * ri + ti * rr;
    }
}

__global__ void k_loss_finish(int nparts, const float *part, float total, float *loss)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nparts; i++) s += part[i];
        *loss = (float)(s / total);
    }
}

// dZ = dH .* GELU'(Z) -> BF16
__global__ void k_gelu_back(size_t n, const float *dH, const float *Z, __nv_bfloat16 *dZ)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dZ[i] = __float2bfloat16(dH[i] * gelu_grad_f(Z[i]));
}

// db[c] = sum_r dZ[r][c] (dZ BF16 [B][N])
__global__ void k_colsum(int B, int N, const __nv_bfloat16 *dZ, float *db)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    float s = 0.f;
    for (int r = 0; r < B; r++) s += __bfloat162float(dZ[(size_t)r * N + c]);
    db[c] = s;
}

__global__ void k_to_bf16(size_t n, const float *x, __nv_bfloat16 *y)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(x[i]);
}

__global__ void k_adam(size_t n, float *w, const float *g, float *m, float *v, __nv_bfloat16 *wb, float lr,
                       float c1, float c2)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = 0.9f * m[i] + 0.1f * gi;
        const float vi = 0.999f * v[i] + 0.001f * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
        w[i] = wi;
        wb[i] = __float2bfloat16(wi);
    }
}

// y = normalised sqrt intensities: x[r][i] = sqrt(max(y, 0)) / sqrt(mean_i y[r][i]) (BF16)
__global__ void k_features(int K, const float *y, __nv_bfloat16 *x)
{
    const int r = blockIdx.x;
    const float *yr = y + (size_t)r * K;
    float s = 0.f;
    for (int i = threadIdx.x; i < K; i += blockDim.x) s += fmaxf(yr[i], 0.f);
    __shared__ float red[32], out[1];
    float v[1] = {s};
    block_sum<1>(v, red, out);
    const float inv = out[0] > 0.f ? rsqrtf(out[0] / (float)K) : 0.f;
    for (int i = threadIdx.x; i < K; i += blockDim.x)
        x[(size_t)r * K + i] = __float2bfloat16(sqrtf(fmaxf(yr[i], 0.f)) * inv);
}

// candidate start: t[n] = (out[n] + i out[N + n]) scaled to ||t||^2 = sum(y) / (J N)
__global__ void k_candidate(int N, int K, const float *out, const float *y, float2 *T)
{
    const int r = blockIdx.x;
    const float *o = out + (size_t)r * 2 * N;
    const float *yr = y + (size_t)r * K;
    float sy = 0.f, sn = 0.f;
    for (int i = threadIdx.x; i < K; i += blockDim.x) sy += fmaxf(yr[i], 0.f);
    for (int n = threadIdx.x; n < N; n += blockDim.x) sn += o[n] * o[n] + o[N + n] * o[N + n];
    __shared__ float red[64], res[2];
    float v[2] = {sy, sn};
    block_sum<2>(v, red, res);
    const float sc = res[1] > 0.f ? sqrtf(res[0] / (float)K) / sqrtf(res[1]) : 0.f;
    for (int n = threadIdx.x; n < N; n += blockDim.x)
        T[(size_t)r * N + n] = make_float2(o[n] * sc, o[N + n] * sc);
}

}  // namespace tmr

using namespace tmr;

struct tmr_mlp {
    int n_in, h1, h2, n_out;
    size_t np;  // parameters
    size_t off[6];
    cudaStream_t stream;
    float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
    __nv_bfloat16 *wb = nullptr;
    long long step = 0;
    // batch scratch
    int cap = 0;
    __nv_bfloat16 *xb = nullptr, *h1b = nullptr, *h2b = nullptr, *dzb = nullptr, *dz2b = nullptr, *dyb = nullptr;
    float *z1 = nullptr, *z2 = nullptr, *y = nullptr, *dh = nullptr, *part = nullptr, *lossd = nullptr;
    float *ta = nullptr;  // aligned targets of the phase-invariant loss [B][out]
    int loss_kind = TMR_LOSS_MSE;
    // tensor-core GEMM: transposed-operand scratch and the barrier-timeout flag
    __nv_bfloat16 *tsa = nullptr, *tsb = nullptr;
    size_t tsa_cap = 0, tsb_cap = 0;
    int *tc_err = nullptr;
};

namespace {

tmr_status mfail(tmr_status st, const char *msg)
{
    set_last_error(msg);
    return st;
}

bool dev_ptr(const void *p) { return tmr::is_device_ptr(p); }

// C[M][N] = sum_k A(m, k) B(k, n), A(m, k) = A[m sam + k sak], B(k, n) = B[k sbk + n sbn]:
// on the tcgen05 tensor cores (gemm_tc.cu) when the shape allows, each operand
// first made K-contiguous (a transpose into the network's scratch when it is
// stored M- or N-contiguous); otherwise the mma.sync tile kernel above.
void gemm(tmr_mlp *m, int M, int N, int K, const __nv_bfloat16 *A, long long sam, long long sak,
          const __nv_bfloat16 *B, long long sbk, long long sbn, float *C)
{
    cudaStream_t s = m->stream;
    if (M >= 128 && N >= 128 && K >= 64 && K % 8 == 0 && m->tc_err) {
        const __nv_bfloat16 *At = A, *Bt = B;
        long long lda = sam, ldb = sbn;
        bool ok = true;
        if (sak != 1) {  // stored [K][M] (sam == 1): transpose to [M][K]
            ok = sam == 1 && (size_t)M * K <= m->tsa_cap;
            if (ok) {
                transpose_bf16(K, M, A, sak, m->tsa, s);
                At = m->tsa;
                lda = K;
            }
        }
        if (ok && sbk != 1) {  // stored [K][N] (sbn == 1): transpose to [N][K]
            ok = sbn == 1 && (size_t)N * K <= m->tsb_cap;
            if (ok) {
                transpose_bf16(K, N, B, sbk, m->tsb, s);
                Bt = m->tsb;
                ldb = K;
            }
        }
        if (ok && lda <= 0x7fffffff && ldb <= 0x7fffffff && gemm_tc_supported(M, N, K, At, (int)lda, Bt, (int)ldb) &&
            gemm_tc(M, N, K, At, (int)lda, Bt, (int)ldb, C, N, m->tc_err, s) == cudaSuccess)
            return;
        cudaGetLastError();
    }
    gemm_sync(M, N, K, A, sam, sak, B, sbk, sbn, C, s);
}

int ew_blocks(size_t n)
{
    size_t b = (n + 255) / 256;
    return (int)(b > 152 * 8 ? 152 * 8 : (b < 1 ? 1 : b));
}

tmr_status ensure_batch(tmr_mlp *m, int B)
{
    if (B <= m->cap) return TMR_OK;
    void **bufs[] = {(void **)&m->xb, (void **)&m->h1b, (void **)&m->h2b, (void **)&m->dzb, (void **)&m->dz2b,
                     (void **)&m->dyb, (void **)&m->z1, (void **)&m->z2, (void **)&m->y, (void **)&m->dh,
                     (void **)&m->ta, (void **)&m->tsa, (void **)&m->tsb};
    for (void **b : bufs)
        if (*b) {
            cudaFree(*b);
            *b = nullptr;
        }
    const size_t big = (size_t)B * (m->n_in > m->n_out ? m->n_in : m->n_out);
    const size_t hid = (size_t)B * (m->h1 > m->h2 ? m->h1 : m->h2);
    const size_t hmax = big > hid ? big : hid;
    bool ok = cudaMalloc(&m->xb, sizeof(__nv_bfloat16) * (size_t)B * m->n_in) == cudaSuccess &&
              cudaMalloc(&m->h1b, sizeof(__nv_bfloat16) * (size_t)B * m->h1) == cudaSuccess &&
              cudaMalloc(&m->h2b, sizeof(__nv_bfloat16) * (size_t)B * m->h2) == cudaSuccess &&
              cudaMalloc(&m->dzb, sizeof(__nv_bfloat16) * hmax) == cudaSuccess &&
              cudaMalloc(&m->dz2b, sizeof(__nv_bfloat16) * hmax) == cudaSuccess &&
              cudaMalloc(&m->dyb, sizeof(__nv_bfloat16) * (size_t)B * m->n_out) == cudaSuccess &&
              cudaMalloc(&m->z1, sizeof(float) * (size_t)B * m->h1) == cudaSuccess &&
              cudaMalloc(&m->z2, sizeof(float) * (size_t)B * m->h2) == cudaSuccess &&
              cudaMalloc(&m->y, sizeof(float) * (size_t)B * m->n_out) == cudaSuccess &&
              cudaMalloc(&m->dh, sizeof(float) * hmax) == cudaSuccess &&
              cudaMalloc(&m->ta, sizeof(float) * (size_t)B * m->n_out) == cudaSuccess;
    // transposed operands of the tensor-core GEMM: A sides [max(out, h1, h2)][B],
    // B sides W3^T, W2^T and [max(in, h1, h2)][B]
    const size_t hmx = (size_t)(m->h1 > m->h2 ? m->h1 : m->h2);
    const size_t amax = (size_t)B * ((size_t)m->n_out > hmx ? (size_t)m->n_out : hmx);
    size_t bmax = (size_t)m->h2 * m->n_out;
    if ((size_t)m->h1 * m->h2 > bmax) bmax = (size_t)m->h1 * m->h2;
    const size_t bb = (size_t)B * ((size_t)m->n_in > hmx ? (size_t)m->n_in : hmx);
    if (bb > bmax) bmax = bb;
    ok = ok && cudaMalloc(&m->tsa, sizeof(__nv_bfloat16) * amax) == cudaSuccess &&
         cudaMalloc(&m->tsb, sizeof(__nv_bfloat16) * bmax) == cudaSuccess;
    m->tsa_cap = ok ? amax : 0;
    m->tsb_cap = ok ? bmax : 0;
    if (!ok) {
        cudaGetLastError();
        return mfail(TMR_ERR_OOM, "MLP batch buffers");
    }
    m->cap = B;
    return TMR_OK;
}

// forward from BF16 features m->xb into m->y (FP32); keeps Z1, Z2, H1, H2
void forward_core(tmr_mlp *m, int B)
{
    cudaStream_t s = m->stream;
    const __nv_bfloat16 *W1 = m->wb + m->off[0], *W2 = m->wb + m->off[2], *W3 = m->wb + m->off[4];
    const float *b1 = m->w + m->off[1], *b2 = m->w + m->off[3], *b3 = m->w + m->off[5];
    // Z1 = X W1^T: A = X [B][n_in], B(k, n) = W1[n][k]
    gemm(m, B, m->h1, m->n_in, m->xb, m->n_in, 1, W1, 1, m->n_in, m->z1);
    k_bias_act<<<ew_blocks((size_t)B * m->h1), 256, 0, s>>>(B, m->h1, m->z1, b1, m->h1b, 1);
    gemm(m, B, m->h2, m->h1, m->h1b, m->h1, 1, W2, 1, m->h1, m->z2);
    k_bias_act<<<ew_blocks((size_t)B * m->h2), 256, 0, s>>>(B, m->h2, m->z2, b2, m->h2b, 1);
    gemm(m, B, m->n_out, m->h2, m->h2b, m->h2, 1, W3, 1, m->h2, m->y);
    k_bias_act<<<ew_blocks((size_t)B * m->n_out), 256, 0, s>>>(B, m->n_out, m->y, b3, nullptr, 0);
}

// gradient of the MSE loss w.r.t. every parameter into m->g; loss (device scalar)
void backward_core(tmr_mlp *m, int B, const float *T, float *loss)
{
    cudaStream_t s = m->stream;
    const __nv_bfloat16 *W2 = m->wb + m->off[2], *W3 = m->wb + m->off[4];
    const int nb = ew_blocks((size_t)B * m->n_out);
    if (m->loss_kind == TMR_LOSS_PHASE) {  // the loss against each row's aligned target
        k_align_targets<<<B, 256, 0, s>>>(m->n_out / 2, m->y, T, m->ta);
        T = m->ta;
    }
    k_mse<<<nb, 256, 0, s>>>(B, m->n_out, m->y, T, m->dyb, m->part);
    k_loss_finish<<<1, 32, 0, s>>>(nb, m->part, (float)((size_t)B * m->n_out), loss);
    // layer 3: dW3 = dY^T H2 ([n_out][B] x [B][h2]); db3 = colsum(dY); dH2 = dY W3
    gemm(m, m->n_out, m->h2, B, m->dyb, 1, m->n_out, m->h2b, m->h2, 1, m->g + m->off[4]);
    k_colsum<<<(m->n_out + 255) / 256, 256, 0, s>>>(B, m->n_out, m->dyb, m->g + m->off[5]);
    gemm(m, B, m->h2, m->n_out, m->dyb, m->n_out, 1, W3, m->h2, 1, m->dh);
    k_gelu_back<<<ew_blocks((size_t)B * m->h2), 256, 0, s>>>((size_t)B * m->h2, m->dh, m->z2, m->dz2b);
    // layer 2
    gemm(m, m->h2, m->h1, B, m->dz2b, 1, m->h2, m->h1b, m->h1, 1, m->g + m->off[2]);
    k_colsum<<<(m->h2 + 255) / 256, 256, 0, s>>>(B, m->h2, m->dz2b, m->g + m->off[3]);
    gemm(m, B, m->h1, m->h2, m->dz2b, m->h2, 1, W2, m->h1, 1, m->dh);
    k_gelu_back<<<ew_blocks((size_t)B * m->h1), 256, 0, s>>>((size_t)B * m->h1, m->dh, m->z1, m->dzb);
    // layer 1
    gemm(m, m->h1, m->n_in, B, m->dzb, 1, m->h1, m->xb, m->n_in, 1, m->g + m->off[0]);
    k_colsum<<<(m->h1 + 255) / 256, 256, 0, s>>>(B, m->h1, m->dzb, m->g + m->off[1]);
}

}  // namespace

namespace tmr {
// used by the learned start of tmr_retrieve: features of rows [r0, r0+B) of y
// -> candidate starts T (rows r0 ..)
cudaError_t mlp_propose(tmr_mlp *m, const float *y, int B, int N, int J, float2 *T, cudaStream_t s)
{
    if (ensure_batch(m, B) != TMR_OK) return cudaErrorMemoryAllocation;
    cudaStream_t keep = m->stream;
    m->stream = s;
    k_features<<<B, 256, 0, s>>>(J * N, y, m->xb);
    forward_core(m, B);
    k_candidate<<<B, 256, 0, s>>>(N, J * N, m->y, y, T);
    m->stream = keep;
    return cudaGetLastError();
}
int mlp_in(const tmr_mlp *m) { return m->n_in; }
int mlp_out(const tmr_mlp *m) { return m->n_out; }
}  // namespace tmr

extern "C" {

tmr_status tmr_mlp_create(tmr_mlp **out, int n_in, int n_h1, int n_h2, int n_out, unsigned long long seed,
                          void *stream)
{
    set_last_error("");
    if (!out || n_in <= 0 || n_h1 <= 0 || n_h2 <= 0 || n_out <= 0) return mfail(TMR_ERR_INVALID_ARG, "bad MLP size");
    tmr_mlp *m = new tmr_mlp();
    m->n_in = n_in;
    m->h1 = n_h1;
    m->h2 = n_h2;
    m->n_out = n_out;
    m->stream = (cudaStream_t)stream;
    const size_t sz[6] = {(size_t)n_h1 * n_in, (size_t)n_h1, (size_t)n_h2 * n_h1, (size_t)n_h2,
                          (size_t)n_out * n_h2, (size_t)n_out};
    size_t o = 0;
    for (int i = 0; i < 6; i++) {
        m->off[i] = o;
        o += sz[i];
    }
    m->np = o;
    const bool ok = cudaMalloc(&m->w, sizeof(float) * o) == cudaSuccess &&
                    cudaMalloc(&m->m, sizeof(float) * o) == cudaSuccess &&
                    cudaMalloc(&m->v, sizeof(float) * o) == cudaSuccess &&
                    cudaMalloc(&m->g, sizeof(float) * o) == cudaSuccess &&
                    cudaMalloc(&m->wb, sizeof(__nv_bfloat16) * o) == cudaSuccess &&
                    cudaMalloc(&m->part, sizeof(float) * 152 * 8) == cudaSuccess &&
                    cudaMalloc(&m->lossd, sizeof(float) * 4) == cudaSuccess &&
                    cudaMalloc(&m->tc_err, sizeof(int)) == cudaSuccess &&
                    cudaMemset(m->tc_err, 0, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        tmr_mlp_destroy(m);
        return mfail(TMR_ERR_OOM, "MLP parameters");
    }
    // He-style start: W ~ U(-s, s) with s = sqrt(3 / fan_in) (Philox), biases 0
    float *hw = (float *)malloc(sizeof(float) * o);
    for (int l = 0; l < 3; l++) {
        const int fan_in = l == 0 ? n_in : (l == 1 ? n_h1 : n_h2);
        const float s = sqrtf(3.f / (float)fan_in);
        for (size_t i = 0; i < sz[2 * l]; i++) {
            const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), (uint32_t)l, 0u),
                                          make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
            hw[m->off[2 * l] + i] = s * (2.f * ((float)r.x * 0x1p-32f) - 1.f);
        }
        for (size_t i = 0; i < sz[2 * l + 1]; i++) hw[m->off[2 * l + 1] + i] = 0.f;
    }
    tmr_status st = tmr_mlp_set_params(m, hw);
    free(hw);
    if (st != TMR_OK) {
        tmr_mlp_destroy(m);
        return st;
    }
    *out = m;
    return TMR_OK;
}

size_t tmr_mlp_num_params(const tmr_mlp *m) { return m ? m->np : 0; }

tmr_status tmr_mlp_set_params(tmr_mlp *m, const float *params)
{
    set_last_error("");
    if (!m || !params) return mfail(TMR_ERR_INVALID_ARG, "NULL argument");
    if (cudaMemcpyAsync(m->w, params, sizeof(float) * m->np, cudaMemcpyDefault, m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->m, 0, sizeof(float) * m->np, m->stream) != cudaSuccess ||
        cudaMemsetAsync(m->v, 0, sizeof(float) * m->np, m->stream) != cudaSuccess)
        return mfail(TMR_ERR_CUDA, "set params");
    k_to_bf16<<<ew_blocks(m->np), 256, 0, m->stream>>>(m->np, m->w, m->wb);
    m->step = 0;
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return mfail(TMR_ERR_CUDA, "set params sync");
    return TMR_OK;
}

tmr_status tmr_mlp_get_params(tmr_mlp *m, float *params)
{
    set_last_error("");
    if (!m || !params) return mfail(TMR_ERR_INVALID_ARG, "NULL argument");
    int tc_err = 0;
    if (cudaMemcpyAsync(params, m->w, sizeof(float) * m->np, cudaMemcpyDefault, m->stream) != cudaSuccess ||
        cudaMemcpyAsync(&tc_err, m->tc_err, sizeof(int), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return mfail(TMR_ERR_CUDA, "get params");
    if (tc_err) return mfail(TMR_ERR_TIMEOUT, "a tensor-core GEMM barrier wait ran out");
    return TMR_OK;
}

tmr_status tmr_mlp_forward(tmr_mlp *m, const float *X, int B, float *Y)
{
    set_last_error("");
    if (!m || !X || !Y || B <= 0) return mfail(TMR_ERR_INVALID_ARG, "bad argument");
    if (!dev_ptr(X) || !dev_ptr(Y)) return mfail(TMR_ERR_INVALID_ARG, "X and Y must be device memory");
    tmr_status st = ensure_batch(m, B);
    if (st != TMR_OK) return st;
    k_to_bf16<<<ew_blocks((size_t)B * m->n_in), 256, 0, m->stream>>>((size_t)B * m->n_in, X, m->xb);
    forward_core(m, B);
    if (cudaMemcpyAsync(Y, m->y, sizeof(float) * (size_t)B * m->n_out, cudaMemcpyDeviceToDevice, m->stream) !=
        cudaSuccess)
        return mfail(TMR_ERR_CUDA, "forward copy");
    return cudaGetLastError() == cudaSuccess ? TMR_OK : mfail(TMR_ERR_CUDA, "forward kernels");
}

tmr_status tmr_mlp_grad(tmr_mlp *m, const float *X, const float *T, int B, float *loss, float *grad)
{
    set_last_error("");
    if (!m || !X || !T || B <= 0) return mfail(TMR_ERR_INVALID_ARG, "bad argument");
    if (!dev_ptr(X) || !dev_ptr(T) || (loss && !dev_ptr(loss)) || (grad && !dev_ptr(grad)))
        return mfail(TMR_ERR_INVALID_ARG, "arrays must be device memory");
    tmr_status st = ensure_batch(m, B);
    if (st != TMR_OK) return st;
    k_to_bf16<<<ew_blocks((size_t)B * m->n_in), 256, 0, m->stream>>>((size_t)B * m->n_in, X, m->xb);
    forward_core(m, B);
    backward_core(m, B, T, loss ? loss : m->lossd);
    if (grad && cudaMemcpyAsync(grad, m->g, sizeof(float) * m->np, cudaMemcpyDeviceToDevice, m->stream) != cudaSuccess)
        return mfail(TMR_ERR_CUDA, "grad copy");
    return cudaGetLastError() == cudaSuccess ? TMR_OK : mfail(TMR_ERR_CUDA, "grad kernels");
}

tmr_status tmr_mlp_train_step(tmr_mlp *m, const float *X, const float *T, int B, float lr, float *loss)
{
    tmr_status st = tmr_mlp_grad(m, X, T, B, loss, nullptr);
    if (st != TMR_OK) return st;
    m->step++;
    const float c1 = 1.f - powf(0.9f, (float)m->step), c2 = 1.f - powf(0.999f, (float)m->step);
    k_adam<<<ew_blocks(m->np), 256, 0, m->stream>>>(m->np, m->w, m->g, m->m, m->v, m->wb, lr, c1, c2);
    return cudaGetLastError() == cudaSuccess ? TMR_OK : mfail(TMR_ERR_CUDA, "adam kernel");
}

tmr_status tmr_mlp_set_loss(tmr_mlp *m, int kind)
{
    set_last_error("");
    if (!m) return mfail(TMR_ERR_INVALID_ARG, "NULL network");
    if (kind != TMR_LOSS_MSE && kind != TMR_LOSS_PHASE) return mfail(TMR_ERR_INVALID_ARG, "unknown loss");
    if (kind == TMR_LOSS_PHASE && m->n_out % 2 != 0)
        return mfail(TMR_ERR_INVALID_ARG, "the phase-invariant loss needs an even number of outputs");
    m->loss_kind = kind;
    return TMR_OK;
}

void tmr_mlp_destroy(tmr_mlp *m)
{
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    else cudaDeviceSynchronize();
    void *p[] = {m->w, m->m, m->v, m->g, m->wb, m->xb, m->h1b, m->h2b, m->dzb, m->dz2b, m->dyb,
                 m->z1, m->z2, m->y, m->dh, m->part, m->lossd, m->ta, m->tsa, m->tsb, m->tc_err};
    for (void *q : p)
        if (q) cudaFree(q);
    delete m;
}

}  // extern "C"
