// dense.cu -- the probing operator as an explicit dense matrix (the paper's
// "TM retrieval without FFT", Table 1): Q (K x N, K = J N) with rows
// Q[j N + k][n] = exp(-2 pi i k n / N) d_j[n] (Eq. probingmatrix) built once,
// and the forward model and the gradient of Eq. optTMsmall2 / Eq. derivative
// as complex matrix products over the batch of rows:
//   Z = T Q^T (M x K), then r = y - |Z|^2, U = Z .* r, G = -4 U conj(Q).
// The products are plain library GEMMs (cuBLAS, FP32 complex; or FP32
// emulated on the tensor cores by three BF16 terms per operand), the
// elementwise steps and the row losses are kernels here.  cuBLAS works in
// column-major order: a row-major r x c matrix is its c x r transpose there.
#include <cublas_v2.h>

#include <cmath>

#include "common.cuh"
#include "cost.cuh"
#include "internal.h"

namespace tmr {

// Q[i][n], i = j N + k: exp(-2 pi i ((k n) mod N) / N) d_j[n], the phase in FP64
__global__ void k_make_q(int N, int J, const float2 *__restrict__ masks, float2 *__restrict__ Q)
{
    const size_t K = (size_t)J * N, total = K * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / N), n = (int)(e % N);
        const int j = i / N, k = i % N;
        const long long kn = ((long long)k * n) % N;
        double s, c;
        sincospi(-2.0 * (double)kn / N, &s, &c);
        const float2 w = make_float2((float)c, (float)s);
        Q[e] = cmul(w, masks[(size_t)j * N + n]);
    }
}

// Row r of Z (K values): Y = |Z|^2 (forward), or the loss of row r and
// conj(U) with U = c Z (the cost's coefficient, cost.cuh) for the gradient.
__global__ void k_dense_residual(int K, const float2 *__restrict__ Z, const float *__restrict__ y, float *Y,
                                 float2 *Uc, float *loss, int cost)
{
    __shared__ float red[32], tot[1];
    const size_t base = (size_t)blockIdx.x * K;
    float f = 0.f;
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
        const float2 z = Z[base + i];
        if (Y) {
            Y[base + i] = cabs2(z);
        } else {
            const float c = cost_coef(cost, z, y[base + i], f);
            Uc[base + i] = make_float2(c * z.x, -c * z.y);
        }
    }
    if (!Y) {
        float fv[1] = {f};
        block_sum<1>(fv, red, tot);
        if (threadIdx.x == 0 && loss) loss[blockIdx.x] = tot[0];
    }
}

// G = s conj(C) (C = conj(G) / s from the product)
__global__ void k_dense_grad_out(size_t n, const float2 *__restrict__ C, float s, float2 *__restrict__ G)
{
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const float2 c = C[e];
        G[e] = make_float2(s * c.x, -s * c.y);
    }
}

static cublasStatus_t cgemm(cublasHandle_t hb, int mode, cublasOperation_t ta, int m, int n, int k,
                            const float2 *A, int lda, const float2 *B, int ldb, float2 *C, int ldc)
{
    const cuComplex one = make_cuComplex(1.f, 0.f), zero = make_cuComplex(0.f, 0.f);
    const cublasComputeType_t ct = mode == 2 ? CUBLAS_COMPUTE_32F_EMULATED_16BFX9 : CUBLAS_COMPUTE_32F;
    return cublasGemmEx(hb, ta, CUBLAS_OP_N, m, n, k, &one, A, CUDA_C_32F, lda, B, CUDA_C_32F, ldb, &zero, C,
                        CUDA_C_32F, ldc, ct, CUBLAS_GEMM_DEFAULT);
}

DenseState::~DenseState() { release(); }

void DenseState::release()
{
    if (blas) cublasDestroy((cublasHandle_t)blas);
    if (Q) cudaFree(Q);
    if (Z) cudaFree(Z);
    if (C) cudaFree(C);
    blas = nullptr;
    Q = Z = C = nullptr;
}

// Q, the cuBLAS handle and the scratch products, made on first use.
cudaError_t dense_prepare(DenseState &ds, int N, int M, int J, const float2 *masks, cudaStream_t s,
                          size_t *bytes_out)
{
    const size_t K = (size_t)J * N;
    if (!ds.blas) {
        cublasHandle_t hb = nullptr;
        if (cublasCreate(&hb) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
        ds.blas = hb;
    }
    size_t bytes = 0;
    if (!ds.Q) {
        cudaError_t e = cudaMalloc(&ds.Q, sizeof(float2) * K * N);
        if (e != cudaSuccess) return e;
        bytes += sizeof(float2) * K * N;
        k_make_q<<<1024, 256, 0, s>>>(N, J, masks, ds.Q);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (!ds.Z) {
        cudaError_t e = cudaMalloc(&ds.Z, sizeof(float2) * K * (M > 0 ? M : 1));
        if (e != cudaSuccess) return e;
        e = cudaMalloc(&ds.C, sizeof(float2) * K * (M > 0 ? M : 1));
        if (e != cudaSuccess) return e;
        bytes += 2 * sizeof(float2) * K * (M > 0 ? M : 1);
    }
    if (bytes_out) *bytes_out = bytes;
    cublasSetStream((cublasHandle_t)ds.blas, s);
    return cudaSuccess;
}

// Z = T Q^T: column-major Z^T (K x M) = Q (K x N) T^T (N x M), with Q's
// column-major storage Q^T (N x K, ld N) taken transposed.
static cudaError_t dense_fields(DenseState &ds, int mode, int N, int M, int J, const float2 *T)
{
    const int K = J * N;
    const cublasStatus_t st = cgemm((cublasHandle_t)ds.blas, mode, CUBLAS_OP_T, K, M, N, ds.Q, N, T, N, ds.Z, K);
    return st == CUBLAS_STATUS_SUCCESS ? cudaSuccess : cudaErrorNotSupported;
}

cudaError_t dense_forward(DenseState &ds, int mode, int N, int M, int J, const float2 *T, float *Y, cudaStream_t s)
{
    if (M == 0) return cudaSuccess;
    cudaError_t e = dense_fields(ds, mode, N, M, J, T);
    if (e != cudaSuccess) return e;
    k_dense_residual<<<M, 256, 0, s>>>(J * N, ds.Z, nullptr, Y, nullptr, nullptr, 0);
    return cudaGetLastError();
}

// conj(G) / s = conj(U) Q: column-major conj(G)^T (N x M) = Q^T (N x K, ld N) conj(U)^T (K x M, ld K)
cudaError_t dense_grad(DenseState &ds, int mode, int N, int M, int J, const float2 *T, const float *y, float *loss,
                       float2 *G, int cost, cudaStream_t s)
{
    if (M == 0) return cudaSuccess;
    const int K = J * N;
    cudaError_t e = dense_fields(ds, mode, N, M, J, T);
    if (e != cudaSuccess) return e;
    k_dense_residual<<<M, 256, 0, s>>>(K, ds.Z, y, nullptr, ds.C, loss, cost);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (!G) return cudaSuccess;
    const cublasStatus_t st = cgemm((cublasHandle_t)ds.blas, mode, CUBLAS_OP_N, N, M, K, ds.Q, N, ds.C, K, ds.Z, N);
    if (st != CUBLAS_STATUS_SUCCESS) return cudaErrorNotSupported;
    k_dense_grad_out<<<1024, 256, 0, s>>>((size_t)M * N, ds.Z, cost_grad_scale(cost), G);
    return cudaGetLastError();
}

}  // namespace tmr
