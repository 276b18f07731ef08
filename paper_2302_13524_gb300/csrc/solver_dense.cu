// solver_dense.cu -- the persistent solver with the matrix-vector transform
// policy XfDenseMV (xform.cuh): Algorithm 1 without FFT, for the paper's
// Table 1 comparison (powers of two 64 .. 4096, one mask per CTA).
#include "solver_impl.cuh"

namespace tmr {

#define TMR_DENSE_N(NN)                                                                   \
    case NN:                                                                              \
        if (what == 0) return (long long)solver_smem<XfDenseMV<NN>, 1>(NN, p->J, p->m);    \
        return (long long)launch_solver_t<XfDenseMV<NN>, 1>(*p, s, clusters_out);

// what == 0: shared-memory bytes; what == 1: launch
long long solver_dispatch_dense(int N, int G, int what, const SolverParams *p, cudaStream_t s, int *clusters_out)
{
    if (G != 1) return what == 0 ? 0 : (long long)cudaErrorInvalidValue;
    switch (N) {
        TMR_DENSE_N(64)
        TMR_DENSE_N(128)
        TMR_DENSE_N(256)
        TMR_DENSE_N(512)
        TMR_DENSE_N(1024)
        TMR_DENSE_N(2048)
        TMR_DENSE_N(4096)
    default: return what == 0 ? 0 : (long long)cudaErrorInvalidValue;
    }
}

// W_N^m = exp(-2 pi i m / N), m < N, in FP64 rounded once
int dense_mv_table(int N, float2 *out)
{
    if (!fft_supported(N)) return -1;
    if (out)
        for (int m = 0; m < N; m++) {
            double s, c;
            const double ph = -2.0 * M_PI * (double)m / (double)N;
            s = std::sin(ph);
            c = std::cos(ph);
            out[m] = make_float2((float)c, (float)s);
        }
    return N;
}

}  // namespace tmr
