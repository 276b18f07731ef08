// solver_mx.cu -- instantiations of the persistent solver for mixed precision
// (tensor-core transforms, FP16 intensities, BF16 L-BFGS pairs; one mask per
// CTA) at N = 256 and 4096; solver_mx2.cu holds N = 1024 and 2048.
#include "solver_impl.cuh"

namespace tmr {

long long solver_dispatch_mixed2(int N, int what, const SolverParams *p, cudaStream_t s, int *clusters_out);

long long solver_dispatch_mixed(int N, int G, int what, const SolverParams *p, cudaStream_t s, int *clusters_out)
{
    if (G != 1) return what == 0 ? 0 : (long long)cudaErrorInvalidValue;
    if (N == 256) {
        if (what == 0) return (long long)solver_smem<XfMixed<256>, 1>(N, p->J, p->m);
        return (long long)launch_solver_t<XfMixed<256>, 1>(*p, s, clusters_out);
    }
    if (N == 4096) {
        if (what == 0) return (long long)solver_smem<XfMixed<4096>, 1>(N, p->J, p->m);
        return (long long)launch_solver_t<XfMixed<4096>, 1>(*p, s, clusters_out);
    }
    return solver_dispatch_mixed2(N, what, p, s, clusters_out);
}

}  // namespace tmr
