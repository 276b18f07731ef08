// solver_mx.cu -- instantiations of the persistent solver for mixed precision
// (tensor-core transforms, FP16 intensities, BF16 L-BFGS pairs; one mask per
// CTA) at N = 256 and N = 4096.
#include "solver_impl.cuh"

namespace tmr {

long long solver_dispatch_mixed(int N, int G, int what, const SolverParams *p, cudaStream_t s, int *clusters_out)
{
    if (G == 1 && N == 256) {
        if (what == 0) return (long long)solver_smem<XfMixed<256>, 1>(N, p->J, p->m);
        return (long long)launch_solver_t<XfMixed<256>, 1>(*p, s, clusters_out);
    }
    if (G == 1 && N == 4096) {
        if (what == 0) return (long long)solver_smem<XfMixed<4096>, 1>(N, p->J, p->m);
        return (long long)launch_solver_t<XfMixed<4096>, 1>(*p, s, clusters_out);
    }
    return what == 0 ? 0 : (long long)cudaErrorInvalidValue;
}

}  // namespace tmr
