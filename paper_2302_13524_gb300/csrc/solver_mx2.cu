// solver_mx2.cu -- mixed-precision solver instantiations at N = 1024 and 2048
// (one mask per CTA); dispatched from solver_mx.cu.
#include "solver_impl.cuh"

namespace tmr {

long long solver_dispatch_mixed2(int N, int what, const SolverParams *p, cudaStream_t s, int *clusters_out)
{
    if (N == 1024) {
        if (what == 0) return (long long)solver_smem<XfMixed<1024>, 1>(N, p->J, p->m);
        return (long long)launch_solver_t<XfMixed<1024>, 1>(*p, s, clusters_out);
    }
    if (N == 2048) {
        if (what == 0) return (long long)solver_smem<XfMixed<2048>, 1>(N, p->J, p->m);
        return (long long)launch_solver_t<XfMixed<2048>, 1>(*p, s, clusters_out);
    }
    return what == 0 ? 0 : (long long)cudaErrorInvalidValue;
}

}  // namespace tmr
