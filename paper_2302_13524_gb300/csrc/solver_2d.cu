// solver_2d.cu -- instantiations of the persistent solver with the 2D probing
// DFT (XfPow2D, xform.cuh): N = 512 (G = 1, 2, 4 masks per CTA) and N = 4096
// (G = 1).
#include "solver_impl.cuh"

namespace tmr {

long long solver_dispatch_2d(int N, int G, int what, const SolverParams *p, cudaStream_t s, int *clusters_out)
{
#define TMR_SOLVER_2D(NN, GG)                                                                  \
    if (N == NN && G == GG) {                                                                  \
        if (what == 0) return (long long)solver_smem<XfPow2D<NN>, GG>(NN, p->J, p->m);           \
        return (long long)launch_solver_t<XfPow2D<NN>, GG>(*p, s, clusters_out);                 \
    }
    TMR_SOLVER_2D(512, 1)
    TMR_SOLVER_2D(512, 2)
    TMR_SOLVER_2D(512, 4)
    TMR_SOLVER_2D(4096, 1)
#undef TMR_SOLVER_2D
    return what == 0 ? 0 : (long long)cudaErrorInvalidValue;
}

}  // namespace tmr
