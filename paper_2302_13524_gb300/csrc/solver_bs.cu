// solver_bs.cu -- instantiations of the persistent solver for lengths that are
// not powers of two (Bluestein transforms of length L = 512 .. 8192, one mask
// per CTA).
#include "solver_impl.cuh"

namespace tmr {

#define TMR_SOLVER_BLUE(LL, NEE)                                                         \
    if (L == LL && ne == NEE) {                                                          \
        if (what == 0) return (long long)solver_smem<XfBlue<LL, NEE>, 1>(N, p->J, p->m);  \
        return (long long)launch_solver_t<XfBlue<LL, NEE>, 1>(*p, s, clusters_out);       \
    }

long long solver_dispatch_blue(int N, int G, int what, const SolverParams *p, cudaStream_t s, int *clusters_out)
{
    int L = 0, ne = 0;
    if (G != 1 || !xform_blue_shape(N, &L, &ne)) return what == 0 ? 0 : (long long)cudaErrorInvalidValue;
    TMR_SOLVER_BLUE(512, 8)
    TMR_SOLVER_BLUE(1024, 8)
    TMR_SOLVER_BLUE(2048, 8)
    TMR_SOLVER_BLUE(4096, 8)
    TMR_SOLVER_BLUE(8192, 5)
    TMR_SOLVER_BLUE(8192, 6)
    TMR_SOLVER_BLUE(8192, 7)
    TMR_SOLVER_BLUE(8192, 8)
    return what == 0 ? 0 : (long long)cudaErrorInvalidValue;
}

}  // namespace tmr
