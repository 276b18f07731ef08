// solver_bs2.cu -- Bluestein solver instantiations at L = 8192 (N in
// (2731, 4096], 6..8 registers per thread; and, as schedule 32, N in
// (2048, 2731] with 6 registers); dispatched from solver_bs.cu and solver.cu.
#include "solver_impl.cuh"

namespace tmr {

long long solver_dispatch_blue8192(int N, int ne, int what, const SolverParams *p, cudaStream_t s,
                                   int *clusters_out)
{
#define TMR_SOLVER_BLUE8192(NEE)                                                           \
    if (ne == NEE) {                                                                      \
        if (what == 0) return (long long)solver_smem<XfBlue<8192, NEE>, 1>(N, p->J, p->m);  \
        return (long long)launch_solver_t<XfBlue<8192, NEE>, 1>(*p, s, clusters_out);       \
    }
    TMR_SOLVER_BLUE8192(6)
    TMR_SOLVER_BLUE8192(7)
    TMR_SOLVER_BLUE8192(8)
#undef TMR_SOLVER_BLUE8192
    return what == 0 ? 0 : (long long)cudaErrorInvalidValue;
}

}  // namespace tmr
