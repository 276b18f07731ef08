// solver_bs.cu -- instantiations of the persistent solver for lengths that are
// not powers of two (Bluestein transforms of length L = 512 .. 8192, with the
// split-output form at L = 4096 for N in (2048, 2731]; one mask per CTA);
// solver_bs2.cu holds L = 8192.
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
    if (N > 2048 && L == 4096) {  // split outputs at L = 4096
        if (ne == 5) {
            if (what == 0) return (long long)solver_smem<XfBlueSplit<5>, 1>(N, p->J, p->m);
            return (long long)launch_solver_t<XfBlueSplit<5>, 1>(*p, s, clusters_out);
        }
        if (what == 0) return (long long)solver_smem<XfBlueSplit<6>, 1>(N, p->J, p->m);
        return (long long)launch_solver_t<XfBlueSplit<6>, 1>(*p, s, clusters_out);
    }
    TMR_SOLVER_BLUE(512, 8)
    TMR_SOLVER_BLUE(1024, 8)
    TMR_SOLVER_BLUE(2048, 8)
    TMR_SOLVER_BLUE(4096, 8)
    if (L == 8192) return solver_dispatch_blue8192(N, ne, what, p, s, clusters_out);
    return what == 0 ? 0 : (long long)cudaErrorInvalidValue;
}

}  // namespace tmr
