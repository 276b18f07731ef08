// solver_p2.cu -- instantiations of the persistent cluster solver for the
// larger powers of two (N = 1024, 2048, 4096); solver.cu holds N <= 512 and
// the variant queries.
#include "solver_impl.cuh"

namespace tmr {

#define TMR_SOLVER_N_G(NN, GG)                                                                  \
    if (N == NN && G == GG) {                                                                   \
        if constexpr (GG * fft_threads(NN) <= 512) {                                            \
            if (what == 0) return (long long)solver_smem<XfPow2<NN>, GG>(NN, p->J, p->m);        \
            return (long long)launch_solver_t<XfPow2<NN>, GG>(*p, s, clusters_out);              \
        }                                                                                       \
    }
#define TMR_SOLVER_N(NN) TMR_SOLVER_N_G(NN, 1) TMR_SOLVER_N_G(NN, 2) TMR_SOLVER_N_G(NN, 4)

// what == 0: shared-memory bytes of the variant; what == 1: launch it.
long long solver_dispatch_pow2_large(int N, int G, int what, const SolverParams *p, cudaStream_t s,
                                     int *clusters_out)
{
    TMR_SOLVER_N(1024)
    TMR_SOLVER_N(2048)
    TMR_SOLVER_N(4096)
    return what == 0 ? 0 : (long long)cudaErrorInvalidValue;
}

}  // namespace tmr
