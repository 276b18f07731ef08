// solver_amp2.cu -- the cluster solver with the amplitude cost for
// N = 1024, 2048, 4096 (G = 1, 2, 4 masks per CTA where they fit).
#include "solver_impl.cuh"

namespace tmr {

#define TMR_AMP_N_G(NN, GG)                                                                     \
    if (N == NN && G == GG) {                                                                   \
        if constexpr (GG * fft_threads(NN) <= 512)                                              \
            return launch_solver_t<XfPow2<NN>, GG, COST_AMPLITUDE>(p, s, clusters_out);          \
    }
#define TMR_AMP_N(NN) TMR_AMP_N_G(NN, 1) TMR_AMP_N_G(NN, 2) TMR_AMP_N_G(NN, 4)

cudaError_t launch_solver_amp_large(int N, int G, const SolverParams &p, cudaStream_t s, int *clusters_out)
{
    TMR_AMP_N(1024)
    TMR_AMP_N(2048)
    TMR_AMP_N(4096)
    return cudaErrorInvalidValue;
}

}  // namespace tmr
