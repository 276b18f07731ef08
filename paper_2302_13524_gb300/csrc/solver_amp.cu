// solver_amp.cu -- the cluster solver with the amplitude cost (cost.cuh) for
// powers of two up to 512, G = 1, 2, 4 masks per CTA; solver_amp2.cu holds
// N = 1024 .. 4096 and solver_bs_amp.cu the Bluestein lengths.  Separate translation units from the intensity kernels,
// so that both costs compile in parallel.
#include "solver_impl.cuh"

namespace tmr {

long long solver_launch_blue_amp(int N, const SolverParams &p, cudaStream_t s, int *clusters_out);
cudaError_t launch_solver_amp_large(int N, int G, const SolverParams &p, cudaStream_t s, int *clusters_out);

#define TMR_AMP_N_G(NN, GG)                                                                     \
    if (N == NN && G == GG) {                                                                   \
        if constexpr (GG * fft_threads(NN) <= 512)                                              \
            return launch_solver_t<XfPow2<NN>, GG, COST_AMPLITUDE>(p, s, clusters_out);          \
    }
#define TMR_AMP_N(NN) TMR_AMP_N_G(NN, 1) TMR_AMP_N_G(NN, 2) TMR_AMP_N_G(NN, 4)

bool solver_cost_supported(int N, int G, int prec, int cost)
{
    if (cost == COST_INTENSITY) return true;
    if (cost != COST_AMPLITUDE || prec != 0) return false;
    if (G == kRowSchedule) return N == 512 || N == 1024 || N == 2048;
    if (fft_supported(N)) return (G == 1 || G == 2 || G == 4) && G * fft_threads(N) <= 512;
    int L = 0, ne = 0;
    return G == 1 && xform_blue_shape(N, &L, &ne) && L <= 4096;
}

cudaError_t launch_solver_amp(int N, int G, const SolverParams &p, cudaStream_t s, int *clusters_out)
{
    if (!solver_cost_supported(N, G, p.prec, COST_AMPLITUDE) || G == kRowSchedule) return cudaErrorInvalidValue;
    if (!fft_supported(N)) return (cudaError_t)solver_launch_blue_amp(N, p, s, clusters_out);
    TMR_AMP_N(64)
    TMR_AMP_N(128)
    TMR_AMP_N(256)
    TMR_AMP_N(512)
    if (N >= 1024) return launch_solver_amp_large(N, G, p, s, clusters_out);
    return cudaErrorInvalidValue;
}

}  // namespace tmr
