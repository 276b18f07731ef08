// solver_bs_amp.cu -- the cluster solver with the amplitude cost for lengths
// that are not powers of two: Bluestein transforms of length L = 512 .. 4096
// (split outputs at L = 4096 for N in (2048, 2731]), one mask per CTA.
#include "solver_impl.cuh"

namespace tmr {

long long solver_launch_blue_amp(int N, const SolverParams &p, cudaStream_t s, int *clusters_out)
{
    int L = 0, ne = 0;
    if (!xform_blue_shape(N, &L, &ne)) return (long long)cudaErrorInvalidValue;
    if (N > 2048 && L == 4096)
        return ne == 5 ? (long long)launch_solver_t<XfBlueSplit<5>, 1, COST_AMPLITUDE>(p, s, clusters_out)
                       : (long long)launch_solver_t<XfBlueSplit<6>, 1, COST_AMPLITUDE>(p, s, clusters_out);
    if (ne != 8) return (long long)cudaErrorInvalidValue;
    switch (L) {
    case 512: return (long long)launch_solver_t<XfBlue<512, 8>, 1, COST_AMPLITUDE>(p, s, clusters_out);
    case 1024: return (long long)launch_solver_t<XfBlue<1024, 8>, 1, COST_AMPLITUDE>(p, s, clusters_out);
    case 2048: return (long long)launch_solver_t<XfBlue<2048, 8>, 1, COST_AMPLITUDE>(p, s, clusters_out);
    case 4096: return (long long)launch_solver_t<XfBlue<4096, 8>, 1, COST_AMPLITUDE>(p, s, clusters_out);
    default: return (long long)cudaErrorInvalidValue;
    }
}

}  // namespace tmr
