// solver_row_amp.cu -- the one-CTA-per-row solver with the amplitude cost
// (cost.cuh), in a translation unit of its own so that both costs compile in
// parallel; the intensity kernels are in solver_row.cu.
#include "solver_row.cuh"

namespace tmr {

cudaError_t launch_solver_row_amp(int N, const SolverParams &p, cudaStream_t s, int *ctas_out)
{
    switch (N) {
    case 512: return launch_solver_row_t<512, COST_AMPLITUDE>(p, s, ctas_out);
    case 1024: return launch_solver_row_t<1024, COST_AMPLITUDE>(p, s, ctas_out);
    case 2048: return launch_solver_row_t<2048, COST_AMPLITUDE>(p, s, ctas_out);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tmr
