// solver_row.cu -- instantiations of the one-CTA-per-row solver (solver_row.cuh).
#include "solver_row.cuh"

namespace tmr {

#define TMR_ROW_N(NN)                                                      \
    case NN:                                                               \
        if (what == 0) return (long long)row_smem<NN>(p->J, p->m);         \
        return (long long)launch_solver_row_t<NN>(*p, s, ctas_out);

// what == 0: shared-memory bytes; what == 1: launch (the amplitude cost's
// kernels are instantiated in solver_row_amp.cu).
long long solver_dispatch_row(int N, int what, const SolverParams *p, cudaStream_t s, int *ctas_out)
{
    if (!row_variant_fits(N, p->J)) return what == 0 ? 0 : (long long)cudaErrorInvalidValue;
    if (what == 1 && p->cost == COST_AMPLITUDE) return (long long)launch_solver_row_amp(N, *p, s, ctas_out);
    switch (N) {
        TMR_ROW_N(512)
        TMR_ROW_N(1024)
        TMR_ROW_N(2048)
    default: return what == 0 ? 0 : (long long)cudaErrorInvalidValue;
    }
}

template <int N>
static int row_max_ctas_t(int J, int m)
{
    size_t sm = 0;
    int occ = 0, dev = 0, nsm = 0;
    // the largest tensor-memory need of the schedule (a 16-step Lanczos start)
    // bounds the resident CTAs of every launch
    const int klz = row_tmem_klz(N, J, true, kMaxLanczos);
    if (row_launch_shape<N, COST_INTENSITY>(J, m, klz, &sm, &occ) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return occ * nsm;
}

int solver_row_max_ctas(int N, int J, int m)
{
    if (!row_variant_fits(N, J)) return 0;
    switch (N) {
    case 512: return row_max_ctas_t<512>(J, m);
    case 1024: return row_max_ctas_t<1024>(J, m);
    case 2048: return row_max_ctas_t<2048>(J, m);
    default: return 0;
    }
}

size_t solver_row_pair_stride(int N, int m) { return row_pair_stride(N, m); }

}  // namespace tmr
