// solver.cu -- instantiations of the persistent solver for power-of-two N and
// the variant queries of both transform kinds.
#include "solver_impl.cuh"

namespace tmr {

// Masks per CTA that have a kernel for length N: powers of two with
// G * threads(N) <= 512; other lengths (Bluestein) with G = 1.
bool solver_variant_exists(int N, int G, int prec)
{
    if (prec == 2) return (G == 1 || G == 2 || G == 4) && (N == 512 || N == 4096) && G * fft_threads(N) <= 512;
    if (prec == 3) return G == 1 && fft_supported(N);
    if (G == kRowSchedule) return prec == 0 && (N == 512 || N == 1024 || N == 2048);
    if (G == kBlueFullSchedule) return prec == 0 && N > 2048 && N <= 2731;
    if (G != 1 && G != 2 && G != 4) return false;
    if (prec != 0) return G == 1 && mixed_supported(N);
    if (fft_supported(N)) return G * fft_threads(N) <= 512;
    return G == 1 && xform_supported(N);
}

#define TMR_SOLVER_N_G(NN, GG)                                                                  \
    if (N == NN && G == GG) {                                                                   \
        if constexpr (GG * fft_threads(NN) <= 512) {                                            \
            if (what == 0) return (long long)solver_smem<XfPow2<NN>, GG>(NN, p->J, p->m);        \
            return (long long)launch_solver_t<XfPow2<NN>, GG>(*p, s, clusters_out);              \
        }                                                                                       \
    }
#define TMR_SOLVER_N(NN) TMR_SOLVER_N_G(NN, 1) TMR_SOLVER_N_G(NN, 2) TMR_SOLVER_N_G(NN, 4)

// N = 1024 .. 4096 (solver_p2.cu: a translation unit of its own, compiled in parallel)
long long solver_dispatch_pow2_large(int N, int G, int what, const SolverParams *p, cudaStream_t s,
                                     int *clusters_out);

// what == 0: shared-memory bytes of the variant; what == 1: launch it.
static long long solver_dispatch(int N, int G, int what, const SolverParams *p, cudaStream_t s,
                                 int *clusters_out)
{
    if (G == kRowSchedule) return solver_dispatch_row(N, what, p, s, clusters_out);
    if (G == kBlueFullSchedule) return solver_dispatch_blue8192(N, 6, what, p, s, clusters_out);
    if (p->prec == 2) return solver_dispatch_2d(N, G, what, p, s, clusters_out);
    if (p->prec == 3) return solver_dispatch_dense(N, G, what, p, s, clusters_out);
    if (p->prec != 0) return solver_dispatch_mixed(N, G, what, p, s, clusters_out);
    if (!fft_supported(N)) return solver_dispatch_blue(N, G, what, p, s, clusters_out);
    TMR_SOLVER_N(64)
    TMR_SOLVER_N(128)
    TMR_SOLVER_N(256)
    TMR_SOLVER_N(512)
    if (N >= 1024) return solver_dispatch_pow2_large(N, G, what, p, s, clusters_out);
    return what == 0 ? 0 : (long long)cudaErrorInvalidValue;
}

size_t solver_smem_bytes(int N, int J, int m, int G, int prec)
{
    SolverParams p{};
    p.N = N;
    p.J = J;
    p.m = m;
    p.prec = prec;
    if (!solver_schedule_valid(N, J, G, prec)) return 0;
    return (size_t)solver_dispatch(N, G, 0, &p, nullptr, nullptr);
}

bool solver_schedule_valid(int N, int J, int G, int prec)
{
    if (!solver_variant_exists(N, G, prec) || J < 1) return false;
    if (G == kRowSchedule) return J * (N / 16) <= 512;
    if (G == kBlueFullSchedule) return true;  // one mask per CTA
    return J % G == 0;
}

cudaError_t launch_solver(int N, int G, const SolverParams &p, cudaStream_t s, int *clusters_out)
{
    if (p.M == 0) return cudaSuccess;
    if (!solver_schedule_valid(N, p.J, G, p.prec) || p.N != N) return cudaErrorInvalidValue;
    if (!solver_cost_supported(N, G, p.prec, p.cost)) return cudaErrorInvalidValue;
    if (p.cost == COST_AMPLITUDE && G != kRowSchedule) return launch_solver_amp(N, G, p, s, clusters_out);
    return (cudaError_t)solver_dispatch(N, G, 1, &p, s, clusters_out);
}

}  // namespace tmr
