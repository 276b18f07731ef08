// noalloc.cu -- tmr_retrieve_rows_static: the per-row solver without any
// allocation, for callers that may not call cudaMalloc.
//
// The solver kernel needs two pieces of scratch beyond the caller's arrays: a
// row work counter and the FFT twiddle table.  Here they live in one
// file-scope device array (kStaticScratchBytes, 64 KiB) that every GPU which
// loads the library holds until the process exits.  Host code never passes
// the symbol itself to a kernel (in host code it is only a stand-in): the
// device address comes from cudaGetSymbolAddress, fetched once per device
// with that device current, on the first call made on that device, and kept
// for the life of the process: after cudaDeviceReset the module is loaded
// again and the array may move, so the entry point must not be used on a
// device that was reset after its first call there.
//
// The twiddle table is filled on the device (k_fill_twiddles, sincospi in
// FP64 rounded to FP32): the host table of the handle path would have to be
// copied from pageable host memory, a copy that blocks the calling thread
// until the stream reaches it.  Both tables round the same FP64
// angles; an FP64 result one ulp off can move the FP32 rounding by one ulp,
// so the table agrees with the host table to 1 ulp of FP32 (6e-8 absolute)
// and the retrieved rows agree with tmr_retrieve's to FP32 rounding.
#include <cstdio>
#include <mutex>

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"
#include "tmr.h"

namespace {

constexpr size_t kStaticScratchBytes = 64 * 1024;
constexpr size_t kCounterBytes = 256;  // the work counter, then the table
constexpr int kMaxDevices = 64;

// [0, 256): row work counter; [256, 64 KiB): twiddle table (<= 8160 float2)
__device__ __align__(256) unsigned char g_tmr_static_scratch[kStaticScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

tmr_status fail(tmr_status st, const char *msg)
{
    tmr::set_last_error(msg);  // read back with tmr_last_error()
    return st;
}

template <int N>
__global__ void k_fill_twiddles(float2 *tw)
{
    using Pl = tmr::FftPlan<N, N / tmr::fft_threads(N)>;
    for (int p = 1; p < Pl::P; p++) {
        const int R = Pl::radix(p), Ns = Pl::ns(p), off = Pl::tw_off(p);
        for (int i = threadIdx.x; i < (R - 1) * Ns; i += blockDim.x) {
            const int r = 1 + i / Ns, j = i % Ns;
            double s, c;
            sincospi(-2.0 * (double)r * (double)j / ((double)Ns * R), &s, &c);
            tw[off + (r - 1) * Ns + j] = make_float2((float)c, (float)s);
        }
    }
}

cudaError_t fill_twiddles(int N, float2 *tw, cudaStream_t s)
{
    switch (N) {
    case 64: k_fill_twiddles<64><<<1, 256, 0, s>>>(tw); break;
    case 128: k_fill_twiddles<128><<<1, 256, 0, s>>>(tw); break;
    case 256: k_fill_twiddles<256><<<1, 256, 0, s>>>(tw); break;
    case 512: k_fill_twiddles<512><<<1, 256, 0, s>>>(tw); break;
    case 1024: k_fill_twiddles<1024><<<1, 256, 0, s>>>(tw); break;
    case 2048: k_fill_twiddles<2048><<<1, 256, 0, s>>>(tw); break;
    case 4096: k_fill_twiddles<4096><<<1, 256, 0, s>>>(tw); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

bool device_ptr(const void *p) { return tmr::is_device_ptr(p); }

}  // namespace

extern "C" tmr_status tmr_retrieve_rows_static(int N, int M, int J, const void *masks,
                                               const float *y, int iters, const tmr_options *opt,
                                               void *T_out, int *row_status, int *row_iters,
                                               float *row_loss, void *stream)
{
    tmr::set_last_error("");
    tmr_options o;
    tmr_default_options(&o);
    if (opt) o = *opt;
    if (N <= 0 || M < 0 || J <= 0 || iters < 0) return fail(TMR_ERR_INVALID_ARG, "bad size or iters");
    if (M == 0) return TMR_OK;  // no rows: nothing is launched, the arrays are not read
    if (!masks || !y || !T_out) return fail(TMR_ERR_INVALID_ARG, "NULL array");
    if (!tmr::fft_supported(N)) return fail(TMR_ERR_UNSUPPORTED, "N must be a power of two in 64..4096");
    if (J > tmr::kMaxMasks) return fail(TMR_ERR_UNSUPPORTED, "J must be at most 8");
    if (o.m < 1 || o.m > tmr::kMaxMem) return fail(TMR_ERR_INVALID_ARG, "opt.m must be in 1..6");
    if (o.init < TMR_INIT_RANDOM || o.init > TMR_INIT_SPECTRAL || o.power_iters < 0 || o.tol < 0)
        return fail(TMR_ERR_INVALID_ARG, "bad option");
    if (o.cost != TMR_COST_INTENSITY && o.cost != TMR_COST_AMPLITUDE) return fail(TMR_ERR_INVALID_ARG, "bad option");
    if (o.lanczos)
        return fail(TMR_ERR_UNSUPPORTED, "the static entry point runs the power iteration (opt.lanczos = 0): "
                                         "the Lanczos vectors need a workspace");
    if (o.precision != TMR_PREC_FP32)
        return fail(TMR_ERR_UNSUPPORTED, "the static entry point runs the FP32 solver only (opt.precision)");
    if (o.probe_n1 != 0)
        return fail(TMR_ERR_UNSUPPORTED, "the static entry point uses the 1D probing DFT (opt.probe_n1 = 0)");
    const int twn = tmr::fft_table_len(N);
    if ((size_t)twn * sizeof(float2) + kCounterBytes > kStaticScratchBytes)
        return fail(TMR_ERR_UNSUPPORTED, "twiddle table larger than the static scratch");
    const void *arrays[] = {masks, y, T_out, row_status, row_iters, row_loss};
    for (const void *a : arrays)
        if (a && !device_ptr(a))
            return fail(TMR_ERR_INVALID_ARG, "every array must be device memory of the current device");

    int dev = 0, smem_optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(TMR_ERR_CUDA, "cudaGetDevice failed or device ordinal too large");
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return fail(TMR_ERR_CUDA, "cudaDeviceGetAttribute failed");
    const size_t smem = tmr::solver_smem_bytes(N, J, o.m, 1);
    if (smem == 0 || smem > (size_t)smem_optin)
        return fail(TMR_ERR_UNSUPPORTED, "per-row state of this (N, J, m) does not fit in shared memory");

    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_tmr_static_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return fail(TMR_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
            }
            g_scratch_addr[dev] = p;
        }
        base = g_scratch_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *queue = (unsigned *)base;
    float2 *tw = (float2 *)((unsigned char *)base + kCounterBytes);
    if (cudaMemsetAsync(queue, 0, sizeof(unsigned), s) != cudaSuccess)
        return fail(TMR_ERR_CUDA, "clearing the work counter failed");
    if (fill_twiddles(N, tw, s) != cudaSuccess) return fail(TMR_ERR_CUDA, "twiddle kernel failed");

    tmr::SolverParams p{};
    p.masks = (const float2 *)masks;
    p.tw = tw;
    p.y = y;
    p.T_init = nullptr;
    p.T_out = (float2 *)T_out;
    p.row_status = row_status;
    p.row_iters = row_iters;
    p.row_loss = row_loss;
    p.Zd = nullptr;
    p.queue = queue;
    p.Nd = 0;
    p.M = M;
    p.N = N;
    p.J = J;
    p.iters = iters;
    p.m = o.m;
    p.init = o.init;
    p.power_iters = o.power_iters;
    p.cost = o.cost;
    p.seed = o.seed;
    p.clip = (float)o.clip;
    p.tol = o.tol;
    const cudaError_t e = tmr::launch_solver(N, 1, p, s, nullptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(TMR_ERR_CUDA, "solver launch failed");
    }
    return TMR_OK;
}
