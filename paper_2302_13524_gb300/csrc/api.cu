// api.cu -- the C ABI of libtmr (declared in include/tmr.h).
//
// Owns the handle (sizes, options, the device copies of the masks, the FFT
// twiddle table and the defocus transfer function, and every scratch buffer),
// validates arguments, stages host arrays through device buffers, and
// sequences the kernels of one retrieval on the handle's stream:
//   solver (per-row Algorithm 1, persistent cluster kernel) -> row energies ->
//   phase-offset fit (cooperative kernel) -> T_out = diag(e^{i phi}) T_est.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "tmr.h"

using namespace tmr;

namespace {
thread_local char g_last_error_buf[512];
}

void tmr::set_last_error(const char *msg)
{
    if (!msg) msg = "";
    snprintf(g_last_error_buf, sizeof(g_last_error_buf), "%s", msg);
}

int tmr::pointer_class(const void *p)
{
    if (!p) return PTR_HOST;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return PTR_HOST;
    }
    if (a.type == cudaMemoryTypeManaged) return PTR_DEVICE;
    if (a.type != cudaMemoryTypeDevice) return PTR_HOST;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PTR_OTHER_DEVICE;
    }
    return a.device == dev ? PTR_DEVICE : PTR_OTHER_DEVICE;
}

bool tmr::is_device_ptr(const void *p) { return pointer_class(p) == PTR_DEVICE; }

namespace {

tmr_status fail(tmr_status st, const std::string &msg)
{
    tmr::set_last_error(msg.c_str());
    return st;
}

tmr_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(e == cudaErrorMemoryAllocation ? TMR_ERR_OOM : TMR_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define TMR_CUDA(call, what)                      \
    do {                                          \
        cudaError_t e__ = (call);                 \
        if (e__ != cudaSuccess) return cuda_fail(e__, what); \
    } while (0)

}  // namespace

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct tmr_handle {
    int N = 0, M = 0, J = 0;
    tmr_options opt{};
    bool has_defocus = false;
    int ny = 0, nx = 0, Nd = 0, dkind = 0;
    bool fit_ran = false;
    float2 *incident = nullptr;  // kind 1: [Nd][N] incident fields
    cudaStream_t stream = nullptr;
    size_t held = 0;
    // persistent device state
    float2 *masks = nullptr, *tw = nullptr, *H = nullptr, *Zd = nullptr;
    double *phi = nullptr, *pf_ws = nullptr, *pf_loss = nullptr;
    float *wts = nullptr;
    unsigned *queue = nullptr, *pf_sync = nullptr;
    int *pf_err = nullptr, *pf_iters = nullptr;
    int *status_scratch = nullptr, *iters_scratch = nullptr;
    float *loss_scratch = nullptr;
    // token allocation of the one-CTA-per-row schedule (its pairs are in tensor
    // memory) and its resident CTA count
    float2 *pairs = nullptr;
    int pair_ctas = 0;
    // the probing operator as a dense matrix (opt.dense), made on first use
    DenseState dense;
    // Lanczos vectors of the spectral start (krylov_units regions of power_iters N)
    float2 *krylov = nullptr;
    int krylov_units = 0;
    // transform table of the full-length Bluestein schedule (2048 < N <= 2731)
    float2 *tw_alt = nullptr;
    // what the autotuner timed when this handle was made (none: given or cached)
    int tune_n = 0;
    int tune_codes[8] = {};
    float tune_ms[8] = {};
    // staging buffers for host arrays, keyed by slot
    DevBuf stage[8];
    // last retrieve, for tmr_sync's numeric check
    const int *last_status = nullptr;
    bool last_had_fit = false;
    int G = 1;  // solver schedule: masks per CTA
    int prec = TMR_PREC_FP32;
    int xk = 0;  // transform kind of the kernels: 0 FP32 1D DFT, 1 mixed, 2 FP32 2D probing DFT,
                 // 3 the matrix-vector DFT of the dense ("without FFT") solver
    void *y16 = nullptr;   // mixed precision: FP16 intensities [M][J][N]
    float *ysc = nullptr;  // and their row scales [M]
    cudaStream_t own_stream = nullptr;  // created for graph capture when the caller gave none
    // captured retrieve graph and the arguments it was captured with
    cudaGraphExec_t gexec = nullptr;
    // learned initialiser
    tmr_mlp *model = nullptr;
    float2 *Tcand = nullptr;
    unsigned *wins = nullptr;
    const void *gkey[9] = {};
    int giters = -1;
};

namespace {

enum { ST_Y = 0, ST_YDEF, ST_TOUT, ST_TIN, ST_STATUS, ST_ITERS, ST_LOSS, ST_PHI };

tmr_status halloc(tmr_handle *h, void **p, size_t bytes, const char *what)
{
    if (h->opt.workspace_limit && h->held + bytes > h->opt.workspace_limit)
        return fail(TMR_ERR_OOM, std::string(what) + ": workspace_limit exceeded");
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(TMR_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
    }
    h->held += bytes;
    return TMR_OK;
}

void hfree(tmr_handle *h, void *p, size_t bytes)
{
    if (p) {
        cudaFree(p);
        h->held -= bytes;
    }
}

// Device view of a caller array: the pointer itself when it is device memory,
// otherwise a staging buffer (copied in when `in`).
tmr_status stage(tmr_handle *h, int slot, const void *src, size_t bytes, bool in, void **dev)
{
    const int pc = pointer_class(src);
    if (pc == PTR_DEVICE) {
        *dev = const_cast<void *>(src);
        return TMR_OK;
    }
    if (pc == PTR_OTHER_DEVICE)
        return fail(TMR_ERR_INVALID_ARG, "array lives on another device than the current one");
    DevBuf &b = h->stage[slot];
    if (b.bytes < bytes) {
        hfree(h, b.p, b.bytes);
        b.p = nullptr;
        b.bytes = 0;
        tmr_status st = halloc(h, &b.p, bytes, "staging buffer");
        if (st != TMR_OK) return st;
        b.bytes = bytes;
    }
    if (in) TMR_CUDA(cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, h->stream), "copy in");
    *dev = b.p;
    return TMR_OK;
}

tmr_status unstage(tmr_handle *h, void *host, const void *dev, size_t bytes, bool *synced)
{
    if (host && dev != host) {
        TMR_CUDA(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, h->stream), "copy out");
        *synced = true;
    }
    return TMR_OK;
}

tmr_status check_launch(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) return cuda_fail(e, what);
    return TMR_OK;
}

// ---- schedule autotuner -----------------------------------------------------
std::mutex g_tune_mu;
std::map<std::string, int> g_tune_mem;

std::map<std::string, int> read_tune_file(const char *path)
{
    std::map<std::string, int> out;
    if (!path) return out;
    std::ifstream f(path);
    if (!f) return out;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string t = ss.str();
    size_t pos = 0;
    while ((pos = t.find('"', pos)) != std::string::npos) {
        const size_t end = t.find('"', pos + 1);
        if (end == std::string::npos) break;
        const std::string key = t.substr(pos + 1, end - pos - 1);
        const size_t colon = t.find(':', end);
        if (colon == std::string::npos) break;
        out[key] = std::atoi(t.c_str() + colon + 1);
        pos = colon + 1;
    }
    return out;
}

void write_tune_file(const char *path, const std::map<std::string, int> &m)
{
    if (!path) return;
    std::ofstream f(path);
    f << "{";
    bool first = true;
    for (auto &kv : m) {
        f << (first ? "\n  " : ",\n  ") << '"' << kv.first << "\": " << kv.second;
        first = false;
    }
    f << "\n}\n";
}

bool schedule_ok(int N, int J, int m, int G, int smem_optin, int prec = 0, int cost = 0)
{
    if (G <= 0 || !solver_schedule_valid(N, J, G, prec) || !solver_cost_supported(N, G, prec, cost)) return false;
    const size_t b = solver_smem_bytes(N, J, m, G, prec);
    return b > 0 && b <= (size_t)smem_optin;
}

// Time every valid schedule on synthetic rows (spectral start, a few power
// and L-BFGS iterations) and return the fastest.
tmr_status autotune(tmr_handle *h, int smem_optin, int *G_out, bool *timed)
{
    *timed = false;
    int cand[5], nc = 0;
    for (int G : {1, 2, 4, kRowSchedule, kBlueFullSchedule})
        if (schedule_ok(h->N, h->J, h->opt.m, G, smem_optin, h->xk, h->opt.cost) && (G != kRowSchedule || h->pairs) &&
            (G != kBlueFullSchedule || h->tw_alt))
            cand[nc++] = G;
    if (nc == 0) {  // the forward model and gradient still work; tmr_retrieve will refuse
        *G_out = 0;
        return TMR_OK;
    }
    if (nc == 1) {  // the only schedule: final without timing
        *G_out = cand[0];
        *timed = true;
        return TMR_OK;
    }
    const int R = 608;
    const size_t K = (size_t)h->J * h->N;
    // the timing rows are temporary device memory of the handle: under a
    // workspace_limit they must fit in what is left, else the first
    // candidate is taken untimed
    const size_t tune_bytes = sizeof(float) * R * K + sizeof(float2) * R * h->N;
    if (h->opt.workspace_limit && h->held + tune_bytes > h->opt.workspace_limit) {
        *G_out = cand[0];  // not timed: not cached either
        return TMR_OK;
    }
    float *y = nullptr;
    float2 *T = nullptr;
    if (cudaMalloc(&y, sizeof(float) * R * K) != cudaSuccess ||
        cudaMalloc(&T, sizeof(float2) * R * h->N) != cudaSuccess) {
        cudaGetLastError();
        if (y) cudaFree(y);
        return fail(TMR_ERR_OOM, "autotuner buffers");
    }
    cudaStream_t s = h->stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch_fill_synthetic(y, R * K, 12345u, s);
    SolverParams p{};
    p.masks = h->masks;
    p.tw = h->tw;
    p.y = y;
    p.T_out = T;
    p.queue = h->queue;
    p.pairs = h->pairs;
    p.pair_ctas = h->pair_ctas;
    p.M = R;
    p.N = h->N;
    p.J = h->J;
    p.iters = 6;
    p.m = h->opt.m;
    p.init = TMR_INIT_SPECTRAL;
    p.power_iters = 4;
    p.cost = h->opt.cost;
    p.clip = 2.f;
    float best = 1e30f;
    int bestG = cand[0];
    tmr_status st = TMR_OK;
    for (int c = 0; c < nc && st == TMR_OK; c++) {
        float ms = 0.f;
        p.tw = cand[c] == kBlueFullSchedule ? h->tw_alt : h->tw;
        for (int rep = 0; rep < 3; rep++) {
            cudaMemsetAsync(h->queue, 0, sizeof(unsigned) * 4, s);
            cudaEventRecord(e0, s);
            cudaError_t e = launch_solver(h->N, cand[c], p, s, nullptr);
            cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                st = cuda_fail(e, "autotuner run");
                break;
            }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms += t;  // the first run warms up
        }
        if (st == TMR_OK) {
            h->tune_codes[h->tune_n] = cand[c];
            h->tune_ms[h->tune_n] = ms / 2.f;
            h->tune_n++;
        }
        if (st == TMR_OK && ms < best) {
            best = ms;
            bestG = cand[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(y);
    cudaFree(T);
    *G_out = bestG;
    *timed = st == TMR_OK;
    return st;
}

std::string tune_key(int dev, int N, int J, int m, int prec, int cost)
{
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    char k[320];
    snprintf(k, sizeof(k), "%s|sm%d%d|N%d|J%d|m%d%s%s", prop.name, prop.major, prop.minor, N, J, m,
             prec == 1 ? "|mixed" : (prec == 2 ? "|2d" : (prec == 3 ? "|densemv" : "")),
             cost == TMR_COST_AMPLITUDE ? "|amp" : "");
    for (char *c = k; *c; c++)
        if (*c == '"' || *c == '\\') *c = '_';
    return k;
}

}  // namespace

extern "C" {

void tmr_default_options(tmr_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->m = 5;
    o->init = TMR_INIT_SPECTRAL;
    o->seed = 0;
    o->power_iters = 100;
    o->clip = 2.0;
    o->tol = 0.0;
    o->phase_iters = 100;
    o->precision = TMR_PREC_FP32;
    o->use_graph = 0;
    o->workspace_limit = 0;
    o->schedule = 0;
    o->tune_cache = nullptr;
    o->wait_spins = 1LL << 24;
    o->withhold_release = 0;
    o->probe_n1 = 0;
}

int tmr_schedule(const tmr_handle *h) { return h ? h->G : 0; }

int tmr_autotune_report(const tmr_handle *h, int *codes, float *ms, int cap)
{
    if (!h) return 0;
    for (int i = 0; i < h->tune_n && i < cap; i++) {
        if (codes) codes[i] = h->tune_codes[i];
        if (ms) ms[i] = h->tune_ms[i];
    }
    return h->tune_n;
}

tmr_status tmr_set_init_model(tmr_handle *h, tmr_mlp *model)
{
    tmr::set_last_error("");
    if (!h) return fail(TMR_ERR_INVALID_ARG, "NULL handle");
    if (model && (mlp_in(model) != h->J * h->N || mlp_out(model) != 2 * h->N))
        return fail(TMR_ERR_INVALID_ARG, "network sizes must be in = J*N, out = 2*N");
    h->model = model;
    return TMR_OK;
}

long long tmr_learned_rows(tmr_handle *h)
{
    if (!h || !h->wins) return -1;
    unsigned v = 0;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess ||
        cudaMemcpy(&v, h->wins, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return (long long)v;
}

const char *tmr_last_error(void) { return g_last_error_buf; }

size_t tmr_workspace_bytes(const tmr_handle *h) { return h ? h->held : 0; }


void tmr_destroy(tmr_handle *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    void *ptrs[] = {h->masks, h->tw, h->H, h->Zd, h->phi, h->pf_ws, h->pf_loss, h->wts, h->queue,
                    h->pf_sync, h->pf_err, h->pf_iters, h->status_scratch, h->iters_scratch,
                    h->loss_scratch, h->Tcand, h->wins, h->y16, h->ysc, h->pairs, h->tw_alt, h->incident,
                    h->krylov};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (auto &b : h->stage)
        if (b.p) cudaFree(b.p);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
}

tmr_status tmr_create(tmr_handle **out, int N, int M, int J, const void *masks,
                      const tmr_defocus_op *dop, const tmr_options *opt, void *stream)
{
    tmr::set_last_error("");
    if (!out) return fail(TMR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (N <= 0 || M < 0 || J <= 0) return fail(TMR_ERR_INVALID_ARG, "N, J must be positive and M >= 0");
    if (!masks) return fail(TMR_ERR_INVALID_ARG, "masks is NULL");
    tmr_options o;
    tmr_default_options(&o);
    if (opt) o = *opt;
    if (o.m < 1 || o.m > kMaxMem) return fail(TMR_ERR_INVALID_ARG, "opt.m must be in 1..6");
    if (o.init < TMR_INIT_RANDOM || o.init > TMR_INIT_LEARNED) return fail(TMR_ERR_INVALID_ARG, "opt.init");
    if (o.power_iters < 0 || o.phase_iters < 0 || o.tol < 0) return fail(TMR_ERR_INVALID_ARG, "negative option");
    if (o.lanczos != 0 && o.lanczos != 1) return fail(TMR_ERR_INVALID_ARG, "opt.lanczos must be 0 or 1");
    if (o.dense < 0 || o.dense > 2) return fail(TMR_ERR_INVALID_ARG, "opt.dense must be 0, 1 or 2");
    if (o.dense && (o.probe_n1 != 0 || o.precision != TMR_PREC_FP32 || !fft_supported(N)))
        return fail(TMR_ERR_UNSUPPORTED,
                    "the dense operator runs FP32 with the 1D DFT (probe_n1 0) for N a power of two in 64..4096");
    if (!(o.phase_tol >= 0.0) || !std::isfinite(o.phase_tol))
        return fail(TMR_ERR_INVALID_ARG, "opt.phase_tol must be finite and >= 0");
    if (o.cost != TMR_COST_INTENSITY && o.cost != TMR_COST_AMPLITUDE)
        return fail(TMR_ERR_INVALID_ARG, "opt.cost must be TMR_COST_INTENSITY or TMR_COST_AMPLITUDE");
    if (o.lanczos && o.power_iters > kMaxLanczos)
        return fail(TMR_ERR_INVALID_ARG, "opt.power_iters (Lanczos steps) must be at most 16 with opt.lanczos");
    if (o.wait_spins < 1 || o.wait_spins > (1LL << 40))
        return fail(TMR_ERR_INVALID_ARG, "opt.wait_spins must be in 1..2^40");
    if (o.precision != TMR_PREC_FP32 && o.precision != TMR_PREC_MIXED)
        return fail(TMR_ERR_INVALID_ARG, "opt.precision must be TMR_PREC_FP32 or TMR_PREC_MIXED");
    if (o.precision == TMR_PREC_MIXED && !mixed_supported(N))
        return fail(TMR_ERR_UNSUPPORTED, "TMR_PREC_MIXED needs N = 256, 1024, 2048 or 4096");
    if (o.probe_n1 < 0) return fail(TMR_ERR_INVALID_ARG, "opt.probe_n1 must be >= 0");
    if (o.probe_n1 != 0 && (o.precision != TMR_PREC_FP32 || N % o.probe_n1 != 0 || fft_table_2d(N, o.probe_n1, nullptr) < 0))
        return fail(TMR_ERR_UNSUPPORTED, "the 2D probing DFT needs FP32 and N = 512 (n1 = 8 or 64) or N = 4096 "
                                         "(n1 = 8, 64 or 512)");
    const int xk = o.precision == TMR_PREC_MIXED ? 1 : (o.probe_n1 ? 2 : (o.dense ? 3 : 0));
    if (!xform_supported(N))
        return fail(TMR_ERR_UNSUPPORTED, "N must be a power of two in 64..4096 or another length in 16..4096");
    if (J > kMaxMasks) return fail(TMR_ERR_UNSUPPORTED, "J must be at most 8");
    int dev = 0;
    TMR_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dop) {
        if (dop->ny <= 0 || dop->nx <= 0 || (long long)dop->ny * dop->nx != M)
            return fail(TMR_ERR_INVALID_ARG, "defocus grid ny*nx must equal M");
        if (dop->kind == TMR_DEFOCUS_SAME_GRID) {
            if (dop->n_defocus < 1 || dop->n_defocus > J * N)
                return fail(TMR_ERR_INVALID_ARG, "n_defocus must be in 1..J*N");
            if (!defocus_supported(dop->ny, dop->nx))
                return fail(TMR_ERR_UNSUPPORTED, "defocus grid sides must be powers of two, grid <= 160 KB");
        } else if (dop->kind == TMR_DEFOCUS_ANGULAR_2X) {
            if (dop->n_defocus < 1 || dop->n_defocus > 65536)
                return fail(TMR_ERR_INVALID_ARG, "n_defocus must be in 1..65536");
            if (!dop->incident) return fail(TMR_ERR_INVALID_ARG, "the 2x defocus operator needs incident fields");
            if (!dop->H && !(dop->wavelength > 0.0 && dop->pixel > 0.0 && dop->na > 0.0 && std::isfinite(dop->z_d) &&
                             std::isfinite(dop->wavelength) && std::isfinite(dop->pixel) && std::isfinite(dop->na)))
                return fail(TMR_ERR_INVALID_ARG, "wavelength, pixel and na must be positive and z_d finite");
            if (!defocus2x_supported(dop->ny, dop->nx))
                return fail(TMR_ERR_UNSUPPORTED,
                            "2x defocus grid sides must be powers of two, three ny x (nx + 1) grids "
                            "and the fit's scratch within 227 KB of shared memory");
        } else {
            return fail(TMR_ERR_INVALID_ARG, "unknown defocus kind");
        }
    }

    int smem_optin = 0;
    TMR_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "attr");
    if (o.cost == TMR_COST_AMPLITUDE && xk != 0 && xk != 3)
        return fail(TMR_ERR_UNSUPPORTED, "the amplitude cost runs on the FP32 1D transforms (precision FP32, probe_n1 0)");
    if (o.schedule != 0 && !schedule_ok(N, J, o.m, o.schedule, smem_optin, xk, o.cost))
        return fail(TMR_ERR_UNSUPPORTED,
                    "opt.schedule must be 1, 2 or 4 (dividing J), 16 (one CTA per row) or 32 (full-length "
                    "Bluestein), and fit the device");

    tmr_handle *h = new tmr_handle();
    h->N = N;
    h->M = M;
    h->J = J;
    h->opt = o;
    h->opt.tune_cache = nullptr;  // the caller's string is not kept
    h->prec = o.precision;
    h->xk = xk;
    h->stream = (cudaStream_t)stream;
    if (!h->stream && o.use_graph) {
        // the legacy default stream cannot be captured: use a blocking stream
        // of our own, which orders itself with the legacy default stream
        if (cudaStreamCreate(&h->own_stream) != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return fail(TMR_ERR_CUDA, "stream for graph capture");
        }
        h->stream = h->own_stream;
    }
    tmr_status st;
#define TRY(x)                    \
    do {                          \
        st = (x);                 \
        if (st != TMR_OK) {       \
            tmr_destroy(h);       \
            return st;            \
        }                         \
    } while (0)
    TRY(halloc(h, (void **)&h->masks, sizeof(float2) * (size_t)J * N, "masks"));
    {
        cudaError_t e = cudaMemcpy(h->masks, masks, sizeof(float2) * (size_t)J * N, cudaMemcpyDefault);
        if (e != cudaSuccess) {
            tmr_destroy(h);
            return cuda_fail(e, "copy masks");
        }
    }
    const int twn = h->xk == 2   ? fft_table_2d(N, o.probe_n1, nullptr)
                    : h->xk == 3 ? dense_mv_table(N, nullptr)
                                 : xform_table_prec(N, h->prec, nullptr);
    std::vector<float2> tw(twn > 0 ? twn : 1);
    if (h->xk == 2) fft_table_2d(N, o.probe_n1, tw.data());
    else if (h->xk == 3) dense_mv_table(N, tw.data());
    else xform_table_prec(N, h->prec, tw.data());
    TRY(halloc(h, (void **)&h->tw, sizeof(float2) * tw.size(), "twiddles"));
    if (cudaMemcpy(h->tw, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        tmr_destroy(h);
        return fail(TMR_ERR_CUDA, "copy twiddles");
    }
    TRY(halloc(h, (void **)&h->queue, sizeof(unsigned) * 4, "queue"));
    TRY(halloc(h, (void **)&h->status_scratch, sizeof(int) * (M > 0 ? M : 1), "status"));
    TRY(halloc(h, (void **)&h->iters_scratch, sizeof(int) * (M > 0 ? M : 1), "iters"));
    TRY(halloc(h, (void **)&h->loss_scratch, sizeof(float) * (M > 0 ? M : 1), "loss"));
    if (dop) {
        h->has_defocus = true;
        h->ny = dop->ny;
        h->nx = dop->nx;
        h->Nd = dop->n_defocus;
        h->dkind = dop->kind;
        const size_t P = (size_t)M;
        TRY(halloc(h, (void **)&h->H, sizeof(float2) * P, "H"));
        if (h->dkind == TMR_DEFOCUS_ANGULAR_2X) {
            TRY(halloc(h, (void **)&h->incident, sizeof(float2) * (size_t)h->Nd * N, "incident fields"));
            if (cudaMemcpy(h->incident, dop->incident, sizeof(float2) * (size_t)h->Nd * N, cudaMemcpyDefault) !=
                cudaSuccess) {
                tmr_destroy(h);
                return fail(TMR_ERR_CUDA, "copy incident fields");
            }
        }
        if (dop->H) {
            if (cudaMemcpy(h->H, dop->H, sizeof(float2) * P, cudaMemcpyDefault) != cudaSuccess) {
                tmr_destroy(h);
                return fail(TMR_ERR_CUDA, "copy H");
            }
        } else {
            cudaError_t e = h->dkind == TMR_DEFOCUS_ANGULAR_2X
                                ? launch_make_H2x(h->ny, h->nx, dop->wavelength, dop->na, dop->z_d, dop->pixel, h->H,
                                                  nullptr)
                                : launch_make_quadratic_H(h->ny, h->nx, dop->coef, h->H, nullptr);
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
            if (e != cudaSuccess) {
                tmr_destroy(h);
                return cuda_fail(e, "make H");
            }
        }
        TRY(halloc(h, (void **)&h->Zd, sizeof(float2) * (size_t)h->Nd * P, "defocus fields"));
        TRY(halloc(h, (void **)&h->phi, sizeof(double) * P, "phi"));
        TRY(halloc(h, (void **)&h->wts, sizeof(float) * P, "weights"));
        const int grid = phase_fit_grid(h->ny, h->nx, h->Nd);
        TRY(halloc(h, (void **)&h->pf_ws, sizeof(double) * phase_fit_workspace_doubles((int)P, h->Nd, o.m, grid),
                   "phase-fit workspace"));
        TRY(halloc(h, (void **)&h->pf_sync, sizeof(unsigned) * 4, "barrier"));
        TRY(halloc(h, (void **)&h->pf_err, sizeof(int) * 4, "error flag"));
        TRY(halloc(h, (void **)&h->pf_iters, sizeof(int) * 4, "phase iters"));
        TRY(halloc(h, (void **)&h->pf_loss, sizeof(double) * 4, "phase loss"));
        cudaMemset(h->pf_err, 0, sizeof(int) * 4);
    }
    // the one-CTA-per-row schedule keeps its L-BFGS pairs in tensor memory; its
    // resident CTA count (pair_ctas, which sizes the Lanczos workspace) is set
    // when that schedule can run (and is asked for or a candidate of the
    // autotuner), with a token allocation (solver_row_pair_stride is 0) that
    // marks the schedule as runnable
    if ((o.schedule == 0 || o.schedule == kRowSchedule) &&
        schedule_ok(N, J, o.m, kRowSchedule, smem_optin, h->xk, o.cost)) {
        const int ctas = solver_row_max_ctas(N, J, o.m);
        const size_t bytes = sizeof(float2) * solver_row_pair_stride(N, o.m) * (size_t)(ctas > 0 ? ctas : 0);
        if (ctas > 0 && (!o.workspace_limit || h->held + bytes <= o.workspace_limit)) {
            TRY(halloc(h, (void **)&h->pairs, bytes, "L-BFGS pair workspace"));
            h->pair_ctas = ctas;
        } else if (o.schedule == kRowSchedule) {
            tmr_destroy(h);
            return fail(TMR_ERR_OOM, "L-BFGS pair workspace of schedule 16 exceeds workspace_limit");
        }
    }
    // the other Bluestein plan's table, when that schedule can run
    if ((o.schedule == 0 || o.schedule == kBlueFullSchedule) &&
        schedule_ok(N, J, o.m, kBlueFullSchedule, smem_optin, h->xk, o.cost)) {
        const int n = xform_table_blue_full(N, nullptr);
        std::vector<float2> t2(n > 0 ? n : 1);
        xform_table_blue_full(N, t2.data());
        TRY(halloc(h, (void **)&h->tw_alt, sizeof(float2) * t2.size(), "full Bluestein table"));
        if (cudaMemcpy(h->tw_alt, t2.data(), sizeof(float2) * t2.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            tmr_destroy(h);
            return fail(TMR_ERR_CUDA, "copy full Bluestein table");
        }
    }
    // solver schedule: given, cached, or autotuned
    if (o.schedule != 0) {
        h->G = o.schedule;
    } else {
        const std::string key = tune_key(dev, N, J, o.m, h->xk, o.cost);
        int G = 0;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_mem.find(key);
            if (it != g_tune_mem.end()) G = it->second;
            if (!G && o.tune_cache) {
                auto fm = read_tune_file(o.tune_cache);
                auto f = fm.find(key);
                if (f != fm.end() && schedule_ok(N, J, o.m, f->second, smem_optin, h->xk, o.cost)) G = f->second;
            }
            if (G == kRowSchedule && !h->pairs) G = 0;  // no pair workspace here: tune again
            if (G == kBlueFullSchedule && !h->tw_alt) G = 0;
        }
        bool timed = true;  // a cached choice was timed when it was made
        if (!G) {
            TRY(autotune(h, smem_optin, &G, &timed));
            if (timed) {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                g_tune_mem[key] = G;
            }
        }
        if (o.tune_cache && G > 0 && timed) {  // the file records the choice, also one made earlier in this process
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto fm = read_tune_file(o.tune_cache);
            auto f = fm.find(key);
            if (f == fm.end() || f->second != G) {
                fm[key] = G;
                write_tune_file(o.tune_cache, fm);
            }
        }
        h->G = G;
    }
    // Lanczos vectors of the spectral start: one region per resident CTA of the
    // one-CTA-per-row schedule, else per cluster (launches are capped at 2 per SM)
    if (o.lanczos && o.power_iters > 0 && h->G > 0 &&
        (o.init == TMR_INIT_SPECTRAL || o.init == TMR_INIT_LEARNED)) {
        int nsm = 0;
        TMR_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "attr");
        int units = h->G == kRowSchedule ? h->pair_ctas : 2 * nsm;
        if (units > M) units = M > 0 ? M : 1;
        const size_t bytes = sizeof(float2) * (size_t)units * lanczos_region(N, o.power_iters);
        if (o.workspace_limit && h->held + bytes > o.workspace_limit) {
            tmr_destroy(h);
            return fail(TMR_ERR_OOM, "Lanczos workspace exceeds workspace_limit");
        }
        TRY(halloc(h, (void **)&h->krylov, bytes, "Lanczos vectors"));
        h->krylov_units = units;
    }
#undef TRY
    *out = h;
    return TMR_OK;
}

// the dense operator's matrix and scratch (opt.dense), made at the first call
static tmr_status dense_ready(tmr_handle *h)
{
    size_t bytes = 0;
    const size_t need = (h->dense.Q ? 0 : sizeof(float2) * (size_t)h->J * h->N * h->N) +
                        (h->dense.Z ? 0 : 2 * sizeof(float2) * (size_t)h->J * h->N * (h->M > 0 ? h->M : 1));
    if (h->opt.workspace_limit && h->held + need > h->opt.workspace_limit)
        return fail(TMR_ERR_OOM, "the dense operator's matrix exceeds workspace_limit");
    const cudaError_t e = dense_prepare(h->dense, h->N, h->M, h->J, h->masks, h->stream, &bytes);
    h->held += bytes;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(TMR_ERR_OOM, "dense operator matrix");
    }
    if (e != cudaSuccess) return cuda_fail(e, "dense operator");
    return TMR_OK;
}

tmr_status tmr_forward(tmr_handle *h, const void *T, float *Y)
{
    tmr::set_last_error("");
    if (!h || !T || !Y) return fail(TMR_ERR_INVALID_ARG, "NULL argument");
    const size_t MN = (size_t)h->M * h->N, MK = MN * h->J;
    void *dT, *dY;
    tmr_status st;
    if (h->opt.dense && (st = dense_ready(h)) != TMR_OK) return st;
    if ((st = stage(h, ST_TIN, T, sizeof(float2) * MN, true, &dT)) != TMR_OK) return st;
    if ((st = stage(h, ST_Y, Y, sizeof(float) * MK, false, &dY)) != TMR_OK) return st;
    if (h->opt.dense) {
        if ((st = check_launch(dense_forward(h->dense, h->opt.dense, h->N, h->M, h->J, (const float2 *)dT,
                                             (float *)dY, h->stream),
                               "dense forward")) != TMR_OK)
            return st;
    } else if ((st = check_launch(launch_forward(h->N, h->M, h->J, (const float2 *)dT, h->masks, h->tw,
                                                 (float *)dY, h->stream, h->xk), "forward kernel")) != TMR_OK)
        return st;
    bool synced = false;
    if ((st = unstage(h, Y, dY, sizeof(float) * MK, &synced)) != TMR_OK) return st;
    if (synced) TMR_CUDA(cudaStreamSynchronize(h->stream), "sync");
    return TMR_OK;
}

tmr_status tmr_grad(tmr_handle *h, const void *T, const float *Y, float *loss, void *G)
{
    tmr::set_last_error("");
    if (!h || !T || !Y) return fail(TMR_ERR_INVALID_ARG, "NULL argument");
    const size_t MN = (size_t)h->M * h->N, MK = MN * h->J;
    void *dT, *dY, *dL = nullptr, *dG = nullptr;
    tmr_status st;
    if ((st = stage(h, ST_TIN, T, sizeof(float2) * MN, true, &dT)) != TMR_OK) return st;
    if ((st = stage(h, ST_Y, Y, sizeof(float) * MK, true, &dY)) != TMR_OK) return st;
    if (loss && (st = stage(h, ST_LOSS, loss, sizeof(float) * h->M, false, &dL)) != TMR_OK) return st;
    if (G && (st = stage(h, ST_TOUT, G, sizeof(float2) * MN, false, &dG)) != TMR_OK) return st;
    if (h->opt.dense) {
        if ((st = dense_ready(h)) != TMR_OK) return st;
        if ((st = check_launch(dense_grad(h->dense, h->opt.dense, h->N, h->M, h->J, (const float2 *)dT,
                                          (const float *)dY, (float *)dL, (float2 *)dG, h->opt.cost, h->stream),
                               "dense gradient")) != TMR_OK)
            return st;
    } else if ((st = check_launch(launch_grad(h->N, h->M, h->J, (const float2 *)dT, h->masks, h->tw,
                                       (const float *)dY, (float *)dL, (float2 *)dG, h->stream, h->xk,
                                       h->opt.cost),
                                              "gradient kernel")) != TMR_OK)
        return st;
    bool synced = false;
    if (loss && (st = unstage(h, loss, dL, sizeof(float) * h->M, &synced)) != TMR_OK) return st;
    if (G && (st = unstage(h, G, dG, sizeof(float2) * MN, &synced)) != TMR_OK) return st;
    if (synced) TMR_CUDA(cudaStreamSynchronize(h->stream), "sync");
    return TMR_OK;
}

// floats of one set of defocus images: [Nd][M] (kind 0) or [Nd][4 M] (kind 1)
static size_t ydef_floats(const tmr_handle *h)
{
    return (size_t)h->Nd * h->M * (h->dkind == TMR_DEFOCUS_ANGULAR_2X ? 4 : 1);
}

// Zd <- the fields c_n of T: probe patterns (kind 0) or incident fields (kind 1)
static cudaError_t defocus_fields(tmr_handle *h, const float2 *dT)
{
    if (h->dkind == TMR_DEFOCUS_ANGULAR_2X)
        return launch_incident_fields(h->M, h->N, h->Nd, dT, h->incident, h->Zd, h->stream);
    return launch_fields(h->N, h->M, h->J, h->Nd, dT, h->masks, h->tw, h->Zd, h->stream, h->xk);
}

static tmr_status run_phase_fit(tmr_handle *h, const float2 *Tin, const float *dYdef, double *dphi,
                                float2 *Tout)
{
    // weights of the constant-phase normalisation: row energies of T_est
    TMR_CUDA(launch_row_energy(h->N, h->M, Tin, h->wts, h->stream), "row energy");
    TMR_CUDA(cudaMemsetAsync(h->pf_sync, 0, sizeof(unsigned) * 4, h->stream), "memset");
    TMR_CUDA(cudaMemsetAsync(h->pf_err, 0, sizeof(int) * 4, h->stream), "memset");
    PhaseFitParams p{};
    p.Zd = h->Zd;
    p.Ydef = dYdef;
    p.H = h->H;
    p.wts = h->wts;
    p.phi = dphi;
    p.Nd = h->Nd;
    p.ny = h->ny;
    p.nx = h->nx;
    p.iters = h->opt.phase_iters;
    p.m = h->opt.m;
    p.ws = h->pf_ws;
    p.sync = h->pf_sync;
    p.err = h->pf_err;
    p.iters_done = h->pf_iters;
    p.loss_out = h->pf_loss;
    p.wait_spins = h->opt.wait_spins;
    p.withhold_release = h->opt.withhold_release != 0;
    p.kind = h->dkind;
    p.tol = h->opt.phase_tol;
    TMR_CUDA(launch_phase_fit(p, h->stream), "phase-fit kernel");
    h->fit_ran = true;
    if (Tout) TMR_CUDA(launch_apply_phase(h->N, h->M, dphi, Tin, Tout, h->stream), "apply phase");
    return TMR_OK;
}

static tmr_status retrieve_impl(tmr_handle *h, const void *T_init, const float *y, const float *y_def,
                                int iters, void *T_out, int *row_status, int *row_iters,
                                float *row_loss)
{
    tmr::set_last_error("");
    if (!h || !y || !T_out) return fail(TMR_ERR_INVALID_ARG, "NULL argument");
    if (iters < 0) return fail(TMR_ERR_INVALID_ARG, "iters must be >= 0");
    if (h->opt.dense && y_def)
        return fail(TMR_ERR_UNSUPPORTED, "the dense (without FFT) solver runs without the phase-offset fit");
    const bool fit = y_def != nullptr;
    if (fit && !h->has_defocus) return fail(TMR_ERR_INVALID_ARG, "y_def given but the handle has no defocus operator");
    {
        int dev = 0, smem_optin = 0;
        TMR_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
        TMR_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "attr");
        if (!schedule_ok(h->N, h->J, h->opt.m, h->G, smem_optin, h->xk, h->opt.cost))
            return fail(TMR_ERR_UNSUPPORTED,
                        "per-row state of this (N, J, m) does not fit in shared memory: lower opt.m");
    }
    const size_t MN = (size_t)h->M * h->N, MK = MN * h->J;
    tmr_status st;
    void *dy, *dT, *dTin = nullptr, *dYd = nullptr, *dS, *dI, *dL;
    if ((st = stage(h, ST_Y, y, sizeof(float) * MK, true, &dy)) != TMR_OK) return st;
    if (T_init && (st = stage(h, ST_TIN, T_init, sizeof(float2) * MN, true, &dTin)) != TMR_OK) return st;
    if (fit && (st = stage(h, ST_YDEF, y_def, sizeof(float) * ydef_floats(h), true, &dYd)) != TMR_OK)
        return st;
    if ((st = stage(h, ST_TOUT, T_out, sizeof(float2) * MN, false, &dT)) != TMR_OK) return st;
    dS = h->status_scratch;
    dI = h->iters_scratch;
    dL = h->loss_scratch;
    if (row_status && (st = stage(h, ST_STATUS, row_status, sizeof(int) * h->M, false, &dS)) != TMR_OK) return st;
    if (row_iters && (st = stage(h, ST_ITERS, row_iters, sizeof(int) * h->M, false, &dI)) != TMR_OK) return st;
    if (row_loss && (st = stage(h, ST_LOSS, row_loss, sizeof(float) * h->M, false, &dL)) != TMR_OK) return st;

    const bool learned = h->opt.init == TMR_INIT_LEARNED && !T_init;
    if (learned) {
        if (!h->model) return fail(TMR_ERR_INVALID_ARG, "TMR_INIT_LEARNED needs tmr_set_init_model");
        if (!h->Tcand) {
            if ((st = halloc(h, (void **)&h->Tcand, sizeof(float2) * (MN ? MN : 1), "proposed starts")) != TMR_OK)
                return st;
            if ((st = halloc(h, (void **)&h->wins, sizeof(unsigned) * 4, "win counter")) != TMR_OK) return st;
        }
        TMR_CUDA(cudaMemsetAsync(h->wins, 0, sizeof(unsigned) * 4, h->stream), "memset");
        const int CH = 2048;  // rows per network batch
        for (int r0 = 0; r0 < h->M; r0 += CH) {
            const int B = h->M - r0 < CH ? h->M - r0 : CH;
            TMR_CUDA(mlp_propose(h->model, (const float *)dy + (size_t)r0 * h->J * h->N, B, h->N, h->J,
                                 h->Tcand + (size_t)r0 * h->N, h->stream),
                     "learned proposals");
        }
    }
    SolverParams p{};
    p.T_cand = learned ? h->Tcand : nullptr;
    // the proposal seeds the power iteration; without one, the solver keeps
    // per row whichever of the proposal and the random start has the lower loss
    p.seed_from_cand = learned && h->opt.power_iters > 0 ? 1 : 0;
    p.judge_cand = learned && h->opt.power_iters == 0 ? 1 : 0;
    p.cand_wins = learned ? h->wins : nullptr;
    p.masks = h->masks;
    p.tw = h->G == kBlueFullSchedule ? h->tw_alt : h->tw;
    p.y = (const float *)dy;
    p.T_init = (const float2 *)dTin;
    p.T_out = (float2 *)dT;
    p.row_status = (int *)dS;
    p.row_iters = (int *)dI;
    p.row_loss = (float *)dL;
    p.Zd = nullptr;  // the fit's fields are made from the final T (below)
    p.queue = h->queue;
    p.pairs = h->pairs;
    p.pair_ctas = h->pair_ctas;
    p.lanczos = h->opt.lanczos;
    p.cost = h->opt.cost;
    p.krylov = h->krylov;
    p.krylov_units = h->krylov_units;
    p.Nd = 0;
    p.M = h->M;
    p.N = h->N;
    p.J = h->J;
    p.iters = iters;
    p.m = h->opt.m;
    p.init = learned ? (h->opt.power_iters > 0 ? TMR_INIT_SPECTRAL : TMR_INIT_RANDOM) : h->opt.init;
    p.power_iters = h->opt.power_iters;
    p.seed = h->opt.seed;
    p.clip = (float)h->opt.clip;
    p.tol = h->opt.tol;
    p.prec = h->xk;
    if (h->prec == TMR_PREC_MIXED) {
        if (!h->y16) {
            if ((st = halloc(h, &h->y16, 2 * (MK ? MK : 1), "FP16 intensities")) != TMR_OK) return st;
            if ((st = halloc(h, (void **)&h->ysc, sizeof(float) * (h->M ? h->M : 1), "row scales")) != TMR_OK)
                return st;
        }
        p.y16 = h->y16;
        p.ysc = h->ysc;
    }
    // the whole retrieve on the stream: (FP16 packing,) solver, then the phase-offset fit
    auto enqueue = [&]() -> tmr_status {
        if (h->prec == TMR_PREC_MIXED)
            TMR_CUDA(launch_pack_f16(h->M, (size_t)h->J * h->N, (const float *)dy, h->y16, h->ysc, h->stream),
                     "FP16 packing");
        TMR_CUDA(cudaMemsetAsync(h->queue, 0, sizeof(unsigned) * 4, h->stream), "memset");
        TMR_CUDA(launch_solver(h->N, h->G, p, h->stream, nullptr), "solver kernel");
        if (fit) {
            TMR_CUDA(defocus_fields(h, (const float2 *)dT), "fields kernel");
            tmr_status s2 = run_phase_fit(h, (const float2 *)dT, (const float *)dYd, h->phi, (float2 *)dT);
            if (s2 != TMR_OK) return s2;
        }
        return TMR_OK;
    };
    const bool all_device = dy == y && dT == T_out && (!T_init || dTin == T_init) &&
                            (!fit || dYd == y_def) && (!row_status || dS == row_status) &&
                            (!row_iters || dI == row_iters) && (!row_loss || dL == row_loss);
    if (h->opt.use_graph && all_device) {
        const void *key[9] = {dy, dT, dTin, dYd, dS, dI, dL, (const void *)(size_t)fit, nullptr};
        bool same = h->gexec && h->giters == iters;
        for (int i = 0; i < 9 && same; i++) same = h->gkey[i] == key[i];
        if (!same) {
            if (h->gexec) {
                cudaGraphExecDestroy(h->gexec);
                h->gexec = nullptr;
            }
            TMR_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
            const tmr_status sc = enqueue();
            cudaGraph_t graph = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(h->stream, &graph);
            if (sc != TMR_OK) {
                if (graph) cudaGraphDestroy(graph);
                return sc;
            }
            if (ec != cudaSuccess) return cuda_fail(ec, "end capture");
            const cudaError_t ei = cudaGraphInstantiate(&h->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (ei != cudaSuccess) {
                h->gexec = nullptr;
                return cuda_fail(ei, "graph instantiate");
            }
            for (int i = 0; i < 9; i++) h->gkey[i] = key[i];
            h->giters = iters;
        }
        TMR_CUDA(cudaGraphLaunch(h->gexec, h->stream), "graph launch");
    } else {
        if ((st = enqueue()) != TMR_OK) return st;
    }
    h->last_status = (const int *)dS;
    h->last_had_fit = fit;
    bool synced = false;
    if ((st = unstage(h, T_out, dT, sizeof(float2) * MN, &synced)) != TMR_OK) return st;
    if (row_status && (st = unstage(h, row_status, dS, sizeof(int) * h->M, &synced)) != TMR_OK) return st;
    if (row_iters && (st = unstage(h, row_iters, dI, sizeof(int) * h->M, &synced)) != TMR_OK) return st;
    if (row_loss && (st = unstage(h, row_loss, dL, sizeof(float) * h->M, &synced)) != TMR_OK) return st;
    if (synced) TMR_CUDA(cudaStreamSynchronize(h->stream), "sync");
    return TMR_OK;
}

tmr_status tmr_retrieve(tmr_handle *h, const float *y, const float *y_def, int iters, void *T_out,
                        int *row_status, int *row_iters, float *row_loss)
{
    return retrieve_impl(h, nullptr, y, y_def, iters, T_out, row_status, row_iters, row_loss);
}

tmr_status tmr_retrieve_from(tmr_handle *h, const void *T_init, const float *y, const float *y_def,
                             int iters, void *T_out, int *row_status, int *row_iters, float *row_loss)
{
    if (!T_init) return fail(TMR_ERR_INVALID_ARG, "T_init is NULL");
    return retrieve_impl(h, T_init, y, y_def, iters, T_out, row_status, row_iters, row_loss);
}

tmr_status tmr_defocus_forward(tmr_handle *h, const void *T, float *Y_def)
{
    tmr::set_last_error("");
    if (h && h->opt.dense) return fail(TMR_ERR_UNSUPPORTED, "the dense operator runs without the defocus calls");
    if (!h || !T || !Y_def) return fail(TMR_ERR_INVALID_ARG, "NULL argument");
    if (!h->has_defocus) return fail(TMR_ERR_UNSUPPORTED, "handle has no defocus operator");
    const size_t MN = (size_t)h->M * h->N;
    void *dT, *dY;
    tmr_status st;
    if ((st = stage(h, ST_TIN, T, sizeof(float2) * MN, true, &dT)) != TMR_OK) return st;
    if ((st = stage(h, ST_YDEF, Y_def, sizeof(float) * ydef_floats(h), false, &dY)) != TMR_OK) return st;
    TMR_CUDA(defocus_fields(h, (const float2 *)dT), "fields kernel");
    TMR_CUDA(h->dkind == TMR_DEFOCUS_ANGULAR_2X
                 ? launch_defocus_forward2x(h->ny, h->nx, h->Nd, h->Zd, h->H, (float *)dY, h->stream)
                 : launch_defocus_forward(h->ny, h->nx, h->Nd, h->Zd, h->H, nullptr, nullptr, (float *)dY, h->stream),
             "defocus kernel");
    bool synced = false;
    if ((st = unstage(h, Y_def, dY, sizeof(float) * ydef_floats(h), &synced)) != TMR_OK) return st;
    if (synced) TMR_CUDA(cudaStreamSynchronize(h->stream), "sync");
    return TMR_OK;
}

tmr_status tmr_defocus_fit(tmr_handle *h, const void *T_est, const float *y_def, double *phi, void *T_out)
{
    tmr::set_last_error("");
    if (h && h->opt.dense) return fail(TMR_ERR_UNSUPPORTED, "the dense operator runs without the defocus calls");
    if (!h || !T_est || !y_def) return fail(TMR_ERR_INVALID_ARG, "NULL argument");
    if (!h->has_defocus) return fail(TMR_ERR_UNSUPPORTED, "handle has no defocus operator");
    const size_t MN = (size_t)h->M * h->N;
    void *dT, *dY, *dP = nullptr, *dO = nullptr;
    tmr_status st;
    if ((st = stage(h, ST_TIN, T_est, sizeof(float2) * MN, true, &dT)) != TMR_OK) return st;
    if ((st = stage(h, ST_YDEF, y_def, sizeof(float) * ydef_floats(h), true, &dY)) != TMR_OK) return st;
    if (phi && (st = stage(h, ST_PHI, phi, sizeof(double) * h->M, false, &dP)) != TMR_OK) return st;
    if (T_out && (st = stage(h, ST_TOUT, T_out, sizeof(float2) * MN, false, &dO)) != TMR_OK) return st;
    TMR_CUDA(defocus_fields(h, (const float2 *)dT), "fields kernel");
    if ((st = run_phase_fit(h, (const float2 *)dT, (const float *)dY, dP ? (double *)dP : h->phi,
                            (float2 *)dO)) != TMR_OK)
        return st;
    h->last_status = nullptr;  // no rows were solved: tmr_sync checks the fit's flag only
    h->last_had_fit = true;
    bool synced = false;
    if (phi && (st = unstage(h, phi, dP, sizeof(double) * h->M, &synced)) != TMR_OK) return st;
    if (T_out && (st = unstage(h, T_out, dO, sizeof(float2) * MN, &synced)) != TMR_OK) return st;
    if (synced) TMR_CUDA(cudaStreamSynchronize(h->stream), "sync");
    return TMR_OK;
}

tmr_status tmr_phase_fit_report(tmr_handle *h, double *loss, int *iters)
{
    tmr::set_last_error("");
    if (!h) return fail(TMR_ERR_INVALID_ARG, "NULL handle");
    if (!h->has_defocus) return fail(TMR_ERR_UNSUPPORTED, "handle has no defocus operator");
    if (!h->fit_ran) return fail(TMR_ERR_INVALID_ARG, "no phase-offset fit has run on this handle");
    TMR_CUDA(cudaStreamSynchronize(h->stream), "sync");
    if (loss) TMR_CUDA(cudaMemcpy(loss, h->pf_loss, sizeof(double), cudaMemcpyDeviceToHost), "read loss");
    if (iters) TMR_CUDA(cudaMemcpy(iters, h->pf_iters, sizeof(int), cudaMemcpyDeviceToHost), "read iterations");
    return TMR_OK;
}

tmr_status tmr_sync(tmr_handle *h, double timeout_s)
{
    tmr::set_last_error("");
    if (!h) return fail(TMR_ERR_INVALID_ARG, "NULL handle");
    const auto t0 = std::chrono::steady_clock::now();
    while (true) {
        cudaError_t e = cudaStreamQuery(h->stream);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(e, "stream");
        if (timeout_s > 0) {
            const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (el > timeout_s) return fail(TMR_ERR_TIMEOUT, "work still running after the timeout");
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    if (h->last_had_fit && h->pf_err) {
        int err = 0;
        TMR_CUDA(cudaMemcpy(&err, h->pf_err, sizeof(int), cudaMemcpyDeviceToHost), "read error flag");
        if (err) return fail(TMR_ERR_TIMEOUT, "phase-offset fit: grid barrier timed out");
    }
    if (h->last_status && h->M > 0 && is_device_ptr(h->last_status)) {
        std::vector<int> st(h->M);
        TMR_CUDA(cudaMemcpy(st.data(), h->last_status, sizeof(int) * h->M, cudaMemcpyDeviceToHost), "read status");
        for (int v : st)
            if (v == TMR_ROW_NUMERIC) return fail(TMR_ERR_NUMERIC, "a row reported non-finite values");
    }
    return TMR_OK;
}

}  // extern "C"
