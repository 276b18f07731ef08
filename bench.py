"""Benchmark: TM retrieval rows/s on the plain paper-scale workload (N=2048 input
modes, M=8192 output pixels on a 128x64 grid, J=4 masks, mode-model fiber TM
with R=1100 modes, Poisson noise at 1e4 photons/pixel, spectral start with 100
power iterations, 100 L-BFGS iterations, then the defocus phase-offset fit on 50
patterns with 100 L-BFGS iterations).

One step = one tmr_retrieve call over the whole TM with inputs resident in HBM.
Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TM rows/s to fidelity>=0.99 (plain vs learned-init+mixed), % of roofline"
UNIT = "rows/s"
WORKLOAD = "plain N=2048 M=8192 (128x64) J=4 modes R=1100 Poisson 1e4"
N_SM_NOMINAL = 152
# measured dense bf16 burst (cuBLAS) of this GPU type, for the tensor-pipe fraction
try:
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as _f:
        MEASURED_BF16_TFLOPS = float(json.load(_f)["bf16_tflops"])
except (OSError, KeyError, ValueError):
    MEASURED_BF16_TFLOPS = 1900.0  # fallback figure
try:
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as _f:
        MEASURED_HBM_GBS = float(json.load(_f)["hbm_gbs"])
except (OSError, KeyError, ValueError):
    MEASURED_HBM_GBS = 6800.0  # fallback figure
# --workload plain (default: the headline line) or batching (uneven convergence
# at a non-power-of-two length, Bluestein transforms, per-row early exit)
WORKLOADS = {
    "plain": dict(N=2048, J=4, R=1100, ny=128, nx=64, photons=1e4, iters=100, tol=0.0,
                  desc=WORKLOAD),
    "batching": dict(N=2286, J=4, R=1100, ny=128, nx=64, photons=(1e3, 1e5), iters=300, tol=1e-7,
                     desc="batching N=2286 M=8192 (128x64) J=4 modes R=1100 Poisson per-row "
                          "log-uniform 1e3..1e5, early exit 1e-7, cap 300"),
    "precision": dict(N=4096, J=4, R=2200, ny=128, nx=128, photons=1e4, iters=100, tol=0.0,
                      desc="precision N=4096 M=16384 (128x128) J=4 modes R=2200 Poisson 1e4"),
    # the step starts from camera frames: half-sampling and the 99.9 % fiber
    # mask (Sec. 2.2), then the plain retrieval of the rows inside the mask
    # failed-row fraction against J with the 2D probing DFT (64 x 64 modes)
    "jsweep": dict(N=4096, J=8, R=2200, ny=64, nx=64, photons=None, iters=200, tol=0.0,
                   desc="jsweep: N=4096 (64x64 2D probing DFT), M=4096, J=3..8, noiseless"),
    # the paper's Table 1 comparison: the probing operator by FFTs against the
    # explicit dense matrix ("without FFT") on 1024 rows (32 x 32 pixels), J = 8
    "dense": dict(N=4096, J=8, R=2200, ny=32, nx=32, photons=None, iters=100, tol=0.0,
                  desc="dense: N=4096, M=1024 (32x32), J=8, modes R=2200, noiseless; FFT vs explicit Q"),
    "camera": dict(N=2048, J=4, R=1100, ny=128, nx=64, photons=3000.0, iters=100, tol=0.0,
                   camera=dict(radius=0.45, leak=1e-3, energy_frac=0.999),
                   desc="camera: 8192 uint16 probe frames + 50 defocus frames of 256x128 pixels, "
                        "fiber disc (radius 0.45 x 64 half-grid pixels) -> half-sampling + 99.9 % "
                        "fiber mask -> retrieval N=2048 J=4 modes R=1100 Poisson 3000 counts"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plain", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "mixed"],
                    help="mixed: FP16 intensities, BF16 pairs, tensor-core split-BF16 DFT "
                         "stages, last 10 iterations FP32 (N = 256 or 4096)")
    ap.add_argument("--iters", type=int, default=None, help="L-BFGS iterations (cap); default per workload")
    ap.add_argument("--start", default="lanczos", choices=["lanczos", "power"],
                    help="spectral start: Lanczos steps (default) or the power iteration")
    ap.add_argument("--power-iters", type=int, default=None,
                    help="operator products of the spectral start (default 16 Lanczos steps, 100 power)")
    ap.add_argument("--phase-iters", type=int, default=100)
    ap.add_argument("--phase-tol", type=float, default=1e-4,
                    help="stop the phase-offset fit once an accepted step lowers its loss by at most "
                         "this fraction (0: only the iteration cap)")
    ap.add_argument("--rows", type=int, default=None, help="override M (grid kept 128 wide)")
    ap.add_argument("--schedule", type=int, default=0,
                    help="solver schedule code (0: the autotuner's choice; a profiler's per-launch overhead "
                         "can sway that choice, so profiled runs pin the schedule the plain run reports)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip the short-budget sweep to the 0.99 bar")
    ap.add_argument("--no-batching", action="store_true",
                    help="skip the batching workload's line that the default plain run measures in a child "
                         "run (also skipped with --no-sweep, which profiled runs pass)")
    ap.add_argument("--no-arms", action="store_true",
                    help="skip the metric's second half (mixed precision and the learned start, "
                         "with the network trained in this run)")
    args = ap.parse_args()
    if args.iters is None:
        args.iters = WORKLOADS[args.workload]["iters"]
    if args.power_iters is None:
        args.power_iters = 16 if args.start == "lanczos" else 100
    args.lanczos = 1 if args.start == "lanczos" else 0
    return args


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest x over all ranks (the slowest rank's time); x itself at world 1."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def batching_child_line(timeout_s: float = 600.0) -> dict:
    """The batching workload (N = 2286 through split-output Bluestein
    transforms, per-row photon levels from 1e3 to 1e5, early exit at a relative
    loss change of 1e-7, the whole matrix in one persistent launch replayed
    from a captured graph) timed by a child run of this script on the same
    GPU, 3 warm-up and 2 timed steps; the fields of its line that the default
    plain line carries beside the headline."""
    cmd = [sys.executable, os.path.abspath(__file__), "--workload", "batching", "--steps", "2", "--warmup", "3",
           "--no-cpu-baseline", "--no-e2e", "--no-sweep", "--no-arms"]
    env = {k: v for k, v in os.environ.items()
           if k not in ("RANK", "LOCAL_RANK", "WORLD_SIZE", "LOCAL_WORLD_SIZE", "MASTER_ADDR", "MASTER_PORT")}
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s, env=env)
        lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
        if r.returncode != 0 or not lines:
            return {"error": f"child exited {r.returncode}: {r.stderr.strip()[-300:]}"}
        c = json.loads(lines[-1])
        roof = c.get("roofline", {})
        return {"workload": c["config"]["workload"], "value": c["value"], "unit": c["unit"],
                "ms_per_step": c["ms_per_step"], "steps": c["steps"], "warmup": c["warmup"],
                "row_iters_mean": c["config"].get("row_iters_mean"),
                "row_iters_max": c["config"].get("row_iters_max"),
                "schedule": c.get("schedule"), "fidelity": c.get("fidelity"),
                "roofline": {k: roof.get(k) for k in ("kernel", "achieved", "peak", "unit", "frac", "solver_ms")},
                "clocks": c.get("clocks"), "gpu_launches": c.get("gpu_launches")}
    except (OSError, ValueError, KeyError, subprocess.TimeoutExpired) as e:
        return {"error": f"{type(e).__name__}: {e}"[:300]}


def job_rows_per_s(rows_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job throughput: every rank's rows over the slowest rank's time."""
    return world * rows_per_rank / seconds


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- algorithmic work
def fft_flops(N: int) -> float:
    """5 N log2 N per complex FFT of length N (standard convention)."""
    return 5.0 * N * math.log2(N)


def solver_flops_per_row(N, J, m, iters, power_iters, lanczos=0) -> float:
    """Algorithmic FP32 flops of one row: the spectral start's products with A
    (power iterations or Lanczos steps), the gradient at the start, and the
    L-BFGS iterations (two FFT batches each, elementwise work, two-loop).  A
    Lanczos step j also orthogonalises against its j + 1 vectors by two
    passes of a complex dot product and an update (32 (j + 1) N flops), in
    all 16 k (k + 1) N for k steps.  The FFT count follows the 5 N log2 N
    convention for every N, also where the library evaluates a length-N DFT
    through longer FFTs (Bluestein).  iters may be the sum of the iterations
    of several rows (then add the start once per row)."""
    K = J * N
    f_batch = J * fft_flops(N)
    f_power = 2 * f_batch + 16 * K
    f_eval = 2 * f_batch + 16 * K
    f_iter = 2 * f_batch + 30 * K + 16 * m * N
    f_gs = 16 * power_iters * (power_iters + 1) * N if lanczos else 0
    return power_iters * f_power + f_gs + f_eval + iters * f_iter


def solver_flops(N, J, m, row_iters, power_iters, lanczos=0) -> float:
    """Algorithmic flops of a launch whose rows ran row_iters iterations each."""
    rows = len(row_iters)
    start = solver_flops_per_row(N, J, m, 0, power_iters, lanczos)
    per_iter = solver_flops_per_row(N, J, m, 1, 0) - solver_flops_per_row(N, J, m, 0, 0)
    return rows * start + per_iter * float(np.sum(row_iters))


def fp32_peak_tflops(n_sm: int, mhz: float) -> float:
    return n_sm * 128 * 2 * mhz * 1e6 / 1e12


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"tmr_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx.append(float(parts[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[4:8]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- reference arm
def cpu_oracle_sample(W, M, iters, power_iters, rows_n, seed=0, keep=None, lanczos=0):
    """Time the FP64 oracle on rows_n sampled rows of workload W.  Returns
    (rows/s, seconds, threads, description); when keep is a dict it receives
    the sample (intensities rounded to float32, the masks, the true rows and
    the oracle's rows) for a comparison with the GPU on the same inputs."""
    import oracle
    import synth
    N, J, R = W["N"], W["J"], W["R"]
    oracle.build()
    rows = synth.sample_rows(M, rows_n, seed=1)
    # the sampled rows of the same fiber: regenerate T and keep the rows
    T = synth.tm_modes(M, N, R, seed=seed, dtype=np.complex64)[rows].astype(np.complex128)
    _, d = synth.mask_phases(J, N, seed=seed)
    d = d.astype(np.complex64).astype(np.complex128)
    Y = oracle.forward(T, d)
    ph = synth.row_photons(dict(photons=W["photons"]), M, seed=seed)[rows]
    Y = synth.shot_noise(Y, synth.photon_scale(Y.mean(), ph), seed=seed, row_ids=rows)
    Y = Y.astype(np.float32)  # the values a float32 caller would pass
    t0 = time.perf_counter()
    Tr, _, _, _ = oracle.retrieve_rows(Y, d, iters, init="lanczos" if lanczos else "spectral",
                                       power_iters=power_iters, clip=2.0, tol=W["tol"], seed=seed)
    dt = time.perf_counter() - t0
    fid = oracle.fidelity_rows(Tr, T)
    if keep is not None:
        keep.update(Y=Y, d=d, T=T, Tr=Tr, fid=fid)
    desc = (f"{len(rows)} sampled rows of the workload, Algorithm 1 only ({power_iters} "
            f"{'Lanczos' if lanczos else 'power'} + "
            f"{iters} L-BFGS iterations, naive O(N^2) DFT, FP64, OpenMP over rows); the global "
            f"phase-offset fit is not in the sample; mean fidelity {fid.mean():.4f}")
    return len(rows) / dt, dt, oracle.num_threads(), desc


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    W = WORKLOADS[args.workload]
    M = args.rows or W["ny"] * W["nx"]
    rows_per_step = max(1, min(16, os.cpu_count() or 8))
    vals = []
    for s in range(args.warmup + args.steps):
        v, dt, cores, desc = cpu_oracle_sample(W, M, args.iters, args.power_iters,
                                               rows_per_step, seed=0, lanczos=args.lanczos)
        if s >= args.warmup:
            vals.append((v, dt))
    value = float(np.mean([v for v, _ in vals]))
    ms = float(np.mean([dt for _, dt in vals])) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": W["desc"], "iters": args.iters, "power_iters": args.power_iters,
                       "start": args.start, "rows_per_step": rows_per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- the metric's second half
def fidelity_rows_t(A, B):
    """|<a, b>| / (||a|| ||b||) per row of two complex device tensors (0 for a zero row)."""
    ip = (A.conj() * B).sum(1).abs()
    den = A.abs().pow(2).sum(1).sqrt() * B.abs().pow(2).sum(1).sqrt()
    return (ip / den.clamp_min(1e-30)) * (den > 0)


def timed_retrieve(tmr, torch, h, y, y_def, iters, T_out, stream):
    """One warm run (graph capture, staging), then one run timed with CUDA
    events on the handle's stream; milliseconds."""
    tmr.tmr_retrieve(h, y, y_def, iters, T_out)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tmr.tmr_retrieve(h, y, y_def, iters, T_out)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def sweep_to_099(tmr, torch, make_handle, y, y_def, Tg, ref_frac, stream, P_list, I_list, world):
    """For every start length P (a handle from make_handle(P)) the smallest
    L-BFGS budget I of I_list whose retrieve (phase fit included) reaches mean
    fidelity >= 0.99 with the fraction of rows >= 0.99 within 0.5 % of
    ref_frac, timed; returns (fastest passing entry or None, all passing)."""
    M, N = Tg.shape
    T_out = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    passing = []
    for P in P_list:
        h = make_handle(P)
        try:
            for it in I_list:
                ms = timed_retrieve(tmr, torch, h, y, y_def, it, T_out, stream)
                f = fidelity_rows_t(T_out, Tg).float().cpu().numpy()
                if f.mean() >= 0.99 and np.mean(f >= 0.99) >= ref_frac - 0.005:
                    passing.append({"power_iters": P, "iters": it, "value": world * M / (ms / 1e3),
                                    "unit": UNIT, "ms_per_step": ms, "mean": float(f.mean()),
                                    "frac_ge_0.99": float(np.mean(f >= 0.99)),
                                    "products": P + it})
                    break
        finally:
            h.close()
    best = dict(max(passing, key=lambda r: r["value"])) if passing else None
    return best, passing


def second_half_arms(tmr, torch, synth, N, M, J, R, m, d, dop, photons, phase_iters, stream, world, iters,
                     power_iters, keep=None, lanczos=0, phase_tol=0.0):
    """The metric's second half on the learned-initialiser workload (the plain
    workload's fiber model drawn as a family: shared input mode basis V, own
    coupling and phases): the network (J N -> 1024 -> 1024 -> 2 N, GELU, BF16
    products on the tensor cores) is trained here on the rows the plain method
    retrieves from the family's 25 training fibers (8 epochs, batch 256,
    phase-invariant loss), then four arms -- spectral and learned start, FP32
    and mixed precision -- run on the held-out fiber 101 with the phase fit:
    rows/s at the configured budget and the fastest (power, L-BFGS) budget that
    meets the 0.99 bar (the start: Lanczos steps when lanczos, else power
    iterations).  Also the network's inference throughput against the
    measured BF16 peak, and (keep: the CPU-baseline sample) each arm's
    fidelity difference to the FP64 oracle on the oracle's sampled rows."""
    from paper_2302_13524_gb300 import learned_init as li
    cfg = synth.CONFIGS["learned"]
    dg = torch.from_numpy(d).cuda()
    out = {"workload": f"learned: family of mode-model fibers (N={N}, M={M}, J={J}, R={R}, shared input "
                       f"basis), {len(cfg['train_fibers'])} training fibers, held-out fiber "
                       f"{cfg['test_fibers'][0]}, Poisson {photons:g}"}
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        gen = torch.Generator(device="cuda")
        gen.manual_seed(4242)
        Xs, Ts = [], []
        with tmr.tmr_create(N, M, J, dg, None, dict(init="spectral", power_iters=16, lanczos=1, m=m),
                            stream=stream.cuda_stream) as hd:
            for f in cfg["train_fibers"]:
                _, yf = li.fiber_data(hd, synth.tm_family_device(M, N, R, f, 0), photons, gen)
                That = torch.empty((M, N), dtype=torch.complex64, device="cuda")
                tmr.tmr_retrieve(hd, yf, None, cfg["iters"], That)
                Xs.append(li.features(yf))
                Ts.append(li.targets(That))
                del yf
        X, Tt = torch.cat(Xs), torch.cat(Ts)
        del Xs, Ts
        stream.synchronize()
        t_data = time.perf_counter() - t0
        h1, h2 = cfg["widths"]
        model = tmr.tmr_mlp_create(J * N, h1, h2, 2 * N, seed=0, stream=stream.cuda_stream)
        t0 = time.perf_counter()
        hist = li.train(model, X, Tt, 8, 256, 3e-4)
        stream.synchronize()
        t_train = time.perf_counter() - t0
        out["training"] = {"rows": int(X.shape[0]), "epochs": 8, "batch": 256, "lr": 3e-4,
                           "loss": "phase-invariant", "loss_per_epoch": [round(v, 5) for v in hist],
                           "seconds_data": t_data, "seconds_train": t_train}
        del X, Tt
        torch.cuda.empty_cache()
        # the held-out fiber with its probe and defocus intensities
        Tg = synth.tm_family_device(M, N, R, cfg["test_fibers"][0], 0)
        with tmr.tmr_create(N, M, J, dg, dop, dict(init="spectral", m=m), stream=stream.cuda_stream) as hf:
            y = torch.empty((M, J, N), dtype=torch.float32, device="cuda")
            y_def = torch.empty((dop["n_defocus"], M), dtype=torch.float32, device="cuda")
            tmr.tmr_forward(hf, Tg, y)
            tmr.tmr_defocus_forward(hf, Tg, y_def)
        s = photons / float(y.mean())
        y = (torch.poisson(y * s, generator=gen) / s).contiguous()
        y_def = (torch.poisson(y_def * s, generator=gen) / s).contiguous()
        # the network's inference on the fiber: 3 products of 2 B n_in h1 + ... flops
        feats = li.features(y)
        yout = torch.empty((M, 2 * N), dtype=torch.float32, device="cuda")
        tmr.tmr_mlp_forward(model, feats, M, yout)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record(stream)
        for _ in range(reps):
            tmr.tmr_mlp_forward(model, feats, M, yout)
        e1.record(stream)
        e1.synchronize()
        mlp_ms = e0.elapsed_time(e1) / reps
        mlp_flops = 2.0 * M * (J * N * h1 + h1 * h2 + h2 * 2 * N)
        tc = mlp_flops / (mlp_ms / 1e3) / 1e12
        out["tensor_roofline"] = {"kernel": "k_gemm_tc (tcgen05.mma, network inference, 3 layers)",
                                  "bound": "tensor", "achieved": tc, "peak": MEASURED_BF16_TFLOPS,
                                  "unit": "TFLOP/s", "frac": tc / MEASURED_BF16_TFLOPS, "ms": mlp_ms,
                                  "flops": mlp_flops, "rows": M,
                                  "peak_basis": "measured cuBLAS bf16 burst (of measured)",
                                  "note": "time includes the features' FP32 -> BF16 conversion and the "
                                          "bias/GELU kernels between the products"}
        del feats, yout

        def opts(init, prec, P):
            return dict(init=init, power_iters=P, clip=2.0, m=m, phase_iters=phase_iters, precision=prec,
                        use_graph=1, lanczos=lanczos, phase_tol=phase_tol)

        def make(init, prec):
            def mk(P):
                h = tmr.tmr_create(N, M, J, dg, dop, opts(init, prec, P), stream=stream.cuda_stream)
                if init == "learned":
                    tmr.tmr_set_init_model(h, model)
                return h
            return mk

        T_out = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        arms = {}
        ref_frac = None
        for init, prec in (("spectral", "fp32"), ("spectral", "mixed"), ("learned", "fp32"), ("learned", "mixed")):
            key = f"{init}+{prec}"
            h = make(init, prec)(power_iters)
            ms = timed_retrieve(tmr, torch, h, y, y_def, iters, T_out, stream)
            f = fidelity_rows_t(T_out, Tg).float().cpu().numpy()
            seeded = tmr.tmr_learned_rows(h) if init == "learned" else None
            h.close()
            if ref_frac is None:
                ref_frac = float(np.mean(f >= 0.99))
            arm = {"at_budget": {"power_iters": power_iters, "iters": iters, "value": world * M / (ms / 1e3),
                                 "unit": UNIT, "ms_per_step": ms, "mean": float(f.mean()),
                                 "frac_ge_0.99": float(np.mean(f >= 0.99))}}
            if seeded is not None:
                arm["rows_seeded_by_network"] = int(seeded)
            if lanczos:
                P_list = tuple(p for p in (16, 14, 12, 10, 8, 6, 4) if p <= power_iters)
            else:
                P_list = (100, 80, 60, 50, 40, 30) if init == "spectral" else (100, 80, 60, 50, 40, 30, 20)
            best, passing = sweep_to_099(tmr, torch, make(init, prec), y, y_def, Tg, ref_frac, stream, P_list,
                                         (10, 20, 30, 50, 75), world)
            arm["to_fidelity_0.99"] = best
            arm["passing"] = [{k: r[k] for k in ("power_iters", "iters", "value", "products")} for r in passing]
            arms[key] = arm
        out["arms"] = arms
        out["criterion"] = ("mean fidelity >= 0.99 and rows >= 0.99 within 0.5 % of the spectral FP32 arm at the "
                            "configured budget; fastest passing (power, L-BFGS) pair; retrieve with the phase "
                            "fit, CUDA events, one warm run first")
        # against the FP64 oracle: the CPU baseline's sampled rows (plain fiber,
        # oracle-made intensities, the configured budget)
        if keep:
            import oracle
            ns = keep["Y"].shape[0]
            dk = torch.from_numpy(keep["d"].astype(np.complex64)).cuda()
            Ts_ = torch.empty((ns, N), dtype=torch.complex64, device="cuda")
            par = {}
            for init, prec in (("spectral", "mixed"), ("learned", "fp32"), ("learned", "mixed")):
                o = opts(init, prec, power_iters)
                o["use_graph"] = 0
                with tmr.tmr_create(N, ns, J, dk, None, o, stream=stream.cuda_stream) as hs:
                    if init == "learned":
                        tmr.tmr_set_init_model(hs, model)
                    tmr.tmr_retrieve(hs, torch.from_numpy(keep["Y"]).cuda(), None, iters, Ts_)
                    stream.synchronize()
                fg = oracle.fidelity_rows(Ts_.cpu().numpy(), keep["T"])
                dfid = np.abs(fg - keep["fid"])
                par[f"{init}+{prec}"] = {"rows": int(ns), "mean_abs_fidelity_diff": float(dfid.mean()),
                                         "max_abs_fidelity_diff": float(dfid.max()),
                                         "frac_within_1e-3": float(np.mean(dfid <= 1e-3))}
            out["oracle_parity"] = par
        model.close()
    return out


# ---------------------------------------------------------------- J-sweep (2D probing DFT)
def run_jsweep(args):
    """Failed-row fraction against the number of masks J = 3 .. 8 with the
    paper's 2D probing DFT (Sec. 2.2: K the 2D DFT of the 64 x 64 phase
    modes, N = 4096), noiseless data from a mode-model TM (R = 2200) on a
    64 x 64 output grid, the spectral start of --start (16 Lanczos steps by
    default) and 200 L-BFGS
    iterations; a row fails when its fidelity to the truth is below 0.99.  The
    paper's simulation (Sec. 3) swept M = 3 .. 9 masks on a measured TM; J = 9
    is beyond this library's 8."""
    import torch
    import paper_2302_13524_gb300 as tmr
    import synth
    N, n1, M, R = 4096, 64, 4096, 2200
    pits, iters = args.power_iters, 200 if args.iters == WORKLOADS[args.workload]["iters"] else args.iters
    T = torch.from_numpy(synth.tm_modes(M, N, R, seed=0, dtype=np.complex64)).cuda()
    out = []
    for J in range(3, 9):
        _, d = synth.mask_phases(J, N, seed=J)
        dg = torch.from_numpy(np.ascontiguousarray(d, dtype=np.complex64)).cuda()
        with tmr.tmr_create(N, M, J, dg, None, dict(probe_n1=n1, init="spectral", power_iters=pits,
                                                      clip=2.0, lanczos=args.lanczos)) as h:
            y = torch.empty((M, J, N), dtype=torch.float32, device="cuda")
            tmr.tmr_forward(h, T, y)
            To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
            tmr.tmr_retrieve(h, y, None, iters, To)  # warm
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            tmr.tmr_retrieve(h, y, None, iters, To)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
        f = fidelity_rows_t(To, T).float().cpu().numpy()
        out.append({"J": J, "failed_frac": float(np.mean(f < 0.99)), "mean": float(f.mean()),
                    "p1": float(np.percentile(f, 1)), "rows_per_s": M / (ms / 1e3), "ms": ms})
        del y, To
    line = {"metric": "failed-row fraction vs J (2D probing DFT)", "unit": "fraction", "n_gpus": 1,
            "higher_is_better": False, "data": "synthetic, noiseless",
            "config": {"workload": f"jsweep: N={N} as 64x64 2D DFT (probe_n1={n1}), M={M} (64x64), modes R={R}, "
                                   f"noiseless, {pits} {'Lanczos' if args.lanczos else 'power'} + {iters} "
                                   f"L-BFGS iterations, J = 3..8",
                       "dtype": "f32"},
            "value": out[-1]["failed_frac"], "sweep": out}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- Table 1: with and without FFT
def run_dense(args):
    """The paper's Table 1 restated on one GPU: the loss and gradient of all
    rows (the work of an L-BFGS iteration that depends on how Q is applied)
    through the FFT path and through the explicit dense Q (cuBLAS complex
    products, FP32 and FP32 emulated on the tensor cores by BF16x9), on
    1024 rows of an N = 4096 mode-model TM with J = 8 masks (the paper:
    1024 rows, N = 8192, M = 8); plus the whole FFT retrieval of those rows.
    Times are CUDA-event means after warm-up."""
    import torch
    import paper_2302_13524_gb300 as tmr
    import synth
    W = WORKLOADS["dense"]
    N, J, R = W["N"], W["J"], W["R"]
    M = W["ny"] * W["nx"]
    T = torch.from_numpy(synth.tm_modes(M, N, R, seed=0, dtype=np.complex64)).cuda()
    _, d = synth.mask_phases(J, N, seed=0)
    dg = torch.from_numpy(np.ascontiguousarray(d, dtype=np.complex64)).cuda()
    y = torch.empty((M, J, N), dtype=torch.float32, device="cuda")
    T1 = (T * 1.05).contiguous()
    loss = torch.empty(M, dtype=torch.float32, device="cuda")
    G = torch.empty((M, N), dtype=torch.complex64, device="cuda")

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {}
    with tmr.tmr_create(N, M, J, dg, None, dict(init="spectral", power_iters=args.power_iters,
                                                lanczos=args.lanczos, clip=2.0)) as h:
        tmr.tmr_forward(h, T, y)
        out["fft"] = timed(lambda: tmr.tmr_grad(h, T1, y, loss, G))
        To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        retr_ms = timed(lambda: tmr.tmr_retrieve(h, y, None, args.iters, To), reps=2)
    G_fft = G.clone()
    errs = {}
    for mode, name in ((1, "dense_fp32"), (2, "dense_bf16x9")):
        try:
            with tmr.tmr_create(N, M, J, dg, None, dict(dense=mode)) as h:
                out[name] = timed(lambda: tmr.tmr_grad(h, T1, y, loss, G))
                errs[name] = float(torch.max(torch.abs(G - G_fft)) / torch.max(torch.abs(G_fft)))
        except tmr.TMRError as e:
            out[name] = None
            errs[name] = str(e)
    # the whole retrieval with and without FFT at the budget that meets the 0.99 bar
    budget_iters = 20
    solves = {}
    for dense in (0, 1):
        with tmr.tmr_create(N, M, J, dg, None, dict(init="spectral", power_iters=args.power_iters,
                                                    lanczos=args.lanczos, clip=2.0, dense=dense)) as h:
            To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
            ms = timed(lambda: tmr.tmr_retrieve(h, y, None, budget_iters, To), reps=1)
            f = fidelity_rows_t(To, T).float().cpu().numpy()
            solves["without_fft" if dense else "with_fft"] = {"ms": ms, "mean_fidelity": float(f.mean()),
                                                               "frac_ge_0.99": float(np.mean(f >= 0.99))}
    gemm_flops = 2 * 8.0 * M * N * (J * N)  # two complex products per gradient
    line = {"metric": "gradient evaluation of all rows: FFT vs dense Q (Table 1)", "unit": "ms",
            "n_gpus": 1, "higher_is_better": False, "data": "synthetic, noiseless",
            "config": {"workload": W["desc"], "dtype": "f32"},
            "value": out["fft"], "eval_ms": out,
            "speedup_fft_over_dense": {k: (v / out["fft"] if v else None) for k, v in out.items() if k != "fft"},
            "dense_tflops": {k: (gemm_flops / (v / 1e3) / 1e12 if v else None) for k, v in out.items()
                             if k != "fft"},
            "dense_rel_error_vs_fft": errs,
            "fft_retrieval_ms": retr_ms,
            "retrieval_same_budget": dict(solves, budget=f"{args.power_iters} "
                                          f"{'Lanczos' if args.lanczos else 'power'} + {budget_iters} L-BFGS",
                                          speedup=solves["without_fft"]["ms"] / solves["with_fft"]["ms"]),
            "fft_retrieval": f"{args.power_iters} {'Lanczos' if args.lanczos else 'power'} + {args.iters} "
                             f"L-BFGS iterations"}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- our arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "jsweep":
        return run_jsweep(args)
    if args.workload == "dense":
        return run_dense(args)
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import paper_2302_13524_gb300 as tmr
    import synth

    W = WORKLOADS[args.workload]
    N, J, R = W["N"], W["J"], W["R"]
    ny, nx = W["ny"], W["nx"]
    M = args.rows or ny * nx
    if M != ny * nx:
        nx = 64
        ny = M // nx
        assert ny * nx == M, "--rows must be a multiple of 64"
    Nd, m = 50, 5
    seed = 1000 * rank  # every rank retrieves its own fiber (independent problems)
    stream = torch.cuda.Stream()

    # ---- synthetic inputs (not timed) ----
    T = synth.tm_modes(M, N, R, seed=seed, dtype=np.complex64)
    cam = W.get("camera")
    if cam:  # light leaves the fiber core only: rows outside the disc nearly dark
        disc = synth.fiber_disc(ny, nx, cam["radius"])
        T[~disc] *= np.float32(cam["leak"])
    _, d = synth.mask_phases(J, N, seed=seed)
    d = np.ascontiguousarray(d, dtype=np.complex64)
    Tg = torch.from_numpy(T).cuda()
    dg = torch.from_numpy(d).cuda()
    # the retrieve replays a captured CUDA graph (captured during the warm-up);
    # host-buffer calls (the e2e leg) launch directly
    opt = dict(init="spectral", power_iters=args.power_iters, clip=2.0, m=m,
               phase_iters=args.phase_iters, seed=seed, tol=W["tol"], precision=args.precision,
               use_graph=1, lanczos=args.lanczos, phase_tol=args.phase_tol)
    if args.schedule:
        opt["schedule"] = args.schedule
    dop = dict(ny=ny, nx=nx, n_defocus=Nd, coef=0.05)
    h = tmr.tmr_create(N, M, J, dg, dop, opt, stream=stream.cuda_stream)
    sched = tmr.tmr_schedule(h)
    y = torch.empty((M, J, N), dtype=torch.float32, device="cuda")
    y_def = torch.empty((Nd, M), dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        tmr.tmr_forward(h, Tg, y)
        tmr.tmr_defocus_forward(h, Tg, y_def)
        gen = torch.Generator(device="cuda")
        gen.manual_seed(seed + 7)
        ph = W["photons"]
        if isinstance(ph, tuple):  # photon level per row, log-uniform
            u = torch.rand(M, generator=gen, device="cuda", dtype=torch.float64)
            ph = torch.exp(math.log(ph[0]) + u * (math.log(ph[1]) - math.log(ph[0])))
        # photons per pixel averaged over the lit rows (the fiber core, for the camera workload)
        y_lit = y[torch.from_numpy(disc).cuda()] if cam else y
        s_row = (ph / float(y_lit.mean())) * torch.ones(M, dtype=torch.float64, device="cuda")
        del y_lit
        s_y = s_row.float().view(M, 1, 1)
        counts = torch.poisson(y * s_y, generator=gen)
        y = counts / s_y
        s_d = s_row.float().view(1, M)
        counts_d = torch.poisson(y_def * s_d, generator=gen)
        y_def = counts_d / s_d
    stream.synchronize()
    T_out = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    status = torch.empty(M, dtype=torch.int32, device="cuda")

    def step():
        tmr.tmr_retrieve(h, y, y_def, args.iters, T_out, status)

    prep = None
    if cam:
        # camera frames: the photon counts of each half-grid pixel repeated over
        # its 2 x 2 camera pixels, uint16 (carried as int16 bits)
        K, Hc, Wc = J * N, 2 * ny, 2 * nx

        def to_frames(c, n):
            c = c.reshape(n, ny, nx).clamp(max=65535).to(torch.int32)
            c = torch.where(c > 32767, c - 65536, c).to(torch.int16)
            return c.repeat_interleave(2, 1).repeat_interleave(2, 2).contiguous()
        with torch.cuda.stream(stream):
            frames = to_frames(counts.view(M, K).t(), K)
            frames_d = to_frames(counts_d, Nd)
        stream.synchronize()
        del counts, counts_d
        y = torch.empty((M, J, N), dtype=torch.float32, device="cuda")
        y_def = torch.empty((Nd, M), dtype=torch.float32, device="cuda")
        mask_p = torch.empty(M, dtype=torch.uint8, device="cuda")
        n_in = torch.empty(1, dtype=torch.int32, device="cuda")
        wb = tmr.tmr_preprocess_workspace_bytes(K, Hc, Wc, 0)
        ws = torch.empty(wb, dtype=torch.uint8, device="cuda")

        def preprocess():
            tmr.tmr_preprocess(frames, K, Hc, Wc, 0, cam["energy_frac"], y, mask_p, None, n_in, ws, wb,
                               stream=stream.cuda_stream)
            tmr.tmr_half_sample(frames_d, Nd, Hc, Wc, 0, y_def, stream=stream.cuda_stream)

        def step():  # noqa: F811 -- the camera step: preprocessing, then the retrieve
            preprocess()
            tmr.tmr_retrieve(h, y, y_def, args.iters, T_out, status)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---- warm-up ----
    for _ in range(args.warmup):
        step()
    stream.synchronize()

    # ---- timed region: K full steps, inputs (256 MB) larger than L2 ----
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    ev1.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world)
    value = job_rows_per_s(M, world, ms / 1e3)

    # ---- quality of the result (after timing) ----
    def fidelity(A, B):
        ip = (A.conj() * B).sum(1).abs()
        den = A.abs().pow(2).sum(1).sqrt() * B.abs().pow(2).sum(1).sqrt()
        return torch.where(den > 0, ip / den, torch.zeros_like(ip))
    fid = fidelity(T_out, Tg).float().cpu().numpy()
    num = (T_out.conj() * Tg).sum().abs()
    mfid = float(num / (T_out.abs().pow(2).sum().sqrt() * Tg.abs().pow(2).sum().sqrt()))
    if cam:
        # the rows inside the fiber are the ones solved; the rest come back zero
        fid = fid[disc]
        inside = int(n_in.item())
        prep_in = mask_p.cpu().numpy().astype(bool)
        # preprocessing alone: algorithmic bytes = the kept camera rows read
        # once (their DRAM sectors carry the skipped columns) + y written once
        ev_a = torch.cuda.Event(enable_timing=True)
        ev_b = torch.cuda.Event(enable_timing=True)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        pts = []
        for _ in range(5):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev_a.record(stream)
            tmr.tmr_preprocess(frames, K, Hc, Wc, 0, cam["energy_frac"], y, mask_p, None, n_in, ws, wb,
                               stream=stream.cuda_stream)
            ev_b.record(stream)
            ev_b.synchronize()
            pts.append(ev_a.elapsed_time(ev_b))
        p_ms = float(np.median(pts))
        p_bytes = K * ny * Wc * 2 + M * K * 4
        gbs = p_bytes / (p_ms / 1e3) / 1e9
        prep = {"ms": p_ms, "bytes": p_bytes, "GB/s": gbs, "peak": MEASURED_HBM_GBS,
                "frac": gbs / MEASURED_HBM_GBS, "rows_inside_mask": inside,
                "mask_covers_disc": float(np.mean(prep_in[disc])),
                "mask_outside_disc": int(np.sum(prep_in[~disc])),
                "kernels": "k_prep_rows, k_prep_energy, k_prep_select, k_prep_zero (L2 flushed "
                           "before each call)"}

    # ---- solver kernel alone (the dominant kernel): roofline ----
    ev2 = torch.cuda.Event(enable_timing=True)
    ev3 = torch.cuda.Event(enable_timing=True)
    ns = max(2, args.steps // 2)
    row_iters = torch.empty(M, dtype=torch.int32, device="cuda")
    ev2.record(stream)
    for _ in range(ns):
        tmr.tmr_retrieve(h, y, None, args.iters, T_out, status, row_iters)
    ev3.record(stream)
    ev3.synchronize()
    solver_ms = ev2.elapsed_time(ev3) / ns
    its = row_iters.cpu().numpy()
    worked = status.cpu().numpy() != tmr.TMR_ROW_ZERO  # zero rows (outside a fiber mask) do no work
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    flops = solver_flops(N, J, m, its[worked], args.power_iters, args.lanczos)
    achieved = flops / (solver_ms / 1e3) / 1e12
    peak_max = fp32_peak_tflops(n_sm, 2070.0)
    # DRAM bytes of the solver, from one ncu capture of the current kernel
    # (dram__bytes_read.sum + dram__bytes_write.sum) on the plain workload at
    # 4096 rows with the 16-step Lanczos start: k_solver_row<2048> read
    # 138.84 MB and wrote 42.29 MB; traffic grows with the rows, so a full
    # 8192-row launch moves twice that.
    kname = (f"k_solver_row<{N}> (one CTA per row)" if sched == 16
             else f"k_solver<{'XfPow2' if N & (N - 1) == 0 else 'XfBlue'}, {sched}> (cluster of {J // max(sched, 1)} CTAs)")
    traffic, tbasis = None, "no capture of this kernel and workload"
    if (args.workload == "plain" and sched == 16 and args.precision == "fp32" and args.lanczos
            and args.power_iters == 16):
        traffic = (138835456 + 42292480) * (M / 4096.0)
        tbasis = ("ncu capture of k_solver_row<2048> at 4096 rows (138.84 MB read + 42.29 MB written), "
                  "scaled by rows; algorithmic bytes per 4096 rows: y 134.2 MB read, T 67.1 MB written "
                  "(output rows still dirty in L2 at the kernel's end are written back after it)")
    roof = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak_max,
            "unit": "TFLOP/s", "frac": achieved / peak_max, "traffic": traffic,
            "traffic_basis": tbasis,
            "peak_basis": f"FP32 FFMA {n_sm} SMs x 128 lanes x 2 x 2070 MHz (max clock)",
            "solver_ms": solver_ms, "flops_per_launch": flops}
    if clk and clk.get("sm_mhz"):
        roof["frac_at_measured_clock"] = achieved / fp32_peak_tflops(n_sm, clk["sm_mhz"])
    if args.precision == "mixed":
        # tensor-pipe work of the split-BF16 DFT stages: per transform, A
        # radix-16 passes of N/128 groups x 12 mma.m16n8k16 and B radix-8 passes
        # of N/64 groups x 3 (4096 flops each), N = 16^A 8^B with A largest; the
        # power iterations, the start and all but the last 10 iterations use them
        lg = int(round(math.log2(N)))
        a16 = (3 if lg >= 12 else 0) if lg % 3 == 0 else (1 if lg % 3 == 1 else 2)
        b8 = (lg - 4 * a16) // 3
        per_transform = (a16 * (N // 128) * 12 + b8 * (N // 64) * 3) * 4096
        tc_iters = np.maximum(its - 10, 0) if args.iters > 10 else np.zeros_like(its)
        n_tr = 2 * J * (M * (args.power_iters + 1) + float(np.sum(tc_iters)))
        tc = per_transform * n_tr / (solver_ms / 1e3) / 1e12
        roof["tensor"] = {"achieved": tc, "unit": "TFLOP/s", "peak": MEASURED_BF16_TFLOPS,
                          "frac": tc / MEASURED_BF16_TFLOPS,
                          "basis": "split-BF16 mma.sync flops of the DFT stages; peak = measured "
                                   "cuBLAS bf16 burst"}

    # ---- smallest budget that meets the 0.99 bar (the whole retrieve, phase
    # fit included): mean fidelity >= 0.99 and the fraction of rows >= 0.99
    # within 0.5 % of the configured budget's ----
    # The budget has two parts, the power iterations of the spectral start and
    # the L-BFGS iterations; for each start length the smallest L-BFGS budget
    # that passes is timed, and the fastest passing pair is reported.
    to099 = None
    if not args.no_sweep and args.iters > 10:
        ref_frac = float(np.mean(fid >= 0.99))
        tried = []
        for pits in sorted({args.power_iters} | ({12, 8} if args.lanczos else {50, 30}), reverse=True):
            if pits > args.power_iters:
                continue
            hp = h if pits == args.power_iters else tmr.tmr_create(
                N, M, J, dg, dop, dict(opt, power_iters=pits), stream=stream.cuda_stream)
            for it in (10, 20, 30, 50, 75):
                if it >= args.iters:
                    break
                if cam:
                    preprocess()
                tmr.tmr_retrieve(hp, y, y_def, it, T_out, status)  # warm (graph, staging)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if cam:
                    preprocess()
                tmr.tmr_retrieve(hp, y, y_def, it, T_out, status)
                e1.record(stream)
                e1.synchronize()
                f_it = fidelity(T_out, Tg).float().cpu().numpy()
                if cam:
                    f_it = f_it[disc]
                if f_it.mean() >= 0.99 and np.mean(f_it >= 0.99) >= ref_frac - 0.005:
                    t_it = e0.elapsed_time(e1)
                    tried.append({"power_iters": pits, "iters": it, "value": world * M / (t_it / 1e3),
                                  "unit": UNIT, "ms_per_step": t_it, "mean": float(f_it.mean()),
                                  "frac_ge_0.99": float(np.mean(f_it >= 0.99))})
                    break
            if hp is not h:
                hp.close()
        if tried:
            to099 = dict(max(tried, key=lambda r: r["value"]))
            to099["criterion"] = ("mean >= 0.99 and rows >= 0.99 within 0.5 % of the configured budget's; "
                                  "fastest passing (start steps, L-BFGS) pair")
            to099["passing"] = [{k: r[k] for k in ("power_iters", "iters", "value")} for r in tried]

    # ---- end to end through the C ABI with host buffers ----
    e2e = None  # (the camera step's preprocessing takes device frames only)
    if not args.no_e2e and not cam:
        y_h = y.cpu().pin_memory()
        yd_h = y_def.cpu().pin_memory()
        T_h = torch.empty((M, N), dtype=torch.complex64).pin_memory()
        tmr.tmr_retrieve(h, y_h, yd_h, args.iters, T_h)  # staging buffers allocated here
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            tmr.tmr_retrieve(h, y_h, yd_h, args.iters, T_h)
        dt = max_over_ranks((time.perf_counter() - t0) / args.steps, world)
        e2e = {"value": job_rows_per_s(M, world, dt), "unit": UNIT,
               "h2d_bytes_per_step": int(y_h.numel() * 4 + yd_h.numel() * 4),
               "d2h_bytes_per_step": int(T_h.numel() * 8), "ms_per_step": dt * 1e3}

    cpu = None
    keep = {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt, cores, desc = cpu_oracle_sample(W, M, args.iters, args.power_iters,
                                               rows_n=max(1, min(16, os.cpu_count() or 8)), seed=seed,
                                               keep=keep, lanczos=args.lanczos)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
               "seconds": dt}
        # the same sampled rows (oracle-made intensities) through the library with
        # this run's options: the error of this arithmetic against the FP64 oracle
        import oracle
        ns = keep["Y"].shape[0]
        Ts = torch.empty((ns, N), dtype=torch.complex64, device="cuda")
        with tmr.tmr_create(N, ns, J, torch.from_numpy(keep["d"].astype(np.complex64)).cuda(), None,
                            opt) as hs:
            tmr.tmr_retrieve(hs, torch.from_numpy(keep["Y"]).cuda(), None, args.iters, Ts)
            torch.cuda.synchronize()
        Tg = Ts.cpu().numpy()
        fg = oracle.fidelity_rows(Tg, keep["T"])
        agree = oracle.fidelity_rows(Tg, keep["Tr"])
        dfid = np.abs(fg - keep["fid"])
        cpu["oracle_parity"] = {"rows": int(ns), "precision": args.precision,
                                "mean_abs_fidelity_diff": float(dfid.mean()),
                                "max_abs_fidelity_diff": float(dfid.max()),
                                "frac_within_1e-3": float(np.mean(dfid <= 1e-3)),
                                "gpu_vs_oracle_row_fidelity_mean": float(agree.mean()),
                                "gpu_vs_oracle_row_fidelity_min": float(agree.min())}

    h.close()
    arms = None
    if (rank == 0 and not args.no_arms and args.workload == "plain" and args.precision == "fp32"
            and args.rows is None and args.iters > 10):
        torch.cuda.empty_cache()
        arms = second_half_arms(tmr, torch, synth, N, M, J, R, m, d, dop, W["photons"], args.phase_iters,
                                stream, world, args.iters, args.power_iters,
                                keep=keep if cpu is not None else None, lanczos=args.lanczos,
                                phase_tol=args.phase_tol)
    batching = None
    if (rank == 0 and world == 1 and args.workload == "plain" and args.rows is None and not args.no_batching
            and not args.no_sweep):
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        batching = batching_child_line()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.precision == "fp32" else "mixed f16/bf16/f32 (f64 phase fit)",
                "data": "synthetic",
                "config": {"workload": W["desc"], "N": N, "M": M, "J": J, "grid": [ny, nx],
                           "R": R, "photons": W["photons"], "init": "spectral", "tol": W["tol"],
                           "precision": args.precision,
                           "start": f"{args.power_iters} {'Lanczos steps' if args.lanczos else 'power iterations'}",
                           "power_iters": args.power_iters, "iters": args.iters, "m": m,
                           "row_iters_mean": float(its[worked].mean()), "row_iters_max": int(its.max()),
                           "rows_solved": int(worked.sum()),
                           "n_defocus": Nd, "phase_iters": args.phase_iters, "phase_tol": args.phase_tol,
                           "l2": f"inputs larger than L2 (y is {M * J * N * 4 >> 20} MB)",
                           "parallelism": f"{world} independent TMs, one per GPU"},
                "schedule": {"code": sched, "layout": "one CTA per row (16 points per thread)" if sched == 16
                             else f"{sched} masks per CTA, cluster of {J // max(sched, 1)} CTAs per row",
                             "autotuned": not args.schedule, "cuda_graph": True},
                "fidelity": {"mean": float(fid.mean()), "p1": float(np.percentile(fid, 1)),
                             "frac_ge_0.99": float(np.mean(fid >= 0.99)),
                             "matrix_after_phase_fit": mfid},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "to_fidelity_0.99": to099,
                # kernels per timed step: k_solver, k_fields, k_row_energy,
                # k_phase_fit, k_apply_phase (+ k_pack_f16 in mixed precision;
                # + k_prep_rows, k_prep_energy, k_prep_select, k_prep_zero and
                # k_half_sample for the camera workload)
                "gpu_launches": ((6 if args.precision == "mixed" else 5) + (5 if cam else 0)) * args.steps}
        if batching is not None:
            line["batching"] = batching
        if arms is not None:
            line["learned_init_mixed"] = arms
            line["roofline"]["tensor_mlp"] = arms.get("tensor_roofline")
        if cam:
            line["preprocess"] = prep
            line["fidelity"]["rows"] = "rows inside the fiber disc"
            line["config"]["frames"] = f"{J * N} + {Nd} uint16 frames of {2 * ny}x{2 * nx}"
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
