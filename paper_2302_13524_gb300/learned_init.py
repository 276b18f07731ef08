"""Training and evaluation of the learned initialiser (TMR_INIT_LEARNED).

Data: fibers of one family (shared input mode basis, own coupling and phases),
their intensities made by tmr_forward with Poisson noise, and the rows the
plain method retrieves from them (spectral start + L-BFGS through
tmr_retrieve).  Features are sqrt(y) / sqrt(mean y) per row (the same the
library computes for inference); targets are the retrieved rows scaled to
norm sqrt(N), as [Re t, Im t], compared with the network's output up to a
global phase (TMR_LOSS_PHASE).  Training runs tmr_mlp_train_step (the
library's BF16 kernels).  At retrieval the proposal seeds the spectral power
iteration (TMR_INIT_LEARNED), so a proposal closer to the leading eigenvector
than a random vector needs fewer power iterations.

Everything numeric on the path runs in libtmr; torch only holds device
buffers and draws the noise of the synthetic data.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import _lib as tmr


def fiber_data(h, T, photons: float, gen: torch.Generator):
    """(T on device, noisy intensities y) for one fiber (a numpy array or a
    complex64 device tensor) through tmr_forward."""
    M, N = T.shape
    if isinstance(T, torch.Tensor):
        Tg = T.to(device="cuda", dtype=torch.complex64).contiguous()
    else:
        Tg = torch.from_numpy(np.ascontiguousarray(T, dtype=np.complex64)).cuda()
    y = torch.empty((M, h.J, N), dtype=torch.float32, device="cuda")
    tmr.tmr_forward(h, Tg, y)
    s = photons / float(y.mean())
    y = torch.poisson(y * s, generator=gen) / s
    return Tg, y.contiguous()


def features(y: torch.Tensor) -> torch.Tensor:
    M = y.shape[0]
    yf = y.reshape(M, -1).clamp_min(0)
    return (yf.sqrt() / (yf.mean(1, keepdim=True).sqrt() + 1e-30)).contiguous()


def targets(T_hat: torch.Tensor) -> torch.Tensor:
    """Retrieved rows scaled to norm sqrt(N), as [Re t, Im t].  Their global
    phases are left as the solver returned them: the network is trained with
    the phase-invariant loss (TMR_LOSS_PHASE), which compares each output row
    with the nearest rotation of its target."""
    t = T_hat / (T_hat.abs().pow(2).sum(1, keepdim=True).sqrt() + 1e-30) * (T_hat.shape[1] ** 0.5)
    return torch.cat([t.real, t.imag], 1).float().contiguous()


def fidelity(A: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
    ip = (A.conj() * B).sum(1).abs()
    den = A.abs().pow(2).sum(1).sqrt() * B.abs().pow(2).sum(1).sqrt()
    return torch.where(den > 0, ip / den, torch.zeros_like(ip))


def build_dataset(tm_fn, fibers, N, M, J, masks, photons, iters, power_iters, seed=0):
    """Retrieve every fiber with the plain method; returns (X, Tt) on device."""
    Xs, Ts = [], []
    dg = torch.from_numpy(np.ascontiguousarray(masks, dtype=np.complex64)).cuda()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    with tmr.tmr_create(N, M, J, dg, None, dict(init="spectral", power_iters=power_iters)) as h:
        for f in fibers:
            _, y = fiber_data(h, tm_fn(f), photons, gen)
            T_hat = torch.empty((M, N), dtype=torch.complex64, device="cuda")
            tmr.tmr_retrieve(h, y, None, iters, T_hat)
            torch.cuda.synchronize()
            Xs.append(features(y))
            Ts.append(targets(T_hat))
    return torch.cat(Xs), torch.cat(Ts)


def train(model: tmr.MLP, X: torch.Tensor, Tt: torch.Tensor, epochs: int, batch: int, lr: float, seed=0):
    """Adam over shuffled mini-batches of the phase-invariant loss; returns the
    mean loss of each epoch's batches."""
    tmr.tmr_mlp_set_loss(model, tmr.TMR_LOSS_PHASE)
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    hist = []
    n = X.shape[0]
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).cuda()
        acc = torch.zeros(1, dtype=torch.float32, device="cuda")
        nb = 0
        for i in range(0, n - batch + 1, batch):
            idx = perm[i:i + batch]
            tmr.tmr_mlp_train_step(model, X[idx].contiguous(), Tt[idx].contiguous(), batch, lr, loss)
            acc += loss
            nb += 1
        torch.cuda.synchronize()
        hist.append(float(acc.item()) / max(nb, 1))
    return hist


ARMS = (("random", "fp32"), ("spectral", "fp32"), ("learned", "fp32"), ("spectral", "mixed"),
        ("learned", "mixed"))


def to_099(res, ref_frac, rows):
    """Per arm: among the (power iterations, L-BFGS iterations) budgets whose
    mean fidelity is >= 0.99 and whose fraction of rows >= 0.99 is within
    0.5 % of ref_frac, the fastest (retrieve wall time per fiber, the learned
    start's network included) and the one with the fewest operator products
    (power + L-BFGS iterations: each applies Q and Q^H once), with rows/s."""
    out = {}
    for init, prec in ARMS:
        key = f"{init}+{prec}"
        ok = []
        for k, r in res.items():
            if not k.startswith(key + "/"):
                continue
            if r["mean"] >= 0.99 and r["frac_ge_0_99"] >= ref_frac - 0.005:
                ok.append((r["ms_per_fiber"], r["power_iters"] + r["iters"], r))
        if not ok:
            out[key] = None
            continue
        fast = min(ok, key=lambda t: (t[0], t[1]))[2]
        few = min(ok, key=lambda t: (t[1], t[0]))[2]
        out[key] = dict(fastest=dict(power_iters=fast["power_iters"], iters=fast["iters"],
                                     rows_per_s=rows / (fast["ms_per_fiber"] / 1e3), mean=fast["mean"],
                                     frac_ge_0_99=fast["frac_ge_0_99"]),
                        fewest_products=dict(power_iters=few["power_iters"], iters=few["iters"],
                                             products=few["power_iters"] + few["iters"],
                                             rows_per_s=rows / (few["ms_per_fiber"] / 1e3)))
    return out


def evaluate(model, tm_fn, fibers, N, M, J, masks, photons, budgets, seed=1, arms=ARMS):
    """For every start (random, spectral, learned), arithmetic (FP32, mixed)
    and budget (power iterations, L-BFGS iterations): mean fidelity, fraction
    of rows >= 0.99 and retrieve time per fiber on held-out fibers.  The
    random start takes no power iterations, so its budgets are (0, I)."""
    dg = torch.from_numpy(np.ascontiguousarray(masks, dtype=np.complex64)).cuda()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    data = []
    with tmr.tmr_create(N, M, J, dg, None, dict(init="spectral")) as h0:
        for f in fibers:
            data.append(fiber_data(h0, tm_fn(f), photons, gen))
    out = {}
    for init, prec in arms:
        pits = sorted({p for p, _ in budgets}) if init != "random" else [0]
        for p in pits:
            opt = dict(init=init, power_iters=p, precision=prec)
            with tmr.tmr_create(N, M, J, dg, None, opt) as h:
                if init == "learned":
                    tmr.tmr_set_init_model(h, model)
                for pp, it in budgets:
                    if init != "random" and pp != p:
                        continue
                    fids, ms, kept = [], 0.0, 0
                    for Tg, y in data:
                        To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
                        tmr.tmr_retrieve(h, y, None, it, To)  # warm
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        tmr.tmr_retrieve(h, y, None, it, To)
                        torch.cuda.synchronize()
                        ms += (time.perf_counter() - t0) * 1e3
                        fids.append(fidelity(To, Tg).float().cpu().numpy())
                        if init == "learned":
                            kept += tmr.tmr_learned_rows(h)
                    fi = np.concatenate(fids)
                    out[f"{init}+{prec}/{p}/{it}"] = dict(
                        power_iters=p, iters=it, mean=float(fi.mean()), frac_ge_0_99=float(np.mean(fi >= 0.99)),
                        ms_per_fiber=ms / len(data),
                        raw_proposal_rows=(kept / fi.size) if init == "learned" else None)
    return out


def main(argv=None):
    """Train on the family's training fibers and report held-out results as one JSON line."""
    import argparse
    import json
    import os
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--rows", type=int, default=8192, help="rows per fiber")
    ap.add_argument("--train-fibers", type=int, default=25)
    ap.add_argument("--test-fibers", type=int, default=5)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--power-budgets", default="20,30,40,50,60,80,100")
    ap.add_argument("--iter-budgets", default="10,15,20,30,50")
    ap.add_argument("--power-iters", type=int, default=100, help="power iterations of the training retrieves")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    cfg = synth.CONFIGS["learned"]
    N, J, R = cfg["N"], cfg["J"], cfg["R"]
    M = a.rows
    _, d = synth.mask_phases(J, N, seed=0)

    def tm_fn(f):
        return synth.tm_family(M, N, R, fiber_seed=f, basis_seed=0)

    t0 = time.perf_counter()
    X, Tt = build_dataset(tm_fn, cfg["train_fibers"][:a.train_fibers], N, M, J, d, cfg["photons"],
                          cfg["iters"], a.power_iters)
    t_data = time.perf_counter() - t0
    h1, h2 = cfg["widths"]
    with tmr.tmr_mlp_create(J * N, h1, h2, 2 * N, seed=0) as model:
        t0 = time.perf_counter()
        hist = train(model, X, Tt, a.epochs, a.batch, a.lr)
        t_train = time.perf_counter() - t0
        del X, Tt
        torch.cuda.empty_cache()
        pb = [int(b) for b in a.power_budgets.split(",")]
        ib = [int(b) for b in a.iter_budgets.split(",")]
        budgets = [(p, i) for p in pb for i in ib]
        res = evaluate(model, tm_fn, cfg["test_fibers"][:a.test_fibers], N, M, J, d, cfg["photons"], budgets)
    ref = res[f"spectral+fp32/{max(pb)}/{max(ib)}"]["frac_ge_0_99"]
    rep = {"config": dict(N=N, J=J, R=R, rows_per_fiber=M, train_fibers=a.train_fibers,
                          test_fibers=a.test_fibers, widths=[J * N, h1, h2, 2 * N], epochs=a.epochs,
                          batch=a.batch, lr=a.lr, power_iters=a.power_iters),
           "train_loss": hist, "seconds": dict(data=t_data, train=t_train), "held_out": res,
           "to_fidelity_0_99": to_099(res, ref, M)}
    line = json.dumps(rep)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(line + "\n")
    print(line)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
