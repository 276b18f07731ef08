"""Mixed precision (TMR_PREC_MIXED) against the FP64 oracle through the C ABI:
tensor-core split-BF16 transforms (forward model, gradient; radix-16 and
radix-8 passes), FP16 intensities with BF16 L-BFGS pairs in the solver, the
learned start in mixed precision, and the precision workload (N = 4096,
M = 16384, 128 x 128 grid, mode model R = 2200) with its error stated against
the oracle on sampled rows and against the FP32 path on every row.

Bars (stated from the arithmetic): a split BF16 product carries about 16
significant bits, so one 16-point DFT is good to a few 1e-6 relative and a
length-4096 transform (three passes) to about 1e-5; intensities |z|^2 double
that.  The forward model and gradient are held to 1e-4 relative."""
import numpy as np
import pytest

import oracle
import synth
from helpers import c64, f32, problem, assert_rows_close, max_rel_elem_rows, rel_l2_rows, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2302_13524_gb300 as tmr  # noqa: E402

MIXED = tmr.TMR_PREC_MIXED


def handle(N, M, J, d, dop=None, **opt):
    return tmr.tmr_create(N, M, J, to_dev(d), dop, opt or None)


@pytest.mark.parametrize("N", [256, 1024, 2048, 4096])
@pytest.mark.parametrize("J", [4, 3])
def test_tensor_core_forward(N, J):
    M = 4
    T, d, _ = problem(N, M, J, seed=N + J + 1)
    Y_ref = oracle.forward(T.astype(np.complex128), d.astype(np.complex128))
    errs = {}
    for prec in (tmr.TMR_PREC_FP32, MIXED):
        Y = torch.empty((M, J, N), dtype=torch.float32, device="cuda")
        with handle(N, M, J, d, precision=prec) as h:
            tmr.tmr_forward(h, to_dev(T), Y)
            torch.cuda.synchronize()
        errs[prec] = max(rel_l2_rows(to_np(Y), Y_ref), max_rel_elem_rows(to_np(Y), Y_ref))
    assert errs[MIXED] <= 1e-4, errs
    assert errs[tmr.TMR_PREC_FP32] <= 1e-5, errs


@pytest.mark.parametrize("N", [256, 1024, 2048, 4096])
def test_tensor_core_gradient(N):
    M, J = 4, 4
    T, d, _ = problem(N, M, J, seed=5 * N)
    _, _, Y = problem(N, M, J, seed=5 * N + 1)
    loss_ref, G_ref = oracle.loss_grad(T.astype(np.complex128), d.astype(np.complex128),
                                       Y.astype(np.float64))
    loss = torch.empty(M, dtype=torch.float32, device="cuda")
    G = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    with handle(N, M, J, d, precision=MIXED) as h:
        tmr.tmr_grad(h, to_dev(T), to_dev(Y), loss, G)
        torch.cuda.synchronize()
    assert np.max(np.abs(to_np(loss) - loss_ref) / loss_ref) <= 1e-4
    assert_rows_close(to_np(G), G_ref, 1e-4)


def test_mixed_rejects_other_lengths():
    _, d, _ = problem(512, 2, 4)
    with pytest.raises(tmr.TMRError) as ei:
        handle(512, 2, 4, d, precision=MIXED)
    assert ei.value.status == tmr.TMR_ERR_UNSUPPORTED
    _, d, _ = problem(256, 2, 4)
    with pytest.raises(tmr.TMRError) as ei:
        handle(256, 2, 4, d, precision=7)
    assert ei.value.status == tmr.TMR_ERR_INVALID_ARG


def test_mixed_learned_start_seeds_and_falls_back():
    """The learned start with mixed precision: a network whose proposals are
    all zero leaves every row on the Philox seed (the result equals the mixed
    spectral run bit for bit, no row counts as seeded); a network with nonzero
    proposals seeds every row."""
    N, M, J, iters = 256, 24, 4, 20
    T, d, Y = problem(N, M, J, seed=9)

    def run(init, model=None):
        To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        with handle(N, M, J, d, init=tmr.INIT[init], power_iters=40, precision=MIXED) as h:
            if model is not None:
                tmr.tmr_set_init_model(h, model)
            tmr.tmr_retrieve(h, to_dev(Y), None, iters, To)
            torch.cuda.synchronize()
            kept = tmr.tmr_learned_rows(h) if model is not None else None
        return to_np(To), kept

    with tmr.tmr_mlp_create(J * N, 64, 64, 2 * N, seed=5) as zero_net, \
            tmr.tmr_mlp_create(J * N, 64, 64, 2 * N, seed=5) as net:
        tmr.tmr_mlp_set_params(zero_net, np.zeros(zero_net.n_params, np.float32))
        plain, _ = run("spectral")
        z, kz = run("learned", zero_net)
        assert kz == 0
        np.testing.assert_array_equal(z, plain)
        _, ks = run("learned", net)
        assert ks == M


def test_mixed_vs_fp32_at_2048():
    """The plain workload's length and fiber model on 512 rows: mixed and FP32
    runs reach the same fidelity to the ground truth (mean within 1e-3)."""
    N, M, J, iters, pits = 2048, 512, 4, 100, 100
    T = c64(synth.tm_modes(M, N, 1100, seed=3, dtype=np.complex64))
    _, d = synth.mask_phases(J, N, seed=3)
    d = c64(d)
    Yg = torch.empty((M, J, N), dtype=torch.float32, device="cuda")
    fid = {}
    with handle(N, M, J, d) as h:
        tmr.tmr_forward(h, to_dev(T), Yg)
        torch.cuda.synchronize()
    Y = to_np(Yg)
    Yn = to_dev(f32(synth.shot_noise(Y, synth.photon_scale(float(Y.mean()), 1e4), seed=3)))
    for prec in (tmr.TMR_PREC_FP32, MIXED):
        To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        with handle(N, M, J, d, init=tmr.TMR_INIT_SPECTRAL, power_iters=pits, clip=2.0, precision=prec) as h:
            tmr.tmr_retrieve(h, Yn, None, iters, To)
            torch.cuda.synchronize()
        fid[prec] = oracle.fidelity_rows(to_np(To), T)
    assert np.mean(fid[MIXED]) >= 0.99
    assert abs(np.mean(fid[MIXED]) - np.mean(fid[tmr.TMR_PREC_FP32])) <= 1e-3
    assert abs(np.mean(fid[MIXED] >= 0.99) - np.mean(fid[tmr.TMR_PREC_FP32] >= 0.99)) <= 0.01


def _fp16_dequantised(Y):
    """What the handle keeps: each row divided by its largest |y|, rounded to
    FP16, times the row scale (numpy's float16 rounds to nearest even)."""
    Y = np.asarray(Y, np.float32)
    s = np.max(np.abs(Y.reshape(Y.shape[0], -1)), axis=1).astype(np.float32)
    s = np.where(s > 0, s, np.float32(1))
    q = (Y * (np.float32(1) / s)[:, None, None]).astype(np.float16).astype(np.float32)
    return q * s[:, None, None]


def test_mixed_small_retrieval():
    """Noiseless i.i.d. rows at N = 256, spectral start, 200 iterations (the
    last 10 in FP32): fidelity within 1e-3 of the oracle's on the FP32 data,
    and a final loss (FP32-evaluated, on the data the handle stores) at the
    FP16 quantisation floor."""
    N, M, J, iters, pits = 256, 48, 4, 200, 100
    T, d, Y = problem(N, M, J, seed=12)
    Tr, _, _, _ = oracle.retrieve_rows(Y, d.astype(np.complex128), iters, init="spectral",
                                       power_iters=pits, clip=2.0)
    To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    loss = torch.empty(M, dtype=torch.float32, device="cuda")
    st = torch.empty(M, dtype=torch.int32, device="cuda")
    with handle(N, M, J, d, init=tmr.TMR_INIT_SPECTRAL, power_iters=pits, clip=2.0, precision=MIXED) as h:
        tmr.tmr_retrieve(h, to_dev(Y), None, iters, To, st, None, loss)
        torch.cuda.synchronize()
    fid_g = oracle.fidelity_rows(to_np(To), T)
    fid_o = oracle.fidelity_rows(Tr, T)
    assert np.mean(np.abs(fid_g - fid_o) <= 1e-3) >= 0.95, (fid_g, fid_o)
    Yq = _fp16_dequantised(Y)
    floor = np.sum((Yq.astype(np.float64) - Y) ** 2, axis=(1, 2))  # f(T_true) on the stored data
    ok = (fid_o > 0.9999) & (fid_g > 0.9999)
    assert ok.mean() >= 0.5
    assert np.all(to_np(loss)[ok] <= 2.0 * floor[ok] + 1e-6 * np.sum(Y[ok] ** 2, axis=(1, 2)))


def test_mixed_numeric_and_zero_rows():
    N, M, J = 256, 4, 4
    T, d, Y = problem(N, M, J, seed=13)
    Y = Y.copy()
    Y[0] = 0.0
    Y[2, 1, 5] = np.inf
    To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    st = torch.empty(M, dtype=torch.int32, device="cuda")
    with handle(N, M, J, d, precision=MIXED) as h:
        tmr.tmr_retrieve(h, to_dev(Y), None, 30, To, st)
        torch.cuda.synchronize()
    s = to_np(st)
    assert s[0] == tmr.TMR_ROW_ZERO and s[2] == tmr.TMR_ROW_NUMERIC
    assert np.all(np.isfinite(to_np(To)))


def test_precision_workload_sampled_rows():
    """N = 4096, M = 16384 (128 x 128), J = 4, mode model R = 2200, Poisson
    1e4, spectral start, 100 iterations (the last 10 FP32).  Stated error of
    the mixed path: against the FP32 GPU path on every row (fidelity to the
    ground truth and to each other), against the FP64 oracle on 4 sampled
    rows at a short budget from the same intensities, and, per transform
    (forward model, loss, gradient), against the oracle on 256 sampled rows."""
    cfg = synth.CONFIGS["precision"]
    N, M, J = cfg["N"], cfg["M"], cfg["J"]
    T = c64(synth.tm_modes(M, N, cfg["R"], seed=0, dtype=np.complex64))
    _, d = synth.mask_phases(J, N, seed=0)
    d = c64(d)
    rows = synth.sample_rows(M, 4, seed=0)
    pits, iters = 100, cfg["iters"]
    Yg = torch.empty((M, J, N), dtype=torch.float32, device="cuda")
    out = {}
    with handle(N, M, J, d, init=tmr.TMR_INIT_SPECTRAL, power_iters=pits, clip=2.0) as h:
        tmr.tmr_forward(h, to_dev(T), Yg)
        torch.cuda.synchronize()
        Y_clean = to_np(Yg)
        del Yg
        scale = synth.photon_scale(float(Y_clean.mean()), cfg["photons"])
        Yn = torch.from_numpy(f32(synth.shot_noise(Y_clean, scale, seed=0))).cuda()
        To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        tmr.tmr_retrieve(h, Yn, None, iters, To)
        torch.cuda.synchronize()
        out["fp32"] = to_np(To)
    with handle(N, M, J, d, init=tmr.TMR_INIT_SPECTRAL, power_iters=pits, clip=2.0, precision=MIXED) as h:
        To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        tmr.tmr_retrieve(h, Yn, None, iters, To)
        torch.cuda.synchronize()
        out["mixed"] = to_np(To)
    fid32 = oracle.fidelity_rows(out["fp32"], T)
    fidmx = oracle.fidelity_rows(out["mixed"], T)
    assert np.mean(fidmx) >= 0.99 and np.mean(fidmx >= 0.99) >= np.mean(fid32 >= 0.99) - 0.01
    assert abs(np.mean(fidmx) - np.mean(fid32)) <= 1e-3
    # short budget on the sampled rows: mixed path vs the oracle
    short = 15
    Ys = Yn[torch.from_numpy(rows).cuda()].contiguous()
    Tm = torch.empty((len(rows), N), dtype=torch.complex64, device="cuda")
    with handle(N, len(rows), J, d, init=tmr.TMR_INIT_SPECTRAL, power_iters=30, clip=2.0,
                precision=MIXED) as h:
        tmr.tmr_retrieve(h, Ys, None, short, Tm)
        torch.cuda.synchronize()
    Tr, _, _, _ = oracle.retrieve_rows(to_np(Ys), d.astype(np.complex128), short, init="spectral",
                                       power_iters=30, clip=2.0)
    fm = oracle.fidelity_rows(to_np(Tm), T[rows])
    fo = oracle.fidelity_rows(Tr, T[rows])
    assert np.mean(np.abs(fm - fo) <= 1e-3) >= 3 / 4, (fm, fo)
    # per-transform error of the mixed arithmetic against the FP64 oracle on 256
    # sampled rows of the workload: intensities of the true rows, and the loss
    # and gradient at rows perturbed by 30 % of their norm (large residuals)
    r256 = synth.sample_rows(M, 256, seed=2)
    Tt = T[r256]
    rng = np.random.default_rng(3)
    Tp = c64(Tt + 0.3 * (rng.standard_normal(Tt.shape) + 1j * rng.standard_normal(Tt.shape)) / np.sqrt(2 * N))
    Y_or = oracle.forward(Tt.astype(np.complex128), d.astype(np.complex128))
    loss_or, G_or = oracle.loss_grad(Tp.astype(np.complex128), d.astype(np.complex128), Y_or)
    Yg = torch.empty((256, J, N), dtype=torch.float32, device="cuda")
    lg = torch.empty(256, dtype=torch.float32, device="cuda")
    Gg = torch.empty((256, N), dtype=torch.complex64, device="cuda")
    with handle(N, 256, J, d, precision=MIXED) as h:
        tmr.tmr_forward(h, to_dev(Tt), Yg)
        tmr.tmr_grad(h, to_dev(Tp), to_dev(f32(Y_or)), lg, Gg)
        torch.cuda.synchronize()
    e_fwd = max(rel_l2_rows(to_np(Yg), Y_or), max_rel_elem_rows(to_np(Yg), Y_or))
    e_loss = float(np.max(np.abs(to_np(lg) - loss_or) / loss_or))
    e_grad = max(rel_l2_rows(to_np(Gg), G_or), max_rel_elem_rows(to_np(Gg), G_or))
    print(f"mixed vs FP64 oracle on 256 rows (N = 4096): forward {e_fwd:.2e}, loss {e_loss:.2e}, "
          f"gradient {e_grad:.2e}")
    assert e_fwd <= 1e-4 and e_loss <= 1e-4 and e_grad <= 1e-4
