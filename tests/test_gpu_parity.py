"""GPU (libtmr, sm_103a) against the FP64 oracle, element by element on the same
seeded inputs, through the C ABI.  Bars: forward/gradient relative error
<= 1e-5 (FP32 arithmetic), recovered-row fidelity within 1e-3 of the oracle's."""
import numpy as np
import pytest

import oracle
import synth
from helpers import c64, f32, problem, assert_rows_close, rel_l2_rows, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2302_13524_gb300 as tmr  # noqa: E402

ALL_N = [64, 128, 256, 512, 1024, 2048, 4096]


def handle(N, M, J, d, dop=None, **opt):
    return tmr.tmr_create(N, M, J, to_dev(d), dop, opt or None)


# ------------------------------------------------------------ forward model
@pytest.mark.parametrize("N", ALL_N)
@pytest.mark.parametrize("J", [4, 3])
def test_forward_parity(N, J):
    M = 5
    T, d, _ = problem(N, M, J, seed=N + J)
    Y_ref = oracle.forward(T.astype(np.complex128), d.astype(np.complex128))
    Y = torch.empty((M, J, N), dtype=torch.float32, device="cuda")
    with handle(N, M, J, d) as h:
        tmr.tmr_forward(h, to_dev(T), Y)
        torch.cuda.synchronize()
    assert_rows_close(to_np(Y), Y_ref, 1e-5)


@pytest.mark.parametrize("N", ALL_N)
def test_grad_parity(N):
    M, J = 6, 4
    T, d, _ = problem(N, M, J, seed=3 * N)
    _, _, Y = problem(N, M, J, seed=3 * N + 1)  # intensities of another TM: large residuals
    _, d2, _ = problem(N, M, J, seed=3 * N)
    loss_ref, G_ref = oracle.loss_grad(T.astype(np.complex128), d.astype(np.complex128),
                                       Y.astype(np.float64))
    loss = torch.empty(M, dtype=torch.float32, device="cuda")
    G = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    with handle(N, M, J, d) as h:
        tmr.tmr_grad(h, to_dev(T), to_dev(Y), loss, G)
        torch.cuda.synchronize()
    assert np.max(np.abs(to_np(loss) - loss_ref) / loss_ref) <= 1e-5
    assert_rows_close(to_np(G), G_ref, 1e-5)


def test_grad_host_buffers_match_device():
    N, M, J = 256, 7, 4
    T, d, Y = problem(N, M, J, seed=11)
    T2 = c64(T * 0.9 + 0.01)
    lossh = np.empty(M, np.float32)
    Gh = np.empty((M, N), np.complex64)
    with handle(N, M, J, d) as h:
        tmr.tmr_grad(h, T2, Y, lossh, Gh)  # host arrays: staged by the library
        G = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        tmr.tmr_grad(h, to_dev(T2), to_dev(Y), None, G)
        torch.cuda.synchronize()
    np.testing.assert_array_equal(Gh, to_np(G))
    loss_ref, _ = oracle.loss_grad(T2.astype(np.complex128), d.astype(np.complex128), Y)
    assert np.max(np.abs(lossh - loss_ref) / loss_ref) <= 1e-5


# ------------------------------------------------------------ initialisation
@pytest.mark.parametrize("N,J", [(64, 4), (2048, 4), (512, 3), (1024, 8)])
@pytest.mark.parametrize("init,pits,tol", [("random", 0, 1e-5), ("bp", 0, 1e-5),
                                           ("spectral", 10, 1e-4)])
def test_init_parity(N, J, init, pits, tol):
    M = 6
    _, d, Y = problem(N, M, J, seed=N + 7 * J)
    T0_ref = oracle.init(Y, d.astype(np.complex128), init, seed=42, power_iters=pits, clip=2.0)
    T0 = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    with handle(N, M, J, d, init=tmr.INIT[init], seed=42, power_iters=pits, clip=2.0) as h:
        tmr.tmr_retrieve(h, to_dev(Y), None, 0, T0)
        torch.cuda.synchronize()
    assert_rows_close(to_np(T0), T0_ref, tol)


# ------------------------------------------------------------ L-BFGS steps
@pytest.mark.parametrize("N,J", [(256, 4), (2048, 4), (128, 3)])
def test_first_step_parity(N, J):
    M = 4
    T, d, Y = problem(N, M, J, seed=5 + N)
    rng = np.random.default_rng(N)
    T_init = c64(T + 0.3 * (rng.standard_normal(T.shape) + 1j * rng.standard_normal(T.shape)) / np.sqrt(N))
    Tn = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    loss = torch.empty(M, dtype=torch.float32, device="cuda")
    with handle(N, M, J, d) as h:
        tmr.tmr_retrieve_from(h, to_dev(T_init), to_dev(Y), None, 1, Tn, row_loss=loss)
        torch.cuda.synchronize()
    for r in range(M):
        ref = oracle.lbfgs_step(Y[r].astype(np.float64), d.astype(np.complex128),
                                T_init[r].astype(np.complex128))
        assert_rows_close(to_np(Tn)[r:r + 1], ref["t"][None], 1e-5)
        assert abs(to_np(loss)[r] - ref["loss"]) <= 1e-4 * ref["loss"] + 1e-6 * np.sum(Y[r] ** 2)


@pytest.mark.parametrize("iters", [2, 5, 12])
def test_few_steps_parity(iters):
    N, M, J = 512, 6, 4
    T, d, Y = problem(N, M, J, seed=iters)
    rng = np.random.default_rng(iters)
    T_init = c64(T + 0.3 * (rng.standard_normal(T.shape) + 1j * rng.standard_normal(T.shape)) / np.sqrt(N))
    Tn = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    its = torch.empty(M, dtype=torch.int32, device="cuda")
    with handle(N, M, J, d) as h:
        tmr.tmr_retrieve_from(h, to_dev(T_init), to_dev(Y), None, iters, Tn, row_iters=its)
        torch.cuda.synchronize()
    Tr, _, it_ref, _ = oracle.retrieve_rows(Y, d.astype(np.complex128), iters, T_init=T_init)
    assert np.all(to_np(its) == it_ref)
    assert_rows_close(to_np(Tn), Tr, 1e-4 * iters)


# ------------------------------------------------------------ whole path, tiny
def _tiny_inputs(init):
    cfg = synth.CONFIGS["tiny"]
    N, M, J = cfg["N"], cfg["M"], cfg["J"]
    T, d, Y = problem(N, M, J, seed=0)
    Nd = cfg["n_defocus"]
    C = oracle.defocus_fields(T.astype(np.complex128), d.astype(np.complex128), Nd)
    Yd = f32(oracle.defocus_forward(C, cfg["grid"], coef=cfg["defocus_coef"]))
    return cfg, T, d, Y, Yd


@pytest.mark.parametrize("init", ["random", "spectral"])
def test_tiny_whole_path_parity(init):
    cfg, T, d, Y, Yd = _tiny_inputs(init)
    N, M, J, Nd = cfg["N"], cfg["M"], cfg["J"], cfg["n_defocus"]
    ny, nx = cfg["grid"]
    iters = cfg["iters"]
    ref = oracle.retrieve_tm(Y, d.astype(np.complex128), Yd, cfg["grid"], iters, init=init, seed=0,
                             power_iters=50, clip=2.0, coef=cfg["defocus_coef"])
    To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    st = torch.empty(M, dtype=torch.int32, device="cuda")
    dop = dict(ny=ny, nx=nx, n_defocus=Nd, coef=cfg["defocus_coef"])
    with handle(N, M, J, d, dop, init=tmr.INIT[init], seed=0, power_iters=50, clip=2.0) as h:
        tmr.tmr_retrieve(h, to_dev(Y), to_dev(Yd), iters, To, row_status=st)
        tmr.tmr_sync(h, 60.0)
    Tg = to_np(To)
    fid_g = oracle.fidelity_rows(Tg, T)
    fid_o = oracle.fidelity_rows(ref["T"], T)
    close = np.abs(fid_g - fid_o) <= 1e-3
    # per-row fidelity within 1e-3 of the oracle's and equal failure counts,
    # each to within 1 % of the rows (1 of 128): a row whose FP32 and FP64
    # trajectories part at a bifurcation of the non-convex landscape may settle
    # differently.  (The oracle itself moves no row under relative changes of
    # 6e-8 to y, so the bar is not looser than its own spread.)
    n_off = int(np.sum(~close))
    n_fail_g, n_fail_o = int(np.sum(fid_g < 0.99)), int(np.sum(fid_o < 0.99))
    print(f"{init}: rows off by > 1e-3: {n_off}; failures gpu {n_fail_g} oracle {n_fail_o}")
    assert n_off <= int(0.01 * M), (fid_g, fid_o)
    assert abs(n_fail_g - n_fail_o) <= int(0.01 * M)
    if init == "spectral":
        assert np.mean(fid_g) >= 0.97
        # the phase fit ties the rows together: one global phase is left
        ok = (fid_o > 0.999) & (fid_g > 0.999)
        mf_g = oracle.matrix_fidelity(Tg[ok], T[ok])
        mf_o = oracle.matrix_fidelity(ref["T"][ok], T[ok])
        assert mf_o > 0.999 and abs(mf_g - mf_o) <= 1e-3


# ------------------------------------------------------------ defocus
def test_defocus_forward_parity():
    cfg, T, d, Y, Yd = _tiny_inputs("random")
    N, M, J, Nd = cfg["N"], cfg["M"], cfg["J"], cfg["n_defocus"]
    ny, nx = cfg["grid"]
    out = torch.empty((Nd, M), dtype=torch.float32, device="cuda")
    with handle(N, M, J, d, dict(ny=ny, nx=nx, n_defocus=Nd, coef=0.05)) as h:
        tmr.tmr_defocus_forward(h, to_dev(T), out)
        torch.cuda.synchronize()
    assert_rows_close(to_np(out), Yd, 1e-5)


@pytest.mark.parametrize("grid,Nd", [((16, 8), 24), ((32, 32), 50)])
def test_phase_fit_parity_planted(grid, Nd):
    ny, nx = grid
    M, N, J = ny * nx, 64, 4
    T, d, _ = problem(N, M, J, seed=ny)
    C = oracle.defocus_fields(T.astype(np.complex128), d.astype(np.complex128), Nd)
    Yd = f32(oracle.defocus_forward(C, grid))
    rng = np.random.default_rng(1)
    phi_star = rng.uniform(-np.pi, np.pi, M)
    T_est = c64(np.exp(-1j * phi_star)[:, None] * T)
    C_est = oracle.defocus_fields(T_est.astype(np.complex128), d.astype(np.complex128), Nd)
    wts = np.sum(np.abs(T_est.astype(np.complex128)) ** 2, axis=1)
    phi_o, _, _ = oracle.phase_fit(C_est, Yd, grid, iters=100, weights=wts)
    phi = torch.empty(M, dtype=torch.float64, device="cuda")
    To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    with handle(N, M, J, d, dict(ny=ny, nx=nx, n_defocus=Nd, coef=0.05), phase_iters=100) as h:
        tmr.tmr_defocus_fit(h, to_dev(T_est), to_dev(Yd), phi, To)
        tmr.tmr_sync(h, 60.0)
    err = np.angle(np.exp(1j * (to_np(phi) - phi_o)))
    assert np.max(np.abs(err)) <= 1e-4
    assert oracle.matrix_fidelity(to_np(To), T) >= 1 - 1e-6


# ------------------------------------------------------------ edge cases
def test_zero_nan_and_ragged_rows():
    N, M, J = 256, 37, 4  # 37 rows: not a multiple of the cluster count
    T, d, Y = problem(N, M, J, seed=9)
    Y = Y.copy()
    Y[3] = 0
    Y[10, 2, 5] = np.nan
    To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    st = torch.empty(M, dtype=torch.int32, device="cuda")
    its = torch.empty(M, dtype=torch.int32, device="cuda")
    with handle(N, M, J, d, init=tmr.TMR_INIT_SPECTRAL, power_iters=60) as h:
        tmr.tmr_retrieve(h, to_dev(Y), None, 40, To, st, its)
        with pytest.raises(tmr.TMRError) as ei:
            tmr.tmr_sync(h, 60.0)
        assert ei.value.status == tmr.TMR_ERR_NUMERIC
    s = to_np(st)
    assert s[3] == tmr.TMR_ROW_ZERO and np.all(to_np(To)[3] == 0) and to_np(its)[3] == 0
    assert s[10] == tmr.TMR_ROW_NUMERIC and np.all(to_np(To)[10] == 0)
    rest = [r for r in range(M) if r not in (3, 10)]
    assert np.all(np.isin(s[rest], [tmr.TMR_ROW_MAXITER, tmr.TMR_ROW_CONVERGED]))
    _, _, it_o, st_o = oracle.retrieve_rows(Y, d.astype(np.complex128), 40, init="spectral",
                                            power_iters=60)
    assert st_o[3] == oracle.ROW_ZERO and st_o[10] == oracle.ROW_NUMERIC


def test_invalid_arguments():
    N, M, J = 64, 4, 4
    _, d, Y = problem(N, M, J)
    for bad_n in (8, 5000):  # outside 16..4096
        with pytest.raises(tmr.TMRError) as ei:
            tmr.tmr_create(bad_n, M, J, to_dev(np.ones(J * bad_n, np.complex64)))
        assert ei.value.status == tmr.TMR_ERR_UNSUPPORTED
    with pytest.raises(tmr.TMRError) as ei:
        tmr.tmr_create(N, M, 9, to_dev(np.ones(9 * N, np.complex64)))
    assert ei.value.status == tmr.TMR_ERR_UNSUPPORTED
    with pytest.raises(tmr.TMRError) as ei:
        tmr.tmr_create(N, M, J, to_dev(d), dict(ny=3, nx=1, n_defocus=2))
    assert ei.value.status == tmr.TMR_ERR_INVALID_ARG
    with handle(N, M, J, d) as h:
        To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        with pytest.raises(tmr.TMRError) as ei:
            tmr.tmr_retrieve(h, to_dev(Y), None, -1, To)
        assert ei.value.status == tmr.TMR_ERR_INVALID_ARG
    with pytest.raises(tmr.TMRError) as ei:
        tmr.tmr_create(N, M, J, to_dev(d), opt=dict(workspace_limit=1024))
    assert ei.value.status == tmr.TMR_ERR_OOM


# ------------------------------------------------------------ full size, sampled rows
def test_plain_full_size_sampled_rows():
    """The plain workload (N=2048, M=8192, J=4, mode model, Poisson 1e4) in the
    launch configuration the benchmark times; the oracle recomputes 32 sampled
    rows one by one, and every one of them must end within 1e-3 of the
    oracle's fidelity."""
    cfg = synth.CONFIGS["plain"]
    N, M, J = cfg["N"], cfg["M"], cfg["J"]
    T = c64(synth.tm_modes(M, N, cfg["R"], seed=0))
    _, d = synth.mask_phases(J, N, seed=0)
    d = c64(d)
    Yg = torch.empty((M, J, N), dtype=torch.float32, device="cuda")
    iters, pits = 30, 100
    rows = synth.sample_rows(M, 32, seed=0)
    with handle(N, M, J, d, init=tmr.TMR_INIT_SPECTRAL, power_iters=pits, clip=2.0) as h:
        tmr.tmr_forward(h, to_dev(T), Yg)
        torch.cuda.synchronize()
        Y_clean = to_np(Yg)
        Y_or = oracle.forward(T[rows].astype(np.complex128), d.astype(np.complex128))
        assert_rows_close(Y_clean[rows], Y_or, 1e-5)
        scale = synth.photon_scale(float(Y_clean.mean()), cfg["photons"])
        Yn = f32(synth.shot_noise(Y_clean, scale, seed=0))
        To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        tmr.tmr_retrieve(h, to_dev(Yn), None, iters, To)
        torch.cuda.synchronize()
    Tg = to_np(To)
    Yn_o = f32(synth.shot_noise(Y_or, scale, seed=0, row_ids=rows))
    Tr, _, _, _ = oracle.retrieve_rows(Yn_o, d.astype(np.complex128), iters, init="spectral",
                                       power_iters=pits, clip=2.0, row_ids=rows)
    fid_g = oracle.fidelity_rows(Tg[rows], T[rows])
    fid_o = oracle.fidelity_rows(Tr, T[rows])
    assert np.all(np.abs(fid_g - fid_o) <= 1e-3), (fid_g, fid_o)
    assert np.sum(fid_g < 0.99) == np.sum(fid_o < 0.99)
    fid_all = oracle.fidelity_rows(Tg, T)
    assert np.mean(fid_all) >= 0.98


# ------------------------------------------------------------ torch wrapper
def test_retriever_matches_the_functions():
    """The Retriever class is marshalling only: its outputs equal those of the
    C-ABI functions bit for bit, and it refuses tensors of the wrong dtype,
    shape, device or layout."""
    N, M, J, Nd, grid = 256, 16, 4, 20, (4, 4)
    T, d, Y = problem(N, M, J, seed=31)
    C = oracle.defocus_fields(T.astype(np.complex128), d.astype(np.complex128), Nd)
    Yd = f32(oracle.defocus_forward(C, grid, coef=0.05))
    dop = dict(ny=grid[0], nx=grid[1], n_defocus=Nd, coef=0.05)
    opt = dict(init=tmr.TMR_INIT_SPECTRAL, power_iters=30)
    Tg, Yg, Ydg, dg = to_dev(T), to_dev(Y), to_dev(Yd), to_dev(d)
    with tmr.Retriever(dg, M, dop, **opt) as r:
        Yr = r.forward(Tg)
        lr, Gr = r.grad(Tg, Yg)
        out = r.retrieve(Yg, Ydg, 25)
        Ydr = r.defocus_forward(Tg)
        with pytest.raises(TypeError):
            r.forward(Tg.to(torch.complex128))
        with pytest.raises(ValueError):
            r.forward(Tg[:, :N // 2])
        with pytest.raises(ValueError):
            r.forward(Tg.cpu())
        with pytest.raises(ValueError):
            r.retrieve(to_dev(np.ascontiguousarray(Y.transpose(0, 2, 1))).transpose(1, 2), None, 5)
        torch.cuda.synchronize()
    with handle(N, M, J, d, dop, **opt) as h:
        Yf = torch.empty_like(Yr)
        tmr.tmr_forward(h, Tg, Yf)
        lf = torch.empty_like(lr)
        Gf = torch.empty_like(Gr)
        tmr.tmr_grad(h, Tg, Yg, lf, Gf)
        Tf = torch.empty_like(out["T"])
        sf = torch.empty_like(out["status"])
        tmr.tmr_retrieve(h, Yg, Ydg, 25, Tf, sf)
        Ydf = torch.empty_like(Ydr)
        tmr.tmr_defocus_forward(h, Tg, Ydf)
        torch.cuda.synchronize()
    for a, b in ((Yr, Yf), (lr, lf), (Gr, Gf), (out["T"], Tf), (out["status"], sf), (Ydr, Ydf)):
        np.testing.assert_array_equal(to_np(a), to_np(b))


def test_intensity_scale_invariance():
    """f(c t') with y' = c^2 y is c^4 f(t'), so the minimiser scales by sqrt(c)
    (Eq. optTMsmall2).  A power-of-two scale passes through the row
    normalisation exactly: T(4096 y) = 64 T(y) and the loss 2^24 times, bit for
    bit.  Photon-count scale (y ~ 1e4 per pixel, where the quartic's c4 would
    leave FP32 range without the normalisation) gives the same fidelities."""
    N, M, J, iters = 1024, 6, 4, 60
    T, d, Y = problem(N, M, J, seed=61, tm="modes", R=300)
    opt = dict(init=tmr.TMR_INIT_SPECTRAL, power_iters=50)

    def run(Yin):
        To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        st = torch.empty(M, dtype=torch.int32, device="cuda")
        it = torch.empty(M, dtype=torch.int32, device="cuda")
        lo = torch.empty(M, dtype=torch.float32, device="cuda")
        with handle(N, M, J, d, **opt) as h:
            tmr.tmr_retrieve(h, to_dev(f32(Yin)), None, iters, To, st, it, lo)
            torch.cuda.synchronize()
        return to_np(To), to_np(st), to_np(it), to_np(lo)

    T1, s1, i1, l1 = run(Y)
    T2, s2, i2, l2 = run(Y * np.float32(4096.0))
    assert np.array_equal(T2, T1 * np.float32(64.0))
    assert np.array_equal(l2, l1 * np.float32(2.0 ** 24))
    assert np.array_equal(s1, s2) and np.array_equal(i1, i2)
    T3, s3, i3, _ = run(Y * np.float32(1e4 / Y.mean()))
    f1 = oracle.fidelity_rows(T1, T)
    f3 = oracle.fidelity_rows(T3, T)
    assert (i3 > 5).all() and np.median(f1) > 0.99  # no row stopped at the start
    np.testing.assert_allclose(f3, f1, atol=1e-3)


# ------------------------------------------------------------ bounded waits
def test_phase_fit_wait_runs_out_and_reports_timeout():
    """The fit's grid barrier is held shut (test hook): every CTA's wait runs
    out after wait_spins polls, the kernel returns, phi is left at its last
    value (zero, the start) and tmr_sync reports TIMEOUT; the context stays
    usable and a handle without the hook fits normally afterwards."""
    ny, nx, Nd = 16, 8, 24
    M, N, J = ny * nx, 64, 4
    T, d, _ = problem(N, M, J, seed=71)
    C = oracle.defocus_fields(T.astype(np.complex128), d.astype(np.complex128), Nd)
    Yd = f32(oracle.defocus_forward(C, (ny, nx)))
    dop = dict(ny=ny, nx=nx, n_defocus=Nd, coef=0.05)
    phi = torch.full((M,), float("nan"), dtype=torch.float64, device="cuda")
    To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    with handle(N, M, J, d, dop, withhold_release=1, wait_spins=1 << 14) as h:
        tmr.tmr_defocus_fit(h, to_dev(T), to_dev(Yd), phi, To)
        with pytest.raises(tmr.TMRError) as ei:
            tmr.tmr_sync(h, 60.0)
        assert ei.value.status == tmr.TMR_ERR_TIMEOUT
        assert "grid barrier" in str(ei.value)
    torch.cuda.synchronize()
    assert np.all(to_np(phi) == 0.0)
    np.testing.assert_array_equal(to_np(To), T)  # diag(e^{i 0}) T
    with handle(N, M, J, d, dop, phase_iters=20) as h:
        tmr.tmr_defocus_fit(h, to_dev(T), to_dev(Yd), phi, To)
        tmr.tmr_sync(h, 60.0)
    assert np.all(np.isfinite(to_np(phi)))
    with pytest.raises(tmr.TMRError) as ei:
        handle(N, M, J, d, dop, wait_spins=0)
    assert ei.value.status == tmr.TMR_ERR_INVALID_ARG


def test_sync_wall_clock_limit_on_a_long_launch():
    """tmr_sync gives up after its wall-clock limit while the retrieve still
    runs (TIMEOUT), and a later tmr_sync with a longer limit returns OK once
    the work is done."""
    N, M, J = 2048, 4096, 4
    _, d, _ = problem(N, 2, J, seed=72)
    rng = np.random.default_rng(72)
    Y = torch.from_numpy(rng.exponential(1.0, (M, J, N)).astype(np.float32)).cuda()
    To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    with handle(N, M, J, d, power_iters=100, schedule=2) as h:
        torch.cuda.synchronize()
        tmr.tmr_retrieve(h, Y, None, 300, To)
        with pytest.raises(tmr.TMRError) as ei:
            tmr.tmr_sync(h, 1e-3)
        assert ei.value.status == tmr.TMR_ERR_TIMEOUT
        tmr.tmr_sync(h, 120.0)
    assert np.all(np.isfinite(to_np(To)))
