"""Lengths N that are not powers of two (Bluestein transforms, 16 <= N <= 4096)
against the FP64 oracle through the C ABI: forward model, gradient, starts,
L-BFGS steps, a whole small retrieval, and the uneven-convergence workload
(N = 2286 = 2 * 3^2 * 127, M = 8192) in one launch with sampled rows.

The oracle's DFT is the naive O(N^2) sum for every N, so it shares nothing
with the chirp-z route the library takes."""
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

# one length per Bluestein shape: L = 512 .. 4096; the split-output form at
# L = 4096 with 5 and 6 registers per thread (2286 is the uneven-convergence
# workload's length, 2731 the largest split length); L = 8192 with 6..8
BLUE_N = [17, 100, 300, 1000, 1500, 2286, 2600, 2731, 2732, 3000, 3500, 4095]


def handle(N, M, J, d, dop=None, **opt):
    return tmr.tmr_create(N, M, J, to_dev(d), dop, opt or None)


@pytest.mark.parametrize("N", BLUE_N)
@pytest.mark.parametrize("J", [4, 3])
def test_forward_parity(N, J):
    M = 3
    T, d, _ = problem(N, M, J, seed=N + J)
    Y_ref = oracle.forward(T.astype(np.complex128), d.astype(np.complex128))
    Y = torch.empty((M, J, N), dtype=torch.float32, device="cuda")
    with handle(N, M, J, d) as h:
        tmr.tmr_forward(h, to_dev(T), Y)
        torch.cuda.synchronize()
    assert_rows_close(to_np(Y), Y_ref, 1e-5)


@pytest.mark.parametrize("N", BLUE_N)
def test_grad_parity(N):
    M, J = 3, 4
    T, d, _ = problem(N, M, J, seed=3 * N)
    _, _, Y = problem(N, M, J, seed=3 * N + 1)  # another TM's intensities: large residuals
    loss_ref, G_ref = oracle.loss_grad(T.astype(np.complex128), d.astype(np.complex128),
                                       Y.astype(np.float64))
    loss = torch.empty(M, dtype=torch.float32, device="cuda")
    G = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    with handle(N, M, J, d) as h:
        tmr.tmr_grad(h, to_dev(T), to_dev(Y), loss, G)
        torch.cuda.synchronize()
    assert np.max(np.abs(to_np(loss) - loss_ref) / loss_ref) <= 1e-5
    assert_rows_close(to_np(G), G_ref, 1e-5)


@pytest.mark.parametrize("N,J", [(100, 4), (2286, 4), (1500, 3)])
@pytest.mark.parametrize("init,pits,tol", [("random", 0, 1e-5), ("bp", 0, 1e-5),
                                           ("spectral", 10, 1e-4)])
def test_init_parity(N, J, init, pits, tol):
    M = 3
    _, d, Y = problem(N, M, J, seed=N + 7 * J)
    T0_ref = oracle.init(Y, d.astype(np.complex128), init, seed=42, power_iters=pits, clip=2.0)
    T0 = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    with handle(N, M, J, d, init=tmr.INIT[init], seed=42, power_iters=pits, clip=2.0) as h:
        tmr.tmr_retrieve(h, to_dev(Y), None, 0, T0)
        torch.cuda.synchronize()
    assert_rows_close(to_np(T0), T0_ref, tol)


def _perturbed(T, N, seed):
    rng = np.random.default_rng(seed)
    return c64(T + 0.3 * (rng.standard_normal(T.shape) + 1j * rng.standard_normal(T.shape)) / np.sqrt(N))


@pytest.mark.parametrize("N,J", [(300, 4), (2286, 4), (1000, 3)])
def test_first_step_parity(N, J):
    M = 3
    T, d, Y = problem(N, M, J, seed=5 + N)
    T_init = _perturbed(T, N, N)
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


@pytest.mark.parametrize("iters", [3, 10])
def test_few_steps_parity(iters):
    N, M, J = 300, 5, 4
    T, d, Y = problem(N, M, J, seed=iters + 1)
    T_init = _perturbed(T, N, iters)
    Tn = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    its = torch.empty(M, dtype=torch.int32, device="cuda")
    with handle(N, M, J, d) as h:
        tmr.tmr_retrieve_from(h, to_dev(T_init), to_dev(Y), None, iters, Tn, row_iters=its)
        torch.cuda.synchronize()
    Tr, _, it_ref, _ = oracle.retrieve_rows(Y, d.astype(np.complex128), iters, T_init=T_init)
    assert np.all(to_np(its) == it_ref)
    assert_rows_close(to_np(Tn), Tr, 1e-4 * iters)


def test_small_whole_retrieval_parity():
    """Noiseless i.i.d. rows at N = 100 (L = 512), random start, 200
    iterations: per-row fidelity against the oracle's."""
    N, M, J, iters = 100, 48, 4, 200
    T, d, Y = problem(N, M, J, seed=21)
    Tr, _, _, _ = oracle.retrieve_rows(Y, d.astype(np.complex128), iters, init="random", seed=3)
    To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    with handle(N, M, J, d, init=tmr.TMR_INIT_RANDOM, seed=3) as h:
        tmr.tmr_retrieve(h, to_dev(Y), None, iters, To)
        torch.cuda.synchronize()
    fid_g = oracle.fidelity_rows(to_np(To), T)
    fid_o = oracle.fidelity_rows(Tr, T)
    assert np.mean(np.abs(fid_g - fid_o) <= 1e-3) >= 0.95, (fid_g, fid_o)
    assert abs(np.mean(fid_g >= 0.99) - np.mean(fid_o >= 0.99)) <= 0.05


def test_zero_nan_and_ragged_rows():
    N, M, J = 1000, 5, 4
    T, d, Y = problem(N, M, J, seed=2)
    Y = Y.copy()
    Y[1] = 0.0
    Y[3, 2, 17] = np.nan
    To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    st = torch.empty(M, dtype=torch.int32, device="cuda")
    with handle(N, M, J, d) as h:
        tmr.tmr_retrieve(h, to_dev(Y), None, 30, To, row_status=st)
        torch.cuda.synchronize()
    s = to_np(st)
    assert s[1] == tmr.TMR_ROW_ZERO and s[3] == tmr.TMR_ROW_NUMERIC
    assert np.all(to_np(To)[1] == 0) and np.all(to_np(To)[3] == 0)
    fid = oracle.fidelity_rows(to_np(To)[[0, 2, 4]], T[[0, 2, 4]])
    assert np.all(np.isfinite(fid))


def test_early_exit_uneven_rows_length_300():
    """Uneven photon levels at a non-power-of-two length: rows stop at their own
    iteration inside one launch; statuses follow the oracle."""
    N, M, J, cap, tol = 300, 32, 4, 300, 1e-7
    T = c64(synth.tm_iid(M, N, 4))
    _, d = synth.mask_phases(J, N, 4)
    d = c64(d)
    Yc = oracle.forward(T.astype(np.complex128), d.astype(np.complex128))
    ph = synth.row_photons(dict(photons=(1e3, 1e5)), M, seed=4)
    Y = f32(synth.shot_noise(Yc, synth.photon_scale(Yc.mean(), ph), seed=4))
    To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    st = torch.empty(M, dtype=torch.int32, device="cuda")
    its = torch.empty(M, dtype=torch.int32, device="cuda")
    with tmr.tmr_create(N, M, J, to_dev(d), None, dict(tol=tol, power_iters=60)) as h:
        tmr.tmr_retrieve(h, to_dev(Y), None, cap, To, st, its)
        torch.cuda.synchronize()
    its_g, st_g = to_np(its), to_np(st)
    assert np.all((st_g == tmr.TMR_ROW_CONVERGED) == (its_g < cap))
    assert its_g.max() > its_g.min()
    _, _, it_o, st_o = oracle.retrieve_rows(Y, d.astype(np.complex128), cap, init="spectral",
                                            power_iters=60, tol=tol)
    assert np.mean(oracle.fidelity_rows(to_np(To), T)) >= 0.97
    assert abs(np.mean(st_g == 1) - np.mean(st_o == 1)) <= 0.15


def test_batching_full_size_sampled_rows():
    """The uneven-convergence workload (N = 2286, M = 8192, J = 4, mode model
    R = 1100, per-row photons log-uniform 1e3..1e5, early exit 1e-7, cap 300)
    in one launch; the oracle recomputes 4 sampled rows at a short budget from
    the same intensities, and the whole matrix is checked for fidelity and
    uneven per-row iteration counts."""
    cfg = synth.CONFIGS["batching"]
    N, M, J = cfg["N"], cfg["M"], cfg["J"]
    T = c64(synth.make_tm(cfg, seed=0))
    _, d = synth.mask_phases(J, N, seed=0)
    d = c64(d)
    rows = synth.sample_rows(M, 4, seed=0)
    Yg = torch.empty((M, J, N), dtype=torch.float32, device="cuda")
    pits = 100
    with handle(N, M, J, d, init=tmr.TMR_INIT_SPECTRAL, power_iters=pits, clip=2.0, tol=cfg["tol"]) as h:
        tmr.tmr_forward(h, to_dev(T), Yg)
        torch.cuda.synchronize()
        Y_clean = to_np(Yg)
        Y_or = oracle.forward(T[rows].astype(np.complex128), d.astype(np.complex128))
        assert_rows_close(Y_clean[rows], Y_or, 1e-5)
        ph = synth.row_photons(cfg, M, seed=0)
        scale = synth.photon_scale(float(Y_clean.mean()), ph)
        Yn = f32(synth.shot_noise(Y_clean, scale, seed=0))
        To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        st = torch.empty(M, dtype=torch.int32, device="cuda")
        its = torch.empty(M, dtype=torch.int32, device="cuda")
        tmr.tmr_retrieve(h, to_dev(Yn), None, cfg["iters"], To, st, its)
        torch.cuda.synchronize()
        # the same rows at a short budget, for the element-wise comparison
        short = 15
        Ts = torch.empty((len(rows), N), dtype=torch.complex64, device="cuda")
    with handle(N, len(rows), J, d, init=tmr.TMR_INIT_SPECTRAL, power_iters=30, clip=2.0) as h2:
        tmr.tmr_retrieve(h2, to_dev(Yn[rows]), None, short, Ts[:len(rows)])
        torch.cuda.synchronize()
    Tr, _, _, _ = oracle.retrieve_rows(Yn[rows], d.astype(np.complex128), short, init="spectral",
                                       power_iters=30, clip=2.0)
    fid_s = oracle.fidelity_rows(to_np(Ts)[:len(rows)], T[rows])
    fid_o = oracle.fidelity_rows(Tr, T[rows])
    assert np.mean(np.abs(fid_s - fid_o) <= 1e-3) >= 3 / 4, (fid_s, fid_o)
    its_g, st_g = to_np(its), to_np(st)
    assert np.all((st_g == tmr.TMR_ROW_CONVERGED) == (its_g < cfg["iters"]))
    assert its_g.max() > its_g.min()
    fid = oracle.fidelity_rows(to_np(To), T)
    assert np.mean(fid) >= 0.99 and np.mean(fid >= 0.99) >= 0.95


def test_large_length_needs_a_short_history():
    """N = 3500 (L = 8192): with m = 5 the per-row state does not fit in shared
    memory, so the handle offers the forward model but refuses to retrieve;
    with m = 1 it retrieves, step for step with the oracle."""
    N, M, J, iters = 3500, 2, 4, 2
    T, d, Y = problem(N, M, J, seed=35)
    T_init = _perturbed(T, N, 35)
    Tn = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    with handle(N, M, J, d, m=5) as h:
        assert tmr.tmr_schedule(h) == 0
        with pytest.raises(tmr.TMRError) as ei:
            tmr.tmr_retrieve_from(h, to_dev(T_init), to_dev(Y), None, iters, Tn)
        assert ei.value.status == tmr.TMR_ERR_UNSUPPORTED
    with handle(N, M, J, d, m=1) as h:
        assert tmr.tmr_schedule(h) == 1
        tmr.tmr_retrieve_from(h, to_dev(T_init), to_dev(Y), None, iters, Tn)
        torch.cuda.synchronize()
    Tr, _, _, _ = oracle.retrieve_rows(Y, d.astype(np.complex128), iters, m=1, T_init=T_init)
    assert_rows_close(to_np(Tn), Tr, 1e-4 * iters)


# ------------------------------------------------------------ transform plans for 2048 < N <= 2731
@pytest.mark.parametrize("N,J", [(2286, 4), (2600, 4)])
def test_full_bluestein_plan_matches_oracle(N, J):
    """Schedule 32 (Bluestein at L = 8192 over the whole output) against the
    oracle step by step, and against schedule 1 (split outputs at L = 4096):
    the same method through another transform plan."""
    M, iters = 6, 4
    T, d, Y = problem(N, M, J, seed=N + 32)
    rng = np.random.default_rng(N)
    T_init = c64(T + 0.3 * (rng.standard_normal(T.shape) + 1j * rng.standard_normal(T.shape)) / np.sqrt(N))
    out = {}
    for G in (1, 32):
        Tn = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        its = torch.empty(M, dtype=torch.int32, device="cuda")
        with handle(N, M, J, d, schedule=G) as h:
            assert tmr.tmr_schedule(h) == G
            tmr.tmr_retrieve_from(h, to_dev(T_init), to_dev(Y), None, iters, Tn, row_iters=its)
            torch.cuda.synchronize()
        out[G] = (to_np(Tn), to_np(its))
    Tr, _, it_ref, _ = oracle.retrieve_rows(Y, d.astype(np.complex128), iters, T_init=T_init)
    for G in (1, 32):
        assert np.all(out[G][1] == it_ref)
        assert_rows_close(out[G][0], Tr, 1e-4 * iters)


def test_autotuner_times_both_bluestein_plans():
    """At N = 2286 the autotuner has two candidates, the split-output plan
    (schedule 1) and the full-length plan (schedule 32): it times both and
    keeps the faster, which a handle made afterwards finds in the cache."""
    N, M, J = 2286, 16, 4
    _, d, Y = problem(N, M, J, seed=77)
    with handle(N, M, J, d, m=3, schedule=0) as h:  # m = 3: a tuning key no other test uses
        rep = tmr.tmr_autotune_report(h)
        G = tmr.tmr_schedule(h)
        To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        tmr.tmr_retrieve(h, to_dev(Y), None, 5, To)
        torch.cuda.synchronize()
    print("autotuner at N = 2286:", rep, "->", G)
    assert set(rep) == {1, 32}
    assert G == min(rep, key=rep.get)
    with handle(N, M, J, d, m=3, schedule=0) as h2:
        assert tmr.tmr_schedule(h2) == G and tmr.tmr_autotune_report(h2) == {}
