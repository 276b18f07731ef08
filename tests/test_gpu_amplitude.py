"""GPU parity of the amplitude cost (opt.cost = TMR_COST_AMPLITUDE: the
Discussion's f = sum (sqrt(y) - |Qt|)^2 for Poisson noise) against the FP64
oracle under oracle.amplitude_cost(): loss and gradient element by element
(1e-5), the first L-BFGS step with the bracketing-Newton line search (1e-5;
the GPU stops its Newton steps at 1e-6 of the step, the oracle at 1e-13), a
few steps, and whole retrievals in every solver layout."""
import numpy as np
import pytest

import oracle
import synth
from helpers import c64, f32, problem, assert_rows_close, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2302_13524_gb300 as tmr  # noqa: E402

AMP = dict(cost="amplitude")


@pytest.mark.parametrize("N", [64, 512, 2048, 4096, 2286, 1000])
def test_amplitude_loss_and_gradient(N):
    M, J = 5, 4
    T, d, _ = problem(N, M, J, seed=N + 1)
    _, _, Y = problem(N, M, J, seed=N + 2)  # intensities of another TM: large residuals
    with oracle.amplitude_cost():
        loss_ref, G_ref = oracle.loss_grad(T.astype(np.complex128), d.astype(np.complex128), Y.astype(np.float64))
    loss = torch.empty(M, dtype=torch.float32, device="cuda")
    G = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    with tmr.tmr_create(N, M, J, to_dev(d), None, AMP) as h:
        tmr.tmr_grad(h, to_dev(T), to_dev(Y), loss, G)
        torch.cuda.synchronize()
    assert np.max(np.abs(to_np(loss) - loss_ref) / loss_ref) <= 1e-5
    assert_rows_close(to_np(G), G_ref, 1e-5)


@pytest.mark.parametrize("N,J,G", [(512, 4, 16), (2048, 4, 16), (256, 4, 1), (256, 4, 2), (2286, 4, 1),
                                   (512, 3, 16)])
def test_amplitude_first_step(N, J, G):
    M = 4
    T, d, Y = problem(N, M, J, seed=7 + N)
    rng = np.random.default_rng(N)
    T_init = c64(T + 0.4 * (rng.standard_normal(T.shape) + 1j * rng.standard_normal(T.shape)) / np.sqrt(N))
    Tn = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    loss = torch.empty(M, dtype=torch.float32, device="cuda")
    with tmr.tmr_create(N, M, J, to_dev(d), None, dict(AMP, schedule=G)) as h:
        assert tmr.tmr_schedule(h) == G
        tmr.tmr_retrieve_from(h, to_dev(T_init), to_dev(Y), None, 1, Tn, row_loss=loss)
        torch.cuda.synchronize()
    with oracle.amplitude_cost():
        for r in range(M):
            ref = oracle.lbfgs_step(Y[r].astype(np.float64), d.astype(np.complex128),
                                    T_init[r].astype(np.complex128))
            assert ref["alpha"] > 0
            assert_rows_close(to_np(Tn)[r:r + 1], ref["t"][None], 1e-5)
            assert abs(to_np(loss)[r] - ref["loss"]) <= 1e-4 * ref["loss"] + 1e-7 * np.sum(Y[r])


@pytest.mark.parametrize("iters", [3, 8])
def test_amplitude_few_steps(iters):
    N, M, J = 256, 4, 4
    T, d, Y = problem(N, M, J, seed=31)
    rng = np.random.default_rng(32)
    T_init = c64(T + 0.3 * (rng.standard_normal(T.shape) + 1j * rng.standard_normal(T.shape)) / np.sqrt(N))
    Tn = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    its = torch.empty(M, dtype=torch.int32, device="cuda")
    with tmr.tmr_create(N, M, J, to_dev(d), None, AMP) as h:
        tmr.tmr_retrieve_from(h, to_dev(T_init), to_dev(Y), None, iters, Tn, row_iters=its)
        torch.cuda.synchronize()
    with oracle.amplitude_cost():
        T_o, _, it_o, _ = oracle.retrieve_rows(Y, d.astype(np.complex128), iters, T_init=T_init)
    assert np.array_equal(to_np(its), it_o)
    assert_rows_close(to_np(Tn), T_o, 1e-4 * iters)


@pytest.mark.parametrize("N,G", [(512, 16), (512, 1), (2286, 1), (1024, 16)])
def test_amplitude_retrieval_matches_oracle_fidelity(N, G):
    """Noiseless rows from the spectral start: each row's final fidelity within
    1e-3 of the oracle's, at most 1 % of the rows (at least one) off."""
    M, J = 32, 4
    T, d, Y = problem(N, M, J, seed=3 * N + G)
    To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    opt = dict(AMP, schedule=G, init="spectral", power_iters=100, clip=2.0)
    with tmr.tmr_create(N, M, J, to_dev(d), None, opt) as h:
        tmr.tmr_retrieve(h, to_dev(Y), None, 60, To)
        tmr.tmr_sync(h, 60.0)
    with oracle.amplitude_cost():
        T_o = oracle.retrieve_rows(Y, d.astype(np.complex128), 60, init="spectral", power_iters=100, clip=2.0)[0]
    fg, fo = oracle.fidelity_rows(to_np(To), T), oracle.fidelity_rows(T_o, T)
    assert np.sum(np.abs(fg - fo) > 1e-3) <= max(1, int(0.01 * M))
    assert abs(np.sum(fg < 0.99) - np.sum(fo < 0.99)) <= max(1, int(0.01 * M))


def test_amplitude_cost_on_poisson_rows():
    """Poisson rows of the plain workload's fiber model (48 rows of an
    8192 x 2048 mode-model TM, 1e4 photons): the amplitude cost reaches mean
    fidelity 0.99 from the Lanczos start as the intensity cost does."""
    N, J, R, M = 2048, 4, 1100, 48
    rows = synth.sample_rows(8192, M, seed=9)
    T = c64(synth.tm_modes(8192, N, R, seed=9)[rows])
    _, d = synth.mask_phases(J, N, seed=9)
    d = c64(d)
    Yc = oracle.forward(T.astype(np.complex128), d.astype(np.complex128))
    Y = f32(synth.shot_noise(Yc, synth.photon_scale(Yc.mean(), 1e4), seed=9))
    out = {}
    for cost in ("intensity", "amplitude"):
        To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        with tmr.tmr_create(N, M, J, to_dev(d), None,
                            dict(cost=cost, init="spectral", power_iters=16, lanczos=1, clip=2.0)) as h:
            tmr.tmr_retrieve(h, to_dev(Y), None, 40, To)
            tmr.tmr_sync(h, 60.0)
        out[cost] = oracle.fidelity_rows(to_np(To), T)
    assert out["intensity"].mean() > 0.99 and out["amplitude"].mean() > 0.99, {k: v.mean() for k, v in out.items()}


def test_amplitude_option_checks_and_static_entry():
    N, M, J = 512, 6, 4
    T, d, Y = problem(N, M, J, seed=4)
    with pytest.raises(tmr.TMRError) as ei:
        tmr.tmr_create(N, M, J, to_dev(d), None, dict(cost=2))
    assert ei.value.status == tmr.TMR_ERR_INVALID_ARG
    # the allocation-free entry runs the same cost
    T1 = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    T2 = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    o = dict(AMP, init="spectral", power_iters=50, schedule=1)
    tmr.tmr_retrieve_rows_static(N, M, J, to_dev(d), to_dev(Y), 20, o, T1)
    with tmr.tmr_create(N, M, J, to_dev(d), None, o) as h:
        tmr.tmr_retrieve(h, to_dev(Y), None, 20, T2)
        torch.cuda.synchronize()
    assert_rows_close(to_np(T1), to_np(T2), 1e-5)
