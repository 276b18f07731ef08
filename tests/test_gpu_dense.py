"""The paper's "without FFT" evaluation (opt.dense: Q as an explicit dense
matrix, the products as complex matrix products over the rows) against the
FP64 oracle and against the FFT path, element by element.  Mode 1 is FP32
(bar 1e-5 of the oracle's row maximum, like the FFT path); mode 2 emulates
FP32 on the tensor cores with three BF16 terms per operand (the same bar)."""
import numpy as np
import pytest

import oracle
from helpers import problem, assert_rows_close, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2302_13524_gb300 as tmr  # noqa: E402


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("N,J", [(64, 4), (512, 4), (2048, 4), (256, 3)])
def test_dense_forward_and_gradient_match_oracle(mode, N, J):
    M = 6
    T, d, _ = problem(N, M, J, seed=N + mode)
    _, _, Y = problem(N, M, J, seed=N + 7)
    Y_ref = oracle.forward(T.astype(np.complex128), d.astype(np.complex128))
    loss_ref, G_ref = oracle.loss_grad(T.astype(np.complex128), d.astype(np.complex128), Y.astype(np.float64))
    Yg = torch.empty((M, J, N), dtype=torch.float32, device="cuda")
    loss = torch.empty(M, dtype=torch.float32, device="cuda")
    G = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    with tmr.tmr_create(N, M, J, to_dev(d), None, dict(dense=mode)) as h:
        tmr.tmr_forward(h, to_dev(T), Yg)
        tmr.tmr_grad(h, to_dev(T), to_dev(Y), loss, G)
        torch.cuda.synchronize()
    assert_rows_close(to_np(Yg), Y_ref, 1e-5)
    assert np.max(np.abs(to_np(loss) - loss_ref) / loss_ref) <= 1e-5
    assert_rows_close(to_np(G), G_ref, 1e-5)


def test_dense_amplitude_gradient_matches_oracle():
    N, M, J = 256, 5, 4
    T, d, _ = problem(N, M, J, seed=3)
    _, _, Y = problem(N, M, J, seed=4)
    with oracle.amplitude_cost():
        loss_ref, G_ref = oracle.loss_grad(T.astype(np.complex128), d.astype(np.complex128), Y.astype(np.float64))
    loss = torch.empty(M, dtype=torch.float32, device="cuda")
    G = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    with tmr.tmr_create(N, M, J, to_dev(d), None, dict(dense=1, cost="amplitude")) as h:
        tmr.tmr_grad(h, to_dev(T), to_dev(Y), loss, G)
        torch.cuda.synchronize()
    assert np.max(np.abs(to_np(loss) - loss_ref) / loss_ref) <= 1e-5
    assert_rows_close(to_np(G), G_ref, 1e-5)


def test_dense_and_fft_paths_agree():
    N, M, J = 1024, 64, 4
    T, d, Y = problem(N, M, J, seed=9)
    out = {}
    for dense in (0, 1):
        loss = torch.empty(M, dtype=torch.float32, device="cuda")
        G = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        with tmr.tmr_create(N, M, J, to_dev(d), None, dict(dense=dense)) as h:
            tmr.tmr_grad(h, to_dev(T * 1.1), to_dev(Y), loss, G)
            torch.cuda.synchronize()
        out[dense] = (to_np(loss), to_np(G))
    assert np.max(np.abs(out[1][0] - out[0][0]) / out[0][0]) <= 2e-5
    assert_rows_close(out[1][1], out[0][1], 2e-5)
    with pytest.raises(tmr.TMRError) as ei:
        tmr.tmr_create(N, M, J, to_dev(d), None, dict(dense=3))
    assert ei.value.status == tmr.TMR_ERR_INVALID_ARG


# ------------------------------------------------ Algorithm 1 without FFT
@pytest.mark.parametrize("N,J", [(256, 4), (1024, 3), (64, 8)])
def test_dense_solver_first_step_matches_oracle(N, J):
    """tmr_retrieve with opt.dense runs Algorithm 1 with the FFTs replaced by
    matrix-vector products: one step from a given start equals the oracle's."""
    M = 4
    T, d, Y = problem(N, M, J, seed=11 + N)
    rng = np.random.default_rng(N)
    T_init = (T + 0.3 * (rng.standard_normal(T.shape) + 1j * rng.standard_normal(T.shape)) / np.sqrt(N))
    T_init = np.ascontiguousarray(T_init, dtype=np.complex64)
    Tn = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    with tmr.tmr_create(N, M, J, to_dev(d), None, dict(dense=1)) as h:
        assert tmr.tmr_schedule(h) == 1
        tmr.tmr_retrieve_from(h, to_dev(T_init), to_dev(Y), None, 1, Tn)
        torch.cuda.synchronize()
    for r in range(M):
        ref = oracle.lbfgs_step(Y[r].astype(np.float64), d.astype(np.complex128), T_init[r].astype(np.complex128))
        assert_rows_close(to_np(Tn)[r:r + 1], ref["t"][None], 1e-5)


def test_dense_solver_retrieval_matches_the_fft_solver():
    """Whole retrievals (Lanczos start, 60 L-BFGS iterations) with and without
    FFT end at the same per-row fidelities (the same algorithm, other rounding)."""
    N, M, J = 512, 48, 4
    T, d, Y = problem(N, M, J, seed=21)
    fids = {}
    for dense in (0, 1):
        To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        with tmr.tmr_create(N, M, J, to_dev(d), None,
                            dict(dense=dense, init="spectral", power_iters=16, lanczos=1, schedule=1)) as h:
            tmr.tmr_retrieve(h, to_dev(Y), None, 60, To)
            tmr.tmr_sync(h, 60.0)
        fids[dense] = oracle.fidelity_rows(to_np(To), T)
    assert np.sum(np.abs(fids[1] - fids[0]) > 1e-3) <= 1
    assert abs(np.sum(fids[1] < 0.99) - np.sum(fids[0] < 0.99)) <= 1


def test_dense_solver_refuses_the_fit_and_other_shapes():
    N, M, J = 64, 128, 4
    _, d, Y = problem(N, M, J, seed=2)
    with tmr.tmr_create(N, M, J, to_dev(d), dict(ny=16, nx=8, n_defocus=8), dict(dense=1)) as h:
        To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        yd = torch.zeros((8, M), dtype=torch.float32, device="cuda")
        with pytest.raises(tmr.TMRError) as ei:
            tmr.tmr_retrieve(h, to_dev(Y), yd, 5, To)
        assert ei.value.status == tmr.TMR_ERR_UNSUPPORTED
    with pytest.raises(tmr.TMRError) as ei:  # not a power of two
        tmr.tmr_create(1000, 4, J, to_dev(np.ones((J, 1000), np.complex64)), None, dict(dense=1))
    assert ei.value.status == tmr.TMR_ERR_UNSUPPORTED
