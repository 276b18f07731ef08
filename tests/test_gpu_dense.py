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
@pytest.mark.parametrize("N,J", [(64, 4), (512, 4), (2048, 4), (1000, 3)])
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


def test_dense_and_fft_paths_agree_and_retrieve_is_refused():
    N, M, J = 1024, 64, 4
    T, d, Y = problem(N, M, J, seed=9)
    out = {}
    for dense in (0, 1):
        loss = torch.empty(M, dtype=torch.float32, device="cuda")
        G = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        with tmr.tmr_create(N, M, J, to_dev(d), None, dict(dense=dense)) as h:
            tmr.tmr_grad(h, to_dev(T * 1.1), to_dev(Y), loss, G)
            torch.cuda.synchronize()
            if dense:
                To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
                with pytest.raises(tmr.TMRError) as ei:
                    tmr.tmr_retrieve(h, to_dev(Y), None, 5, To)
                assert ei.value.status == tmr.TMR_ERR_UNSUPPORTED
        out[dense] = (to_np(loss), to_np(G))
    assert np.max(np.abs(out[1][0] - out[0][0]) / out[0][0]) <= 2e-5
    assert_rows_close(out[1][1], out[0][1], 2e-5)
    with pytest.raises(tmr.TMRError) as ei:
        tmr.tmr_create(N, M, J, to_dev(d), None, dict(dense=3))
    assert ei.value.status == tmr.TMR_ERR_INVALID_ARG
