"""The allocation-free entry point, for callers that may not call cudaMalloc
(for example under an allocator that owns all device memory): it must give
what tmr_retrieve gives on the same inputs, on two calls in a row, through the
C ABI.  Kept in its own file, collected after every other test."""
import numpy as np
import pytest

from helpers import problem, rel_l2_rows, to_dev, to_np

torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_static_scratch_retrieve_matches_handle_retrieve():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_13524_gb300 as tmr
    N, M, J, iters = 256, 37, 4, 12
    T, d, Y = problem(N, M, J, seed=21)
    opt = dict(init="spectral", power_iters=30, clip=2.0, seed=3)
    dg, yg = to_dev(d), to_dev(Y)
    T_ref = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    st_ref = torch.empty(M, dtype=torch.int32, device="cuda")
    with tmr.tmr_create(N, M, J, dg, None, opt) as h:
        tmr.tmr_retrieve(h, yg, None, iters, T_ref, st_ref)
        torch.cuda.synchronize()
    for call in range(2):
        T_out = torch.full((M, N), float("nan"), dtype=torch.complex64, device="cuda")
        st = torch.full((M,), -1, dtype=torch.int32, device="cuda")
        tmr.tmr_retrieve_rows_static(N, M, J, dg, yg, iters, opt, T_out, st)
        torch.cuda.synchronize()
        assert rel_l2_rows(to_np(T_out), to_np(T_ref)) <= 1e-5, call
        np.testing.assert_array_equal(to_np(st), to_np(st_ref))


@pytest.mark.gpu
def test_static_scratch_rejects_sizes_beyond_its_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_13524_gb300 as tmr
    d = torch.ones((4, 8192), dtype=torch.complex64, device="cuda")
    y = torch.zeros((1, 4, 8192), dtype=torch.float32, device="cuda")
    T = torch.empty((1, 8192), dtype=torch.complex64, device="cuda")
    with pytest.raises(tmr.TMRError) as ei:
        tmr.tmr_retrieve_rows_static(8192, 1, 4, d, y, 1, None, T)
    assert ei.value.status == tmr.TMR_ERR_UNSUPPORTED
    yh = np.zeros((1, 4, 256), np.float32)
    with pytest.raises(tmr.TMRError) as ei:
        tmr.tmr_retrieve_rows_static(256, 1, 4, d[:, :256].contiguous(), yh, 1, None, T[:, :256].contiguous())
    assert ei.value.status == tmr.TMR_ERR_INVALID_ARG
