"""The allocation-free entry point, for callers that may not call cudaMalloc
(for example code running under an allocator that owns all device memory, or
a loop that cannot take the device-wide synchronisation a first cudaMalloc
may cause): it must give what tmr_retrieve gives on the same inputs, on two
calls in a row, through the C ABI.  Kept in its own file, collected after
every other test."""
import numpy as np
import pytest

from helpers import max_rel_elem_rows, problem, rel_l2_rows, to_dev, to_np

torch = pytest.importorskip("torch")


def _compare_with_handle(N, M, J, iters, seed, opt):
    import paper_2302_13524_gb300 as tmr
    T, d, Y = problem(N, M, J, seed=seed)
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
        # the static twiddle table may differ from the handle's by 1 ulp of FP32
        assert rel_l2_rows(to_np(T_out), to_np(T_ref)) <= 1e-5, call
        assert max_rel_elem_rows(to_np(T_out), to_np(T_ref)) <= 1e-5, call
        np.testing.assert_array_equal(to_np(st), to_np(st_ref))


@pytest.mark.gpu
def test_static_scratch_retrieve_matches_handle_retrieve():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _compare_with_handle(256, 37, 4, 12, 21, dict(init="spectral", power_iters=30, clip=2.0, seed=3))


@pytest.mark.gpu
def test_static_scratch_largest_table_and_footprint():
    """N = 4096 with J = 8 and m = 6: the largest twiddle table the static
    array holds and the largest per-row footprint the entry point accepts."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _compare_with_handle(4096, 5, 8, 6, 22, dict(init="spectral", power_iters=10, clip=2.0, seed=5, m=6))


@pytest.mark.gpu
def test_static_scratch_no_rows_and_null_arrays():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_13524_gb300 as tmr
    d = torch.ones((4, 256), dtype=torch.complex64, device="cuda")
    tmr.tmr_retrieve_rows_static(256, 0, 4, d, None, 5, None, None)
    torch.cuda.synchronize()


@pytest.mark.gpu
def test_static_scratch_rejects_unsupported_sizes_and_options():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2302_13524_gb300 as tmr
    d = torch.ones((4, 8192), dtype=torch.complex64, device="cuda")
    y = torch.zeros((1, 4, 8192), dtype=torch.float32, device="cuda")
    T = torch.empty((1, 8192), dtype=torch.complex64, device="cuda")
    with pytest.raises(tmr.TMRError) as ei:  # beyond the supported transform lengths
        tmr.tmr_retrieve_rows_static(8192, 1, 4, d, y, 1, None, T)
    assert ei.value.status == tmr.TMR_ERR_UNSUPPORTED
    d2, y2, T2 = d[:, :256].contiguous(), y[:, :, :256].contiguous(), T[:, :256].contiguous()
    with pytest.raises(tmr.TMRError) as ei:  # mixed precision is not offered here
        tmr.tmr_retrieve_rows_static(256, 1, 4, d2, y2, 1, dict(precision="mixed"), T2)
    assert ei.value.status == tmr.TMR_ERR_UNSUPPORTED
    yh = np.zeros((1, 4, 256), np.float32)
    with pytest.raises(tmr.TMRError) as ei:  # host memory
        tmr.tmr_retrieve_rows_static(256, 1, 4, d2, yh, 1, None, T2)
    assert ei.value.status == tmr.TMR_ERR_INVALID_ARG
