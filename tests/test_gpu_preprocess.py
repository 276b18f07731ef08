"""Camera preprocessing through the C ABI (tmr_preprocess, tmr_half_sample)
against the numpy oracle: rows, mask, energies and count bit for bit on
uint16 frames, rows bit for bit and energies to FP64 rounding on float32
frames, the degenerate cases, argument errors, the full camera shape of the
plain workload, and camera frames -> retrieval end to end."""
import numpy as np
import pytest

import oracle
import synth
from helpers import c64, f32, rel_l2_rows, to_dev, to_np
from oracle import preprocess as pp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2302_13524_gb300 as tmr  # noqa: E402


def frames_dev(fr):
    """Device copy of a frame stack; uint16 travels as int16 with the same bits."""
    if fr.dtype == np.uint16:
        return to_dev(fr.view(np.int16))
    return to_dev(fr)


def run(fr, offset, frac):
    out = tmr.preprocess(frames_dev(fr), offset=offset, energy_frac=frac)
    torch.cuda.synchronize()
    return to_np(out["y"]), to_np(out["mask"]).astype(bool), to_np(out["energy"]), int(out["n_inside"].item())


@pytest.mark.parametrize("K,H,W,offset,frac", [(96, 37, 50, 0, 0.999), (300, 20, 21, 1, 0.9),
                                               (33, 64, 64, 0, 1.0), (1, 3, 3, 1, 0.5),
                                               (513, 9, 130, 1, 0.999)])
def test_uint16_frames_match_oracle_exactly(K, H, W, offset, frac):
    fr = synth.camera_frames(K, H, W, seed=K + H)
    y, mask, E, n = run(fr, offset, frac)
    y_o, mask_o, E_o = pp.camera_rows(fr, offset, frac)
    np.testing.assert_array_equal(mask, mask_o)
    np.testing.assert_array_equal(E, E_o.astype(np.float64))
    assert n == int(mask_o.sum())
    assert np.array_equal(y, y_o)


@pytest.mark.parametrize("offset", [0, 1])
def test_float32_frames_match_oracle(offset):
    K, H, W = 200, 30, 41
    fr = (synth.camera_frames(K, H, W, seed=7, dtype=np.float32) * np.float32(0.37)).astype(np.float32)
    y, mask, E, n = run(fr, offset, 0.999)
    y_o, mask_o, E_o = pp.camera_rows(fr, offset, 0.999)
    assert np.array_equal(y, y_o)
    np.testing.assert_allclose(E, E_o, rtol=1e-13, atol=0)
    np.testing.assert_array_equal(mask, mask_o)
    assert n == int(mask_o.sum())
    # a fixed summation order: a second call agrees bit for bit
    y2, mask2, E2, n2 = run(fr, offset, 0.999)
    assert np.array_equal(E, E2) and np.array_equal(mask, mask2) and n == n2


@pytest.mark.parametrize("dtype", [np.uint16, np.float32])
def test_dark_frames_give_an_empty_mask(dtype):
    fr = np.zeros((40, 10, 12), dtype=dtype)
    y, mask, E, n = run(fr, 0, 0.999)
    assert n == 0 and not mask.any() and not y.any() and not E.any()


@pytest.mark.parametrize("bad", [np.nan, np.inf, -1e6])
def test_invalid_float_frames_are_flagged(bad):
    fr = synth.camera_frames(20, 8, 8, seed=3, dtype=np.float32)
    fr[5, 2, 2] = bad
    y, mask, E, n = run(fr, 0, 0.999)
    assert n == -1 and not mask.any() and not y.any()


def test_argument_errors():
    fr = frames_dev(synth.camera_frames(4, 8, 8, seed=1))
    y = torch.empty((16, 4), dtype=torch.float32, device="cuda")
    wb = tmr.tmr_preprocess_workspace_bytes(4, 8, 8, 0)
    ws = torch.empty((wb,), dtype=torch.uint8, device="cuda")
    calls = [
        lambda: tmr.tmr_preprocess(fr, 4, 8, 8, 0, 0.0, y, workspace=ws, workspace_bytes=wb),
        lambda: tmr.tmr_preprocess(fr, 4, 8, 8, 0, 1.5, y, workspace=ws, workspace_bytes=wb),
        lambda: tmr.tmr_preprocess(fr, 4, 8, 8, 0, float("nan"), y, workspace=ws, workspace_bytes=wb),
        lambda: tmr.tmr_preprocess(fr, 4, 8, 8, 0, 0.9, y, workspace=ws, workspace_bytes=wb - 1),
        lambda: tmr.tmr_preprocess(fr, 4, 8, 8, 0, 0.9, y, workspace=None, workspace_bytes=wb),
        lambda: tmr.tmr_preprocess(fr.cpu(), 4, 8, 8, 0, 0.9, y, workspace=ws, workspace_bytes=wb),
        lambda: tmr.tmr_preprocess(fr, 4, 8, 8, 0, 0.9, y.cpu(), workspace=ws, workspace_bytes=wb),
    ]
    for call in calls:
        with pytest.raises(tmr.TMRError) as e:
            call()
        assert e.value.status == tmr.TMR_ERR_INVALID_ARG
    # offset outside {0, 1}, and a half grid without pixels (H = 1, offset 1)
    for K, H, W, off in [(4, 8, 8, 2), (4, 1, 8, 1), (0, 8, 8, 0)]:
        assert tmr.tmr_preprocess_workspace_bytes(K, H, W, off) == 0
    one = torch.zeros((4, 1, 8), dtype=torch.int16, device="cuda")
    with pytest.raises(tmr.TMRError):
        tmr.tmr_preprocess(one, 4, 1, 8, 1, 0.9, torch.empty((0, 4), device="cuda"), workspace=ws,
                           workspace_bytes=wb)
    with pytest.raises(TypeError):
        tmr.preprocess(fr.to(torch.int32))


@pytest.mark.parametrize("dtype,offset", [(np.uint16, 0), (np.float32, 1)])
def test_half_sample_matches_oracle(dtype, offset):
    n, H, W = 50, 33, 26
    fr = synth.camera_frames(n, H, W, seed=11, dtype=dtype)
    ny, nx = pp.half_grid(H, W, offset)
    out = torch.empty((n, ny * nx), dtype=torch.float32, device="cuda")
    tmr.tmr_half_sample(frames_dev(fr), n, H, W, offset, out)
    torch.cuda.synchronize()
    want = pp.half_sample(fr, offset).reshape(n, -1).astype(np.float32)
    assert np.array_equal(to_np(out), want)


def test_camera_shape_of_the_plain_workload():
    """8192 uint16 frames of 256 x 128 pixels -> 8192 rows of 8192 intensities
    on the 128 x 64 half grid: every output compared with the oracle."""
    K, H, W = 8192, 256, 128
    fr = synth.camera_frames(K, H, W, seed=5)
    y, mask, E, n = run(fr, 0, 0.999)
    y_o, mask_o, E_o = pp.camera_rows(fr, 0, 0.999)
    np.testing.assert_array_equal(mask, mask_o)
    np.testing.assert_array_equal(E, E_o.astype(np.float64))
    assert n == int(mask_o.sum()) and 0 < n < K
    assert np.array_equal(y, y_o)


def test_camera_frames_to_retrieval():
    """Camera frames whose kept pixels carry a TM's intensities (rows outside
    a fiber disc dark) and whose other pixels carry noise the preprocessing
    must drop: the rows equal the intensities, the mask is the disc, rows
    inside are retrieved and rows outside come back zero without iterating."""
    N, J, ny, nx = 256, 4, 12, 10
    M, K = ny * nx, J * N
    disc = synth.fiber_disc(ny, nx, 0.4)
    T = c64(synth.tm_iid(M, N, seed=21) * disc[:, None])
    _, d = synth.mask_phases(J, N, seed=21)
    d = c64(d)
    Y = f32(oracle.forward(T.astype(np.complex128), d.astype(np.complex128))).reshape(M, K)
    rng = np.random.default_rng(4)
    fr = rng.uniform(0, 5, size=(K, 2 * ny, 2 * nx)).astype(np.float32)
    fr[:, 0::2, 0::2] = Y.T.reshape(K, ny, nx)
    out = tmr.preprocess(to_dev(fr), offset=0, energy_frac=1.0)
    torch.cuda.synchronize()
    assert np.array_equal(to_np(out["y"]), Y)
    assert np.array_equal(to_np(out["mask"]).astype(bool), disc)
    with tmr.Retriever(to_dev(d), M, init=tmr.TMR_INIT_SPECTRAL, power_iters=50) as r:
        res = r.retrieve(out["y"].view(M, J, N), None, 100)
        torch.cuda.synchronize()
    Tr, status = to_np(res["T"]), to_np(res["status"])
    fid = oracle.fidelity_rows(Tr[disc], T[disc])
    assert np.median(fid) > 0.999
    assert (status[~disc] == tmr.TMR_ROW_ZERO).all() and not Tr[~disc].any()
