"""GPU parity of the Lanczos spectral start (opt.lanczos): the start vector of
every solver layout against the FP64 oracle's Lanczos start, the invariant-
subspace stop, and the retrieval it feeds.  Bars: 2e-4 per entry relative to
the row's largest (FP32 Krylov vectors; the Ritz vector's sensitivity is
rounding over the gap of the top Ritz values), the mixed layouts at 2e-3
(FP16 intensities)."""
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


def start(N, M, J, d, Y, k, **opt):
    T0 = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    o = dict(init="spectral", seed=42, power_iters=k, clip=2.0, lanczos=1)
    o.update(opt)
    with tmr.tmr_create(N, M, J, to_dev(d), None, o) as h:
        tmr.tmr_retrieve(h, to_dev(Y), None, 0, T0)
        tmr.tmr_sync(h, 60.0)
        sched = tmr.tmr_schedule(h)
    return to_np(T0), sched


@pytest.mark.parametrize("N,J,G", [(512, 4, 16), (1024, 4, 16), (2048, 4, 16), (512, 3, 16),
                                   (256, 4, 1), (256, 4, 2), (256, 4, 4), (2048, 4, 1), (4096, 4, 1),
                                   (64, 8, 2)])
@pytest.mark.parametrize("k", [1, 5, 16])
def test_lanczos_start_matches_oracle(N, J, G, k):
    M = 5
    _, d, Y = problem(N, M, J, seed=N + J + G)
    ref = oracle.init(Y, d.astype(np.complex128), "lanczos", seed=42, power_iters=k, clip=2.0)
    T0, sched = start(N, M, J, d, Y, k, schedule=G)
    assert sched == G
    assert_rows_close(T0, ref, 2e-4)


@pytest.mark.parametrize("N,G", [(2286, 1), (2600, 32), (1000, 1)])
def test_lanczos_start_bluestein_layouts(N, G):
    M, J, k = 4, 4, 12
    _, d, Y = problem(N, M, J, seed=N)
    ref = oracle.init(Y, d.astype(np.complex128), "lanczos", seed=42, power_iters=k, clip=2.0)
    T0, sched = start(N, M, J, d, Y, k, schedule=G)
    assert sched == G
    assert_rows_close(T0, ref, 2e-4)


def test_lanczos_start_2d_probing():
    N, n1, M, J, k = 512, 8, 4, 4, 10
    T = c64(synth.tm_iid(M, N, 3))
    _, d = synth.mask_phases(J, N, 3)
    d = c64(d)
    with oracle.probe_2d(n1, N):
        Y = f32(oracle.forward(T.astype(np.complex128), d.astype(np.complex128)))
        ref = oracle.init(Y, d.astype(np.complex128), "lanczos", seed=42, power_iters=k, clip=2.0)
    T0, _ = start(N, M, J, d, Y, k, probe_n1=n1)
    assert_rows_close(T0, ref, 2e-4)


def test_lanczos_start_mixed_precision():
    N, M, J, k = 4096, 3, 4, 12
    _, d, Y = problem(N, M, J, seed=77)
    ref = oracle.init(Y, d.astype(np.complex128), "lanczos", seed=42, power_iters=k, clip=2.0)
    T0, _ = start(N, M, J, d, Y, k, precision="mixed")
    assert_rows_close(T0, ref, 2e-3)


def test_lanczos_stops_on_an_invariant_subspace():
    """Constant intensities: A = I, beta_0 = 0, and the start is the random start."""
    N, M, J = 512, 3, 4
    _, d, _ = problem(N, M, J, seed=1)
    Y = np.full((M, J, N), 2.0, np.float32)
    ref = oracle.init(Y, d.astype(np.complex128), "random", seed=42)
    for G in (16, 1):
        T0, _ = start(N, M, J, d, Y, 8, schedule=G)
        assert_rows_close(T0, ref, 2e-5)


def test_lanczos_start_retrieves_mode_model_rows():
    """16 Lanczos steps and 20 L-BFGS iterations reach the fidelity of the
    oracle's run from its own Lanczos start on noisy mode-model rows (the
    workload's statistics: 12 rows of an 8192 x 2048 mode-model TM, R = 1100)."""
    N, J, R, M = 2048, 4, 1100, 12
    rows = synth.sample_rows(8192, M, seed=5)
    T = c64(synth.tm_modes(8192, N, R, seed=5)[rows])
    _, d = synth.mask_phases(J, N, seed=5)
    d = c64(d)
    Yc = oracle.forward(T.astype(np.complex128), d.astype(np.complex128))
    Y = f32(synth.shot_noise(Yc, synth.photon_scale(Yc.mean(), 1e4), seed=5))
    To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    with tmr.tmr_create(N, M, J, to_dev(d), None,
                        dict(init="spectral", power_iters=16, lanczos=1, clip=2.0)) as h:
        tmr.tmr_retrieve(h, to_dev(Y), None, 20, To)
        tmr.tmr_sync(h, 60.0)
    fg = oracle.fidelity_rows(to_np(To), T)
    T_o = oracle.retrieve_rows(Y, d.astype(np.complex128), 20, init="lanczos", power_iters=16, clip=2.0)[0]
    fo = oracle.fidelity_rows(T_o, T)
    assert fo.mean() > 0.99 and fg.mean() > 0.99
    assert np.sum(np.abs(fg - fo) > 1e-3) <= max(1, int(0.01 * M))


def test_lanczos_options_are_checked():
    N, M, J = 512, 4, 4
    _, d, Y = problem(N, M, J, seed=2)
    for bad in (dict(lanczos=2), dict(lanczos=1, power_iters=17), dict(lanczos=-1)):
        with pytest.raises(tmr.TMRError) as ei:
            tmr.tmr_create(N, M, J, to_dev(d), None, bad)
        assert ei.value.status == tmr.TMR_ERR_INVALID_ARG
    T0 = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    o = tmr.tmr_default_options(lanczos=1, power_iters=8)
    with pytest.raises(tmr.TMRError) as ei:
        tmr.tmr_retrieve_rows_static(N, M, J, to_dev(d), to_dev(Y), 5, o, T0)
    assert ei.value.status == tmr.TMR_ERR_UNSUPPORTED
