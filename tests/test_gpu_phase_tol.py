"""GPU phase-offset fit with a loss-floor stop (opt.phase_tol) against the
FP64 oracle's fit with the same rule, on noisy defocus images (so that the
loss levels off above zero): the same number of accepted steps (within one:
the FP32 loss decides the comparison near the bar) and the same offsets."""
import numpy as np
import pytest

import oracle
import synth
from helpers import c64, f32, problem, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2302_13524_gb300 as tmr  # noqa: E402


@pytest.mark.parametrize("tol", [0.03, 1e-3])
def test_phase_fit_stops_at_the_loss_floor_like_the_oracle(tol):
    ny, nx, Nd, N, J = 16, 8, 24, 64, 4
    M = ny * nx
    grid = (ny, nx)
    T, d, _ = problem(N, M, J, seed=41)
    Yd = oracle.defocus_forward(oracle.defocus_fields(T.astype(np.complex128), d.astype(np.complex128), Nd), grid)
    rng = np.random.default_rng(42)
    Yd = f32(Yd * (1 + 0.02 * rng.standard_normal(Yd.shape)))
    T_est = c64(np.exp(-1j * rng.uniform(-np.pi, np.pi, M))[:, None] * T)
    C = oracle.defocus_fields(T_est.astype(np.complex128), d.astype(np.complex128), Nd)
    wts = np.sum(np.abs(T_est.astype(np.complex128)) ** 2, axis=1)
    phi_o, done_o, loss_o = oracle.phase_fit(C, Yd, grid, iters=200, weights=wts, tol=tol)
    assert done_o < 200
    phi = torch.empty(M, dtype=torch.float64, device="cuda")
    with tmr.tmr_create(N, M, J, to_dev(d), dict(ny=ny, nx=nx, n_defocus=Nd, coef=0.05),
                        dict(phase_iters=200, phase_tol=tol)) as h:
        tmr.tmr_defocus_fit(h, to_dev(T_est), to_dev(Yd), phi, None)
        tmr.tmr_sync(h, 60.0)
        loss, done = tmr.tmr_phase_fit_report(h)
    assert abs(done - done_o) <= 1, (done, done_o)
    assert abs(loss - loss_o) <= 0.05 * loss_o
    if done == done_o:
        err = np.angle(np.exp(1j * (to_np(phi) - phi_o)))
        assert np.max(np.abs(err)) <= 1e-2


def test_phase_tol_is_checked():
    N, M, J = 64, 128, 4
    _, d, _ = problem(N, M, J, seed=1)
    for bad in (-1e-3, float("nan"), float("inf")):
        with pytest.raises(tmr.TMRError) as ei:
            tmr.tmr_create(N, M, J, to_dev(d), dict(ny=16, nx=8, n_defocus=8), dict(phase_tol=bad))
        assert ei.value.status == tmr.TMR_ERR_INVALID_ARG
