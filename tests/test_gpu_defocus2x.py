"""GPU parity of the paper's defocus model (Sec. 2.3, Eq. angularspectrum,
Eq. forwarddefocusImage, Eq. optphase): separate incident fields, the
angular-spectrum kernel with its NA pupil, 2x zero padding of the spectrum.
libtmr (FP32 transforms, FP64 fit) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from oracle import defocus2x as d2
from helpers import c64, f32, problem, assert_rows_close, to_dev, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2302_13524_gb300 as tmr  # noqa: E402

GEOM = dict(wavelength=0.532, na=0.22, z_d=20.0, pixel=0.9)


def incident(Nd, N, seed):
    rng = np.random.default_rng(seed)
    return c64(np.exp(1j * rng.uniform(0, 2 * np.pi, (Nd, N))))


def dop(ny, nx, inc, **geom):
    g = dict(GEOM, **geom)
    return dict(kind=tmr.DEFOCUS_ANGULAR_2X, ny=ny, nx=nx, n_defocus=inc.shape[0], incident=to_dev(inc), **g)


@pytest.mark.parametrize("grid,Nd,N", [((8, 8), 5, 64), ((16, 8), 37, 128), ((64, 32), 3, 256), ((128, 64), 2, 64)])
def test_forward_images_match_oracle(grid, Nd, N):
    ny, nx = grid
    M, J = ny * nx, 4
    T, d, _ = problem(N, M, J, seed=ny + nx)
    inc = incident(Nd, N, seed=Nd)
    h = d2.transfer(ny, nx, **GEOM)
    I_ref = d2.forward(d2.fields(T.astype(np.complex128), inc.astype(np.complex128)), h)
    out = torch.empty((Nd, 4 * M), dtype=torch.float32, device="cuda")
    with tmr.tmr_create(N, M, J, to_dev(d), dop(ny, nx, inc)) as hd:
        tmr.tmr_defocus_forward(hd, to_dev(T), out)
        torch.cuda.synchronize()
    assert_rows_close(to_np(out), I_ref, 1e-5)


def test_given_kernel_replaces_the_computed_one():
    ny, nx, Nd, N, J = 16, 16, 4, 64, 4
    M = ny * nx
    T, d, _ = problem(N, M, J, seed=5)
    inc = incident(Nd, N, seed=6)
    rng = np.random.default_rng(7)
    H = np.exp(1j * rng.uniform(0, 2 * np.pi, (ny, nx))) * (rng.uniform(size=(ny, nx)) > 0.3)
    I_ref = d2.forward(d2.fields(T.astype(np.complex128), inc.astype(np.complex128)), H)
    out = torch.empty((Nd, 4 * M), dtype=torch.float32, device="cuda")
    op = dop(ny, nx, inc)
    op["H"] = to_dev(c64(H))
    with tmr.tmr_create(N, M, J, to_dev(d), op) as hd:
        tmr.tmr_defocus_forward(hd, to_dev(T), out)
        torch.cuda.synchronize()
    assert_rows_close(to_np(out), I_ref, 1e-5)


@pytest.mark.parametrize("grid,Nd", [((8, 8), 12), ((16, 16), 40), ((32, 16), 48)])
def test_phase_fit_recovers_planted_offsets(grid, Nd):
    """T_est = diag(e^{-i phi*}) T: the fit returns phi* up to a constant; both
    fits end at the planted offsets (their L-BFGS paths differ in rounding)."""
    ny, nx = grid
    M, N, J = ny * nx, 64, 4
    T, d, _ = problem(N, M, J, seed=ny * 3 + nx)
    inc = incident(Nd, N, seed=ny)
    h = d2.transfer(ny, nx, **GEOM)
    I = f32(d2.forward(d2.fields(T.astype(np.complex128), inc.astype(np.complex128)), h))
    rng = np.random.default_rng(2)
    phi_star = rng.uniform(-np.pi, np.pi, M)
    T_est = c64(np.exp(-1j * phi_star)[:, None] * T)
    wts = np.sum(np.abs(T_est.astype(np.complex128)) ** 2, axis=1)
    phi_o, f_o, _ = d2.fit(d2.fields(T_est.astype(np.complex128), inc.astype(np.complex128)), I, h,
                           iters=150, weights=wts)
    phi = torch.empty(M, dtype=torch.float64, device="cuda")
    To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    with tmr.tmr_create(N, M, J, to_dev(d), dop(ny, nx, inc), dict(phase_iters=150)) as hd:
        tmr.tmr_defocus_fit(hd, to_dev(T_est), to_dev(I), phi, To)
        tmr.tmr_sync(hd, 60.0)
        f_g, _ = tmr.tmr_phase_fit_report(hd)
    assert f_g <= 1e-6 * float(np.sum(I.astype(np.float64) ** 2)), (f_g, f_o)
    err = np.angle(np.exp(1j * (to_np(phi) - phi_o)))
    assert np.max(np.abs(err)) <= 1e-3, np.max(np.abs(err))
    assert oracle.matrix_fidelity(to_np(To), T) >= 1 - 1e-6


def test_loss_at_gpu_phase_equals_oracle_loss():
    """One evaluation: the fit from phi = 0 with zero iterations leaves phi = 0
    and reports g(0) (Eq. optphase), which the oracle computes independently."""
    ny, nx, Nd, N, J = 16, 8, 9, 64, 4
    M = ny * nx
    T, d, _ = problem(N, M, J, seed=21)
    T2, _, _ = problem(N, M, J, seed=22)
    inc = incident(Nd, N, seed=23)
    h = d2.transfer(ny, nx, **GEOM)
    I = f32(d2.forward(d2.fields(T.astype(np.complex128), inc.astype(np.complex128)), h))
    g0, _ = d2.loss_grad(np.zeros(M), d2.fields(T2.astype(np.complex128), inc.astype(np.complex128)), I, h)
    phi = torch.empty(M, dtype=torch.float64, device="cuda")
    with tmr.tmr_create(N, M, J, to_dev(d), dop(ny, nx, inc), dict(phase_iters=0)) as hd:
        tmr.tmr_defocus_fit(hd, to_dev(T2), to_dev(I), phi, None)
        tmr.tmr_sync(hd, 60.0)
        loss, its = tmr.tmr_phase_fit_report(hd)
        assert its == 0 and abs(loss - g0) <= 1e-4 * g0
    assert np.all(to_np(phi) == 0.0)


def test_whole_retrieval_with_the_papers_defocus_model():
    """Rows solved, then the fit on separate-field defocus images: the matrix
    fidelity after the fit matches the oracle pipeline's."""
    ny, nx, N, J, Nd = 16, 16, 64, 4, 40
    M = ny * nx
    T, d, Y = problem(N, M, J, seed=31)
    inc = incident(Nd, N, seed=32)
    h = d2.transfer(ny, nx, **GEOM)
    I = f32(d2.forward(d2.fields(T.astype(np.complex128), inc.astype(np.complex128)), h))
    To = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    with tmr.tmr_create(N, M, J, to_dev(d), dop(ny, nx, inc), dict(phase_iters=150)) as hd:
        tmr.tmr_retrieve(hd, to_dev(Y), to_dev(I), 100, To)
        tmr.tmr_sync(hd, 60.0)
    Tg = to_np(To)
    fid = oracle.fidelity_rows(Tg, T)
    ok = fid > 0.999
    assert ok.mean() > 0.98  # the oracle's rows all reach 0.999 here
    assert oracle.matrix_fidelity(Tg[ok], T[ok]) > 0.9999


def test_argument_checks():
    ny, nx, N, J = 8, 8, 64, 4
    M = ny * nx
    _, d, _ = problem(N, M, J, seed=1)
    inc = incident(3, N, seed=1)
    bad = [dict(dop(ny, nx, inc), incident=None), dict(dop(ny, nx, inc), wavelength=0.0),
           dict(dop(ny, nx, inc), pixel=-1.0), dict(dop(ny, nx, inc), z_d=float("nan")),
           dict(dop(ny, nx, inc), kind=7)]
    for op in bad:
        with pytest.raises(tmr.TMRError) as ei:
            tmr.tmr_create(N, M, J, to_dev(d), op)
        assert ei.value.status == tmr.TMR_ERR_INVALID_ARG
    with pytest.raises(tmr.TMRError) as ei:  # three 256 x 129 grids do not fit in shared memory
        tmr.tmr_create(N, 256 * 128, J, to_dev(d), dop(256, 128, incident(2, N, seed=2)))
    assert ei.value.status == tmr.TMR_ERR_UNSUPPORTED
    with pytest.raises(ValueError):  # images of the full grid: [Nd, 4 M]
        with tmr.tmr_create(N, M, J, to_dev(d), dop(ny, nx, inc)) as hd:
            tmr.tmr_defocus_forward(hd, to_dev(np.zeros((M, N), np.complex64)),
                                    torch.empty((3, M), dtype=torch.float32, device="cuda"))
