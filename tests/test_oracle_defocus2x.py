"""The oracle's model of the paper's defocus images (Sec. 2.3, Eq.
angularspectrum, Eq. forwarddefocusImage, Eq. optphase, Eq. phasederive),
pinned independently of its numpy FFT route: a dense-matrix brute force of
K2^H P diag(h) K1 on a small grid, the interpolation identity of the zero
padding, the pupil and the kernel's closed form at its frequencies, the
adjoint identity, central finite differences of the phase loss, the constant
phase invariance, and recovery of planted offsets."""
import numpy as np
import pytest

from oracle import defocus2x as d2

GEOM = dict(wavelength=0.532, na=0.22, z_d=20.0, pixel=0.9)


def _rand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_transfer_closed_form_and_pupil():
    ny, nx = 8, 16
    h = d2.transfer(ny, nx, **GEOM)
    lam, na, z, ps = GEOM["wavelength"], GEOM["na"], GEOM["z_d"], GEOM["pixel"]
    for a in range(ny):
        for b in range(nx):
            ky = a if 2 * a < ny else a - ny
            kx = b if 2 * b < nx else b - nx
            u, v = kx / (nx * ps), ky / (ny * ps)
            r = lam * np.hypot(u, v)
            want = np.exp(2j * np.pi / lam * np.sqrt(1 - r * r) * z) if r <= na else 0.0
            assert abs(h[a, b] - want) < 1e-12
    assert np.count_nonzero(h) < h.size  # the pupil cuts some frequencies here


def test_dense_brute_force():
    ny, nx = 4, 4
    M = ny * nx
    rng = np.random.default_rng(1)
    h = np.exp(1j * rng.uniform(0, 2 * np.pi, (ny, nx))) * (rng.uniform(size=(ny, nx)) > 0.2)
    a, b = np.divmod(np.arange(M), nx)
    ky = np.where(2 * a < ny, a, a - ny)
    kx = np.where(2 * b < nx, b, b - nx)
    F1 = np.exp(-2j * np.pi * (np.outer(ky, a) / ny + np.outer(kx, b) / nx))  # [freq][pixel]
    A2, B2 = np.divmod(np.arange(4 * M), 2 * nx)
    F2H = np.exp(2j * np.pi * (np.outer(A2, ky) / (2 * ny) + np.outer(B2, kx) / (2 * nx)))  # [full pixel][freq]
    A = F2H @ np.diag(h.reshape(-1)) @ F1 / M
    x = _rand(rng, M)
    np.testing.assert_allclose(d2.apply(x, h).reshape(-1), A @ x, atol=1e-12)
    v = _rand(rng, 4 * M)
    np.testing.assert_allclose(d2.apply_adjoint(v, h).reshape(-1), A.conj().T @ v, atol=1e-12)


def test_padding_reverses_half_sampling():
    ny, nx = 8, 8
    rng = np.random.default_rng(2)
    x = _rand(rng, ny, nx)
    full = d2.apply(x, np.ones((ny, nx)))
    np.testing.assert_allclose(full[0::2, 0::2], x, atol=1e-12)


def test_phase_loss_gradient_and_invariance():
    ny, nx, Nd = 4, 8, 5
    M = ny * nx
    rng = np.random.default_rng(3)
    h = d2.transfer(ny, nx, **GEOM)
    C = _rand(rng, Nd, M)
    I = d2.forward(C, h, rng.uniform(-1, 1, M))
    phi = rng.uniform(-1, 1, M)
    g, grad = d2.loss_grad(phi, C, I, h)
    eps = 1e-6
    for k in (0, 7, 19, 31):
        e = np.zeros(M)
        e[k] = eps
        fd = (d2.loss_grad(phi + e, C, I, h)[0] - d2.loss_grad(phi - e, C, I, h)[0]) / (2 * eps)
        assert abs(fd - grad[k]) <= 1e-6 * max(1.0, abs(grad[k]))
    assert abs(np.sum(grad)) <= 1e-9 * np.sum(np.abs(grad))  # g(phi + const) = g(phi)
    assert abs(d2.loss_grad(phi + 0.7, C, I, h)[0] - g) <= 1e-9 * g


def test_planted_offsets_are_recovered():
    ny, nx, Nd, N = 8, 8, 12, 32
    M = ny * nx
    rng = np.random.default_rng(4)
    h = d2.transfer(ny, nx, **GEOM)
    T = _rand(rng, M, N) / np.sqrt(2 * N)
    theta = np.exp(1j * rng.uniform(0, 2 * np.pi, (Nd, N)))
    I = d2.forward(d2.fields(T, theta), h)
    phi_star = rng.uniform(-np.pi, np.pi, M)
    T_est = np.exp(-1j * phi_star)[:, None] * T
    phi, g, its = d2.fit(d2.fields(T_est, theta), I, h, iters=200)
    err = np.angle(np.exp(1j * (phi - phi_star)))
    err -= np.angle(np.mean(np.exp(1j * err)))
    assert np.max(np.abs(err)) < 1e-8, (np.max(np.abs(err)), g, its)
