"""The oracle's 2D probing DFT (Sec. 2.2: K the 2D Fourier transform of the
row read as an n1 x n2 array), pinned by numpy's fft2, the adjoint identity,
Parseval, central finite differences of the loss, the 1D DFT restored on
leaving the mode, and exact recovery of a noiseless known row."""
import numpy as np
import pytest

import oracle


def _rand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("N,n1", [(64, 8), (64, 4), (512, 64), (12, 3)])
def test_forward_is_numpy_fft2_column_order(N, n1):
    rng = np.random.default_rng(N + n1)
    J, n2 = 3, N // n1
    T = _rand(rng, 2, N)
    d = np.exp(1j * rng.uniform(0, 2 * np.pi, (J, N)))
    with oracle.probe_2d(n1, N):
        Y, Z = oracle.forward(T, d, return_fields=True)
    for r in range(2):
        for j in range(J):
            X = np.fft.fft2((d[j] * T[r]).reshape(n1, n2))  # X[k1][k2]
            np.testing.assert_allclose(Z[r, j], X.T.reshape(-1), atol=1e-10)  # pattern k1 + n1 k2
    np.testing.assert_allclose(Y, np.abs(Z) ** 2, rtol=1e-12)
    # Parseval: sum_i y_i = J N ||t||^2 (the 2D DFT is also unnormalised)
    np.testing.assert_allclose(Y.sum(axis=(1, 2)), J * N * np.sum(np.abs(T) ** 2, 1), rtol=1e-12)
    # leaving the mode restores the 1D DFT
    Y1 = oracle.forward(T, d)
    np.testing.assert_allclose(Y1[0, 0], np.abs(np.fft.fft(d[0] * T[0])) ** 2, rtol=1e-10)


def test_adjoint_identity_and_gradient():
    rng = np.random.default_rng(7)
    N, n1, J = 64, 8, 4
    T = _rand(rng, 1, N) / 8
    d = np.exp(1j * rng.uniform(0, 2 * np.pi, (J, N)))
    V = _rand(rng, 1, J, N)
    with oracle.probe_2d(n1, N):
        _, Z = oracle.forward(T, d, return_fields=True)
        A = oracle.adjoint(V, d)
        assert abs(np.vdot(Z, V) - np.vdot(T, A)) < 1e-10 * np.abs(np.vdot(Z, V))
        Y = oracle.forward(_rand(rng, 1, N) / 8, d)
        L, G = oracle.loss_grad(T, d, Y)
        h = 1e-6
        for i in (0, 5, 37, 63):
            for part in (1.0, 1j):
                e = np.zeros((1, N), complex)
                e[0, i] = h * part
                fd = (oracle.loss_grad(T + e, d, Y)[0] - oracle.loss_grad(T - e, d, Y)[0]) / (2 * h)
                got = G[0, i].real if part == 1.0 else G[0, i].imag
                assert abs(fd[0] - got) <= 1e-6 * max(1.0, abs(got)), (i, part)


def test_noiseless_recovery_with_the_2d_probe():
    rng = np.random.default_rng(3)
    N, n1, J, M = 64, 8, 4, 6
    T = _rand(rng, M, N) / np.sqrt(2 * N)
    d = np.exp(1j * rng.uniform(0, 2 * np.pi, (J, N)))
    with oracle.probe_2d(n1, N):
        Y = oracle.forward(T, d)
        Tr, _, _, _ = oracle.retrieve_rows(Y, d, 300, init="spectral", power_iters=60, clip=2.0)
    fid = oracle.fidelity_rows(Tr, T)
    assert np.mean(fid > 1 - 1e-10) >= 0.5, fid  # rows that converge are exact up to phase


def test_bad_split_rejected():
    with pytest.raises(ValueError):
        with oracle.probe_2d(5, 64):
            pass
