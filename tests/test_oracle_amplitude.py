"""The oracle's amplitude cost (the Discussion's alternative for Poisson
noise, f = sum (sqrt(y) - |Qt|)^2), pinned independently of its code:
central finite differences of the loss, the Euler-type identity of the
gradient, zero loss and gradient at the truth, the line search against the
closed-form minimiser of the cases where phi is a quadratic, stationarity and
local minimality of the step on random lines, and recovery of a noiseless TM
by Algorithm 1 with this cost."""
import numpy as np

import oracle
import synth


def crandn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)


def phi(z, w, y, al):
    return float(np.sum((np.sqrt(np.maximum(y, 0)) - np.abs(z + al * w)) ** 2))


def test_loss_gradient_finite_differences_and_euler_identity():
    rng = np.random.default_rng(50)
    M, N, J = 3, 32, 4
    _, d = synth.mask_phases(J, N, seed=51)
    T = crandn(rng, M, N) / np.sqrt(N)
    Y = oracle.forward(crandn(rng, M, N) / np.sqrt(N), d)  # intensities of another TM
    with oracle.amplitude_cost():
        f, G = oracle.loss_grad(T, d, Y)
        eps = 1e-6
        for r in range(M):
            for n in (0, 5, 17, 31):
                for unit in (1.0, 1j):
                    Tp, Tm = T.copy(), T.copy()
                    Tp[r, n] += eps * unit
                    Tm[r, n] -= eps * unit
                    fd = (oracle.loss_grad(Tp, d, Y)[0][r] - oracle.loss_grad(Tm, d, Y)[0][r]) / (2 * eps)
                    an = G[r, n].real if unit == 1.0 else G[r, n].imag
                    assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (r, n, unit, fd, an)
    # <t, g> = 2 sum (|z| - a) |z| (real): g = 2 Q^H((|z| - a) z / |z|)
    for r in range(M):
        z = np.concatenate([np.fft.fft(d[j] * T[r]) for j in range(J)])
        a = np.sqrt(Y[r].ravel())
        m = np.abs(z)
        ip = np.vdot(T[r], G[r])
        assert abs(ip.real - 2 * np.sum((m - a) * m)) <= 1e-10 * np.sum(m * m)
        assert abs(ip.imag) <= 1e-10 * np.sum(m * m)
        # the loss itself, from its definition
        assert abs(f[r] - np.sum((a - m) ** 2)) <= 1e-12 * np.sum(a * a)


def test_zero_loss_and_gradient_at_the_truth():
    rng = np.random.default_rng(52)
    M, N, J = 2, 64, 4
    _, d = synth.mask_phases(J, N, seed=53)
    T = crandn(rng, M, N) / np.sqrt(N)
    Y = oracle.forward(T, d)
    with oracle.amplitude_cost():
        f, G = oracle.loss_grad(T * np.exp(0.7j), d, Y)
    assert np.all(f <= 1e-24 * np.sum(Y))
    assert np.max(np.abs(G)) <= 1e-11


def test_step_closed_forms():
    rng = np.random.default_rng(54)
    K = 200
    z, w = crandn(rng, K), crandn(rng, K)
    # y = 0: phi = sum |z + alpha w|^2, minimiser -Re<w, z> / |w|^2 (a descent line: Re<w, z> < 0)
    if np.vdot(w, z).real > 0:
        w = -w
    al = oracle.amp_step(z, w, np.zeros(K))
    assert abs(al - (-np.vdot(w, z).real / np.vdot(w, w).real)) <= 1e-12 * abs(al)
    # collinear fields z = s w (s > 0 real): phi = sum (a - |w| (s + alpha))^2 while s + alpha > 0,
    # minimiser sum |w| (a - |w| s) / sum |w|^2
    s = rng.uniform(1.0, 2.0, K)
    z2 = s * w
    a = np.abs(w) * (s + rng.uniform(0.4, 0.6, K))  # targets further out: a descent line
    want = np.sum(np.abs(w) * (a - np.abs(w) * s)) / np.sum(np.abs(w) ** 2)
    assert np.all(s + want > 0)
    al2 = oracle.amp_step(z2, w, a * a)
    assert abs(al2 - want) <= 1e-12 * abs(want)


def test_step_is_a_stationary_local_minimum():
    rng = np.random.default_rng(55)
    for trial in range(30):
        K = 300
        z = crandn(rng, K)
        y = np.abs(crandn(rng, K)) ** 2 * rng.uniform(0.5, 2.0)
        a = np.sqrt(y)
        m = np.abs(z)
        gz = (m - a) * z / m  # d phi / d conj(z): a descent line is w = -gz (+ noise) scaled
        w = -(gz + 0.3 * crandn(rng, K)) * 10.0 ** rng.uniform(-3, 2)
        d0 = np.sum((m - a) * np.real(np.conj(z) * w) / m)
        if d0 >= 0:
            w = -w
        al = oracle.amp_step(z, w, y)
        assert al > 0
        u = z + al * w
        mu = np.abs(u)
        d1 = np.sum((mu - a) * np.real(np.conj(u) * w) / mu)
        scale = np.sum(np.abs(w) * (np.abs(w) * al + mu + a))
        assert abs(d1) <= 1e-9 * scale, (trial, d1, scale)
        f0 = phi(z, w, y, al)
        assert f0 < phi(z, w, y, 0.0)
        for dl in (1e-3, 1e-2):
            assert f0 <= phi(z, w, y, al * (1 + dl)) + 1e-12 * f0
            assert f0 <= phi(z, w, y, al * (1 - dl)) + 1e-12 * f0


def test_algorithm1_recovers_a_noiseless_tm_with_the_amplitude_cost():
    rng = np.random.default_rng(56)
    M, N, J = 6, 64, 5
    _, d = synth.mask_phases(J, N, seed=57)
    T = crandn(rng, M, N) / np.sqrt(N)
    Y = oracle.forward(T, d)
    with oracle.amplitude_cost():
        Tr, loss, its, st = oracle.retrieve_rows(Y, d, 400, init="spectral", power_iters=200)
    fid = oracle.fidelity_rows(Tr, T)
    assert np.mean(fid > 1 - 1e-10) >= 5 / 6, fid
