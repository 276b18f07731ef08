"""Pins for the FP64 oracle against facts that do not come from the oracle itself:
closed-form DFTs, library routines (numpy.fft, numpy.linalg), Parseval and
phase invariance, finite differences, brute force on tiny inputs and published
known-answer vectors."""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def dense_Q(masks):
    """Explicit probing matrix [F D_1; ...; F D_J] from numpy's FFT of the identity."""
    J, N = masks.shape
    F = np.fft.fft(np.eye(N), axis=0)
    return np.concatenate([F * masks[j][None, :] for j in range(J)], axis=0)


# --------------------------------------------------------------------- DFT
@pytest.mark.parametrize("N", [1, 2, 3, 8, 64, 127, 2286])
def test_dft_matches_numpy(N):
    rng = np.random.default_rng(N)
    x = crandn(rng, N)
    np.testing.assert_allclose(oracle.dft(x, -1), np.fft.fft(x), rtol=0, atol=1e-12 * N)
    np.testing.assert_allclose(oracle.dft(x, +1), N * np.fft.ifft(x), rtol=0, atol=1e-12 * N)


def test_dft_closed_forms():
    N = 16
    delta = np.zeros(N, complex)
    delta[0] = 1
    np.testing.assert_allclose(oracle.dft(delta), np.ones(N), atol=1e-15)
    np.testing.assert_allclose(oracle.dft(np.ones(N)), N * delta, atol=1e-13)
    n = np.arange(N)
    for k0 in (1, 5, 15):
        e = np.exp(2j * np.pi * k0 * n / N)
        expect = np.zeros(N, complex)
        expect[k0] = N
        np.testing.assert_allclose(oracle.dft(e), expect, atol=1e-12)


def test_dft_parseval_and_roundtrip():
    rng = np.random.default_rng(1)
    for N in (7, 64, 100):
        x = crandn(rng, N)
        X = oracle.dft(x)
        assert abs(np.sum(abs(X) ** 2) - N * np.sum(abs(x) ** 2)) < 1e-11 * N * np.sum(abs(x) ** 2)
        np.testing.assert_allclose(oracle.dft(X, +1) / N, x, atol=1e-13)


# ----------------------------------------------------------- forward model
def test_forward_matches_dense_Q():
    rng = np.random.default_rng(2)
    M, N, J = 5, 24, 3
    T = crandn(rng, M, N)
    _, d = synth.mask_phases(J, N, seed=3)
    Y, Z = oracle.forward(T, d, return_fields=True)
    Q = dense_Q(d)
    Zd = (Q @ T.T).T.reshape(M, J, N)
    np.testing.assert_allclose(Z, Zd, atol=1e-12)
    np.testing.assert_allclose(Y, abs(Zd) ** 2, atol=1e-12)


def test_forward_parseval_and_phase_invariance():
    rng = np.random.default_rng(4)
    M, N, J = 6, 32, 4
    T = crandn(rng, M, N)
    _, d = synth.mask_phases(J, N, seed=5)
    Y = oracle.forward(T, d)
    np.testing.assert_allclose(Y.sum((1, 2)), J * N * np.sum(abs(T) ** 2, 1), rtol=1e-12)
    Y2 = oracle.forward(T * np.exp(1j * rng.uniform(0, 6.3, (M, 1))), d)
    np.testing.assert_allclose(Y2, Y, rtol=1e-10, atol=1e-12)


def test_adjoint_is_adjoint_and_matches_dense():
    rng = np.random.default_rng(6)
    M, N, J = 3, 20, 3
    T = crandn(rng, M, N)
    V = crandn(rng, M, J, N)
    _, d = synth.mask_phases(J, N, seed=7)
    _, Z = oracle.forward(T, d, return_fields=True)
    A = oracle.adjoint(V, d)
    for r in range(M):
        assert abs(np.vdot(Z[r].ravel(), V[r].ravel()) - np.vdot(T[r], A[r])) < 1e-10
    Q = dense_Q(d)
    np.testing.assert_allclose(A, (Q.conj().T @ V.reshape(M, -1).T).T, atol=1e-11)


# --------------------------------------------------------- loss / gradient
def test_gradient_finite_differences():
    rng = np.random.default_rng(8)
    N, J = 8, 3
    t = crandn(rng, N) / 3
    _, d = synth.mask_phases(J, N, seed=9)
    y = oracle.forward(crandn(rng, 1, N) / 3, d)[0] + 0.05
    f0, g = oracle.loss_grad(t[None], d, y[None])
    h = 1e-6
    fd = np.zeros(N, complex)
    for n in range(N):
        for part, unit in ((0, 1.0), (1, 1j)):
            tp = t.copy()
            tm = t.copy()
            tp[n] += h * unit
            tm[n] -= h * unit
            fp, _ = oracle.loss_grad(tp[None], d, y[None])
            fm, _ = oracle.loss_grad(tm[None], d, y[None])
            val = (fp[0] - fm[0]) / (2 * h)
            fd[n] += val if part == 0 else 1j * val
    assert np.max(abs(fd - g[0])) < 1e-7 * np.max(abs(g[0]))


def test_gradient_identities():
    rng = np.random.default_rng(10)
    M, N, J = 4, 32, 4
    T = crandn(rng, M, N)
    _, d = synth.mask_phases(J, N, seed=11)
    Y = oracle.forward(crandn(rng, M, N), d)
    f, G = oracle.loss_grad(T, d, Y)
    Yt, Z = oracle.forward(T, d, return_fields=True)
    R = Y - abs(Z) ** 2
    np.testing.assert_allclose(f, np.sum(R ** 2, (1, 2)), rtol=1e-12)
    for r in range(M):
        ip = np.vdot(G[r], T[r])
        # Euler: d/dc f(c t) at c = 1 equals Re(g^H t) = -4 sum r |z|^2
        assert abs(ip.real - (-4 * np.sum(R[r] * abs(Z[r]) ** 2))) < 1e-9 * abs(ip.real)
        # global-phase invariance: Im(g^H t) = 0
        assert abs(ip.imag) < 1e-9 * abs(ip.real)
    f0, G0 = oracle.loss_grad(T, d, Yt)
    assert np.all(f0 < 1e-20 * np.sum(Yt ** 2, (1, 2)))
    assert np.max(abs(G0)) < 1e-9


# -------------------------------------------------------------- inits
def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        rows = [ln.split("|") for ln in fh if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for lhs, rhs in rows:
        words = [int(w, 16) for w in lhs.split()]
        expect = [int(w, 16) for w in rhs.split()]
        got = oracle.philox4x32_10(words[:4], words[4:])
        assert [int(v) for v in got] == expect


def test_random_normals_are_standard():
    from scipy import stats
    x = np.concatenate([oracle.random_cnormal(123, r, 4096) for r in range(4)])
    for part in (x.real, x.imag):
        assert stats.kstest(part, "norm").pvalue > 1e-3
    assert abs(np.mean(abs(x) ** 2) - 2.0) < 0.05
    np.testing.assert_array_equal(oracle.random_cnormal(123, 2, 64), x[2 * 4096:2 * 4096 + 64])


def test_bp_init_is_least_squares():
    rng = np.random.default_rng(12)
    M, N, J = 3, 16, 4
    _, d = synth.mask_phases(J, N, seed=13)
    Y = oracle.forward(crandn(rng, M, N), d)
    T0 = oracle.init(Y, d, "bp")
    Q = dense_Q(d)
    for r in range(M):
        ls = np.linalg.lstsq(Q, np.sqrt(Y[r].ravel()).astype(complex), rcond=None)[0]
        np.testing.assert_allclose(T0[r], ls, atol=1e-12)


def test_spectral_init_is_leading_eigenvector():
    rng = np.random.default_rng(14)
    M, N, J, clip = 3, 16, 4, 2.0
    _, d = synth.mask_phases(J, N, seed=15)
    Y = oracle.forward(crandn(rng, M, N), d)
    T0 = oracle.init(Y, d, "spectral", seed=1, power_iters=3000, clip=clip)
    Q = dense_Q(d)
    for r in range(M):
        y = Y[r].ravel()
        tau = np.minimum(y / y.mean(), clip)
        A = Q.conj().T @ (tau[:, None] * Q) / (J * N)
        w, V = np.linalg.eigh(A)
        v = V[:, -1]
        fid = abs(np.vdot(v, T0[r])) / np.linalg.norm(T0[r])
        assert fid > 1 - 1e-9
        assert abs(np.sum(abs(T0[r]) ** 2) - y.sum() / (J * N)) < 1e-10 * y.sum()


def _krylov_ritz(A, v, k):
    """Rayleigh-Ritz on span{v, A v, ..., A^(k-1) v}: the Krylov matrix built by
    repeated products, an orthonormal basis by QR, the top eigenvector of the
    projected matrix by eigh, mapped back (no Lanczos recurrence)."""
    Kr = np.empty((v.size, k), complex)
    x = v / np.linalg.norm(v)
    for j in range(k):
        Kr[:, j] = x
        x = A @ x
        x /= np.linalg.norm(x)
    B, _ = np.linalg.qr(Kr)
    w, S = np.linalg.eigh(B.conj().T @ A @ B)
    return B @ S[:, -1]


def test_lanczos_start_is_the_krylov_ritz_vector():
    """k Lanczos steps give the Ritz vector of the k-dimensional Krylov space of
    A = Q^H diag(tau) Q / (J N) from the Philox start, at the Parseval norm, with
    Re<t, v_0> >= 0; k = N gives the leading eigenvector of A itself."""
    rng = np.random.default_rng(40)
    M, N, J, clip = 3, 16, 4, 2.0
    _, d = synth.mask_phases(J, N, seed=41)
    Y = oracle.forward(crandn(rng, M, N), d)
    Q = dense_Q(d)
    for k in (3, 6, 9):
        T0 = oracle.init(Y, d, "lanczos", seed=2, power_iters=k, clip=clip)
        for r in range(M):
            y = Y[r].ravel()
            tau = np.minimum(y / y.mean(), clip)
            A = Q.conj().T @ (tau[:, None] * Q) / (J * N)
            v0 = oracle.random_cnormal(2, r, N)
            x = _krylov_ritz(A, v0, k)
            fid = abs(np.vdot(x, T0[r])) / np.linalg.norm(T0[r])
            assert fid > 1 - 1e-10, (k, r, fid)
            assert np.real(np.vdot(v0, T0[r])) > 0
            assert abs(np.sum(abs(T0[r]) ** 2) - y.sum() / (J * N)) < 1e-10 * y.sum()
    T0 = oracle.init(Y, d, "lanczos", seed=2, power_iters=N, clip=clip)
    for r in range(M):
        y = Y[r].ravel()
        tau = np.minimum(y / y.mean(), clip)
        A = Q.conj().T @ (tau[:, None] * Q) / (J * N)
        v = np.linalg.eigh(A)[1][:, -1]
        assert abs(np.vdot(v, T0[r])) / np.linalg.norm(T0[r]) > 1 - 1e-9


def test_lanczos_stops_on_an_invariant_subspace():
    """Constant intensities make tau = 1 and A = Q^H Q / (J N) = I: the first
    step finds beta_0 = 0, and the start is the random start itself."""
    N, J = 32, 4
    _, d = synth.mask_phases(J, N, seed=42)
    Y = np.full((2, J, N), 3.0)
    T_l = oracle.init(Y, d, "lanczos", seed=7, power_iters=8, row_ids=[4, 5])
    T_r = oracle.init(Y, d, "random", seed=7, row_ids=[4, 5])
    np.testing.assert_allclose(T_l, T_r, rtol=0, atol=1e-12)


def test_lanczos_and_power_starts_agree_when_both_converge():
    """Both starts approximate the same leading eigenvector: with enough steps
    each is within 1e-9 of it, hence of the other (up to the global phase)."""
    rng = np.random.default_rng(43)
    M, N, J = 4, 32, 4
    _, d = synth.mask_phases(J, N, seed=44)
    Y = oracle.forward(crandn(rng, M, N), d)
    T_p = oracle.init(Y, d, "spectral", seed=3, power_iters=4000)
    T_l = oracle.init(Y, d, "lanczos", seed=3, power_iters=N)
    f = oracle.fidelity_rows(T_l, T_p)
    assert np.all(f > 1 - 1e-9), f


def test_random_init_parseval_norm_and_rows():
    rng = np.random.default_rng(16)
    M, N, J = 4, 32, 4
    _, d = synth.mask_phases(J, N, seed=17)
    Y = oracle.forward(crandn(rng, M, N), d)
    T0 = oracle.init(Y, d, "random", seed=5, row_ids=[10, 11, 12, 13])
    for r in range(M):
        v = oracle.random_cnormal(5, 10 + r, N)
        assert abs(abs(np.vdot(v, T0[r])) / (np.linalg.norm(v) * np.linalg.norm(T0[r])) - 1) < 1e-12
        np.testing.assert_allclose(np.sum(abs(T0[r]) ** 2), Y[r].sum() / (J * N), rtol=1e-12)


# ----------------------------------------------------- line search, L-BFGS
def test_quartic_argmin_brute_force():
    from scipy.optimize import minimize_scalar
    rng = np.random.default_rng(18)
    for trial in range(200):
        K = 12
        r = rng.standard_normal(K)
        a = rng.standard_normal(K)
        b = abs(rng.standard_normal(K)) * rng.uniform(0.01, 3)
        def phi(al):
            return np.sum((r - 2 * al * a - al * al * b) ** 2)
        c = [np.sum(r * r), np.sum(-4 * r * a), np.sum(4 * a * a - 2 * r * b), np.sum(4 * a * b),
             np.sum(b * b)]
        al = oracle.quartic_argmin(c)
        grid = np.linspace(-10, 10, 20001)
        vals = np.array([phi(g) for g in grid])
        g0 = grid[np.argmin(vals)]
        res = minimize_scalar(phi, bracket=(g0 - 0.002, g0, g0 + 0.002), method="golden",
                              tol=1e-12)
        assert phi(al) <= res.fun + 1e-9 * max(1, abs(res.fun))


def test_line_search_polynomial_equals_loss():
    rng = np.random.default_rng(19)
    N, J = 16, 4
    _, d = synth.mask_phases(J, N, seed=20)
    y = oracle.forward(crandn(rng, 1, N), d)[0]
    t = crandn(rng, N) * 0.5
    out = oracle.lbfgs_step(y, d, t)
    c = out["coef"]
    for al in (-0.3, 0.0, 0.1, 0.7, out["alpha"]):
        f, _ = oracle.loss_grad((t + al * out["p"])[None], d, y[None])
        poly = sum(c[k] * al ** k for k in range(5))
        assert abs(poly - f[0]) < 1e-10 * max(1.0, f[0])
    # exact line search: the new gradient is orthogonal to the direction
    assert abs(np.vdot(out["g"], out["p"]).real) < 1e-8 * np.linalg.norm(out["g"]) * np.linalg.norm(
        out["p"])
    np.testing.assert_allclose(out["p"], -oracle.loss_grad(t[None], d, y[None])[1][0], atol=1e-12)


def test_lbfgs_quadratic_terminates_like_cg():
    rng = np.random.default_rng(21)
    n = 10
    B = rng.standard_normal((n, n))
    A = B @ B.T + n * np.eye(n)
    b = rng.standard_normal(n)
    xs = np.linalg.solve(A, b)
    x = np.zeros(n)
    S, Yl = [], []
    for it in range(n + 1):
        g = A @ x - b
        if np.linalg.norm(g) < 1e-12:
            break
        p = oracle.lbfgs_direction(g, np.array(S).reshape(-1, n), np.array(Yl).reshape(-1, n))
        al = -(g @ p) / (p @ A @ p)
        xn = x + al * p
        S.append(xn - x)
        Yl.append(A @ xn - b - g)
        x = xn
    np.testing.assert_allclose(x, xs, atol=1e-9)
    # secant condition of the newest pair: H y = s  =>  direction(-y) ... p(y) = -s
    p = oracle.lbfgs_direction(Yl[-1], np.array(S[-3:]), np.array(Yl[-3:]))
    np.testing.assert_allclose(p, -S[-1], atol=1e-9)


# -------------------------------------------------------------- Algorithm 1
def test_retrieval_recovers_known_tm_noiseless():
    cfg = dict(synth.CONFIGS["tiny"])
    M, N, J = 48, 32, 4
    T = synth.tm_iid(M, N, seed=0)
    _, d = synth.mask_phases(J, N, seed=0)
    Y = oracle.forward(T, d)
    Tr, loss, it, st = oracle.retrieve_rows(Y, d, iters=300, init="spectral", power_iters=100)
    fid = oracle.fidelity_rows(Tr, T)
    ok = fid > 0.99
    assert ok.mean() >= 0.9
    assert np.all(fid[ok] > 1 - 1e-10)
    assert np.all(loss[ok] < 1e-18 * np.sum(Y[ok] ** 2, (1, 2)))


def test_zero_and_nonfinite_rows():
    rng = np.random.default_rng(22)
    M, N, J = 3, 16, 4
    _, d = synth.mask_phases(J, N, seed=23)
    Y = oracle.forward(crandn(rng, M, N), d)
    Y[1] = 0
    Y[2, 0, 3] = np.nan
    Tr, loss, it, st = oracle.retrieve_rows(Y, d, iters=20)
    assert st[1] == oracle.ROW_ZERO and np.all(Tr[1] == 0) and it[1] == 0
    assert st[2] == oracle.ROW_NUMERIC
    assert st[0] in (oracle.ROW_MAXITER, oracle.ROW_CONVERGED)
    assert oracle.fidelity_rows(np.zeros((1, N)), np.ones((1, N)))[0] == 0


def test_early_exit_tolerance():
    M, N, J = 8, 32, 4
    T = synth.tm_iid(M, N, seed=1)
    _, d = synth.mask_phases(J, N, seed=1)
    Y = synth.shot_noise(oracle.forward(T, d), 1e3, seed=1)  # noise: the loss plateaus
    _, _, it_full, st_full = oracle.retrieve_rows(Y, d, iters=200)
    _, _, it, st = oracle.retrieve_rows(Y, d, iters=200, tol=1e-6)
    assert np.all(st_full == oracle.ROW_MAXITER) and np.all(it_full == 200)
    assert np.all(it <= 200)
    assert np.all((st == oracle.ROW_CONVERGED) == (it < 200))
    assert np.sum(st == oracle.ROW_CONVERGED) >= M // 2


# ------------------------------------------------------ defocus operator
def quad_H(ny, nx, coef):
    ky = np.fft.fftfreq(ny) * ny
    kx = np.fft.fftfreq(nx) * nx
    return np.exp(-1j * coef * (ky[:, None] ** 2 + kx[None, :] ** 2))


def test_defocus_operator_dense_and_unitary():
    rng = np.random.default_rng(24)
    ny, nx = 16, 8
    x = crandn(rng, ny, nx)
    H = quad_H(ny, nx, 0.05)
    np.testing.assert_allclose(oracle.defocus_apply(x, coef=0.05),
                               np.fft.ifft2(H * np.fft.fft2(x)), atol=1e-12)
    np.testing.assert_allclose(oracle.defocus_apply(x, H=H), oracle.defocus_apply(x, coef=0.05),
                               atol=1e-13)
    np.testing.assert_allclose(oracle.defocus_apply(x, coef=0.0), x, atol=1e-13)
    Dx = oracle.defocus_apply(x, coef=0.05)
    assert abs(np.linalg.norm(Dx) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
    np.testing.assert_allclose(oracle.defocus_apply(Dx, coef=0.05, adjoint=True), x, atol=1e-12)
    v = crandn(rng, ny, nx)
    assert abs(np.vdot(Dx, v) - np.vdot(x, oracle.defocus_apply(v, coef=0.05, adjoint=True))) < 1e-10
    # odd sizes follow numpy's signed frequency order too
    x2 = crandn(rng, 5, 7)
    np.testing.assert_allclose(oracle.defocus_apply(x2, coef=0.3),
                               np.fft.ifft2(quad_H(5, 7, 0.3) * np.fft.fft2(x2)), atol=1e-12)


def test_phase_gradient_finite_differences_and_invariance():
    rng = np.random.default_rng(25)
    ny, nx, Nd = 6, 4, 5
    P = ny * nx
    C = crandn(rng, Nd, P)
    Yd = oracle.defocus_forward(C, (ny, nx), phi=rng.uniform(-1, 1, P)) + 0.01
    phi = rng.uniform(-1, 1, P)
    f, g = oracle.phase_loss_grad(phi, C, Yd, (ny, nx))
    h = 1e-6
    fd = np.empty(P)
    for k in range(P):
        e = np.zeros(P)
        e[k] = h
        fd[k] = (oracle.phase_loss_grad(phi + e, C, Yd, (ny, nx))[0]
                 - oracle.phase_loss_grad(phi - e, C, Yd, (ny, nx))[0]) / (2 * h)
    assert np.max(abs(fd - g)) < 1e-6 * np.max(abs(g))
    assert abs(g.sum()) < 1e-9 * np.max(abs(g)) * P
    f2, _ = oracle.phase_loss_grad(phi + 0.7, C, Yd, (ny, nx))
    assert abs(f2 - f) < 1e-10 * f
    # direct evaluation of g from its definition
    u = np.exp(1j * phi)
    direct = sum(np.sum((Yd[n] - abs(np.fft.ifft2(quad_H(ny, nx, 0.05) * np.fft.fft2(
        (C[n] * u).reshape(ny, nx))).ravel()) ** 2) ** 2) for n in range(Nd))
    assert abs(direct - f) < 1e-10 * f


def test_phase_fit_recovers_planted_offsets():
    M, N, J = 128, 16, 4
    grid = (16, 8)
    T = synth.tm_iid(M, N, seed=2)
    _, d = synth.mask_phases(J, N, seed=2)
    Nd = 24
    C_true = oracle.defocus_fields(T, d, Nd)
    Yd = oracle.defocus_forward(C_true, grid)
    rng = np.random.default_rng(26)
    phi_star = rng.uniform(-np.pi, np.pi, M)
    T_est = np.exp(-1j * phi_star)[:, None] * T
    C = oracle.defocus_fields(T_est, d, Nd)
    phi, its, loss = oracle.phase_fit(C, Yd, grid, iters=300)
    err = np.angle(np.exp(1j * (phi - phi_star)))
    err = np.angle(np.exp(1j * (err - np.angle(np.mean(np.exp(1j * err))))))
    assert np.max(abs(err)) < 1e-8
    T_fix = np.exp(1j * phi)[:, None] * T_est
    assert oracle.matrix_fidelity(T_fix, T) > 1 - 1e-10
    assert oracle.matrix_fidelity(T_est, T) < 0.5


def test_phase_fit_tolerance_stops_at_the_first_small_decrease():
    """tol > 0 stops after the first accepted step that lowers the loss by at
    most tol of its value: the same fit capped at k iterations (tol = 0) gives
    the loss after each step, and the stop is the first k where the decrease
    falls below the bar (noisy images, so the loss levels off above zero)."""
    M, N, J = 128, 16, 4
    grid = (16, 8)
    T = synth.tm_iid(M, N, seed=3)
    _, d = synth.mask_phases(J, N, seed=3)
    Nd = 24
    Yd = oracle.defocus_forward(oracle.defocus_fields(T, d, Nd), grid)
    rng = np.random.default_rng(27)
    Yd = Yd * (1 + 0.02 * rng.standard_normal(Yd.shape))
    T_est = np.exp(-1j * rng.uniform(-np.pi, np.pi, M))[:, None] * T
    C = oracle.defocus_fields(T_est, d, Nd)
    losses = [oracle.phase_fit(C, Yd, grid, iters=0)[2]]
    for k in range(1, 41):
        phi_k, done_k, loss_k = oracle.phase_fit(C, Yd, grid, iters=k)
        assert done_k == k
        losses.append(loss_k)
    for tol in (0.1, 0.03, 0.02):
        want = next(k for k in range(1, 41) if losses[k - 1] - losses[k] <= tol * losses[k - 1])
        phi, done, loss = oracle.phase_fit(C, Yd, grid, iters=40, tol=tol)
        assert done == want, (tol, done, want)
        assert loss == losses[want]


# ---------------------------------------------------------- learned-init MLP
def test_mlp_gelu_matches_erf_definition():
    import math
    from oracle import mlp
    xs = np.linspace(-6, 6, 49)
    np.testing.assert_allclose(mlp.gelu(xs), [0.5 * x * (1 + math.erf(x / math.sqrt(2))) for x in xs],
                               atol=1e-15)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(xs), (mlp.gelu(xs + h) - mlp.gelu(xs - h)) / (2 * h),
                               atol=1e-8)


def test_mlp_gradient_finite_differences():
    from oracle import mlp
    rng = np.random.default_rng(30)
    dims = (8, 6, 6, 4)
    n = sum(int(np.prod(s)) for s in mlp.shapes(*dims))
    theta = rng.standard_normal(n) * 0.4
    X = rng.standard_normal((5, 8))
    T = rng.standard_normal((5, 4))
    L, g = mlp.loss_grad(theta, dims, X, T)
    # the loss is the mean squared error of the forward pass
    Y, _ = mlp.forward(theta, dims, X)
    assert abs(L - np.mean((Y - T) ** 2)) < 1e-14
    h = 1e-6
    fd = np.empty(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        fd[i] = (mlp.loss_grad(theta + e, dims, X, T)[0] - mlp.loss_grad(theta - e, dims, X, T)[0]) / (2 * h)
    assert np.max(abs(fd - g)) < 1e-8 * max(1.0, np.max(abs(g)))


def _phase_loss_closed_form(Y, T):
    """min over a of ||y - t e^{-i a}||^2 = ||y||^2 + ||t||^2 - 2 |<y, t>|, summed
    over rows and divided by the number of outputs (rows as complex vectors)."""
    n = Y.shape[1] // 2
    y = Y[:, :n] + 1j * Y[:, n:]
    t = T[:, :n] + 1j * T[:, n:]
    per = np.sum(np.abs(y) ** 2, 1) + np.sum(np.abs(t) ** 2, 1) - 2 * np.abs(np.sum(np.conj(y) * t, 1))
    return np.sum(per) / Y.size


def test_mlp_phase_invariant_loss_gradient():
    """The phase-invariant loss: its value equals the closed form of the
    minimum over the global phase, its gradient matches central differences
    of that closed form (the rotation enters only through the minimum, so the
    envelope theorem must hold), and it ignores a per-row phase of the
    targets."""
    from oracle import mlp
    rng = np.random.default_rng(31)
    dims = (8, 6, 6, 6)
    n = sum(int(np.prod(s)) for s in mlp.shapes(*dims))
    theta = rng.standard_normal(n) * 0.4
    X = rng.standard_normal((5, 8))
    T = rng.standard_normal((5, 6))
    L, g = mlp.loss_grad_phase(theta, dims, X, T)
    Y, _ = mlp.forward(theta, dims, X)
    assert abs(L - _phase_loss_closed_form(Y, T)) < 1e-13
    h = 1e-6
    fd = np.empty(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        fp = _phase_loss_closed_form(mlp.forward(theta + e, dims, X)[0], T)
        fm = _phase_loss_closed_form(mlp.forward(theta - e, dims, X)[0], T)
        fd[i] = (fp - fm) / (2 * h)
    assert np.max(abs(fd - g)) < 1e-7 * max(1.0, np.max(abs(g)))
    # a per-row phase on the targets changes nothing
    ph = np.exp(1j * rng.uniform(0, 2 * np.pi, 5))[:, None]
    t = (T[:, :3] + 1j * T[:, 3:]) * ph
    T2 = np.concatenate([t.real, t.imag], 1)
    L2, g2 = mlp.loss_grad_phase(theta, dims, X, T2)
    assert abs(L2 - L) < 1e-13 and np.max(abs(g2 - g)) < 1e-12
    # targets already aligned with the outputs (<y, t> real, positive): plain MSE
    Ta = Y + 0.01 * rng.standard_normal(Y.shape)
    ya = Y[:, :3] + 1j * Y[:, 3:]
    ta = Ta[:, :3] + 1j * Ta[:, 3:]
    c = np.sum(np.conj(ya) * ta, 1)
    ta = ta * (np.conj(c) / np.abs(c))[:, None]
    Ta = np.concatenate([ta.real, ta.imag], 1)
    assert abs(mlp.loss_grad_phase(theta, dims, X, Ta)[0] - mlp.loss_grad(theta, dims, X, Ta)[0]) < 1e-14


def test_adam_constant_gradient_closed_form():
    """Under a constant gradient g the bias-corrected moments are exactly
    m_hat = g and v_hat = g^2 at every step t (m_t = (1 - b1^t) g,
    v_t = (1 - b2^t) g^2), so after k steps theta = -k lr g / (|g| + eps).
    A missing or stale bias correction (t held at 1, or none) breaks this
    for every t > 1."""
    from oracle import mlp
    g = np.array([0.3, -2.0, 1e-3, 5.0])
    th, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in range(1, 8):
        th, m, v = mlp.adam_step(th, g, m, v, t, lr=0.01)
        np.testing.assert_allclose(th, -t * 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)


def test_adam_two_steps_by_hand():
    """g1 = 1, g2 = -2, lr = 1: m2 = -0.11, v2 = 0.004999, m_hat = -0.11 / 0.19,
    v_hat = 0.004999 / 0.001999, theta2 = -1/(1 + 1e-8) - m_hat / (sqrt(v_hat) + 1e-8)
    (worked out by hand from the definition of Adam, Kingma & Ba 2015)."""
    from oracle import mlp
    th, m, v = mlp.adam_step(np.zeros(1), np.array([1.0]), np.zeros(1), np.zeros(1), 1, lr=1.0)
    th, m, v = mlp.adam_step(th, np.array([-2.0]), m, v, 2, lr=1.0)
    assert abs(m[0] + 0.11) < 1e-15 and abs(v[0] - 0.004999) < 1e-15
    mh, vh = -0.11 / 0.19, 0.004999 / 0.001999
    assert abs(th[0] - (-1.0 / (1.0 + 1e-8) - mh / (np.sqrt(vh) + 1e-8))) < 1e-13
    assert abs(th[0] - (-1.0 + 0.366101)) < 1e-5  # 0.578947 / 1.581376


def test_adam_first_step_is_signed_lr():
    from oracle import mlp
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    th, m, v = mlp.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    # first bias-corrected step: m_hat = g, v_hat = g^2 -> -lr g / (|g| + eps)
    np.testing.assert_allclose(th, -0.01 * g / (np.abs(g) + 1e-8), atol=1e-15)
