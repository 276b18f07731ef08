"""FP64 reference of the paper's own defocus model (numpy).

TEST INFRASTRUCTURE: only the test suite, the benchmark's CPU leg and the
smoke check may use it.

Sec. 2.3, Eq. angularspectrum and Eq. forwarddefocusImage: with n separate
incident fields e^{j theta_n} (length N each) the transmitted fields on the
half-sampled grid are c_n = TM_est e^{j theta_n} (one value per grid pixel),
and the defocus image of pattern n is

    I_n = | K2^H P diag(h) K1 diag(c_n) e^{j phi} |^2

with K1 the 2D DFT of the ny x nx half grid, h the angular-spectrum kernel
h(u, v) = exp(j 2 pi / lambda sqrt(1 - (lambda u)^2 - (lambda v)^2) z_d) p(u, v)
and the pupil p = 1 where lambda sqrt(u^2 + v^2) <= NA, else 0, on the half
grid's frequencies u = kx / (nx ps), v = ky / (ny ps) (signed FFT-order
indices, ps the pixel of the half grid), P the zero padding of the spectrum to
the full 2ny x 2nx grid (frequency index k of a side of n points goes to
k mod 2n, signed k in [-n/2, n/2)), and K2^H the inverse 2D DFT of the full
grid.  Readings: K2^H carries the factor 1 / (ny nx), so that with h = 1 the
full-grid field at the even pixels (2a, 2b) equals the half-grid field at
(a, b) (the padding "reverses the half-sampling"); I_n is the full-grid image,
row-major 2ny x 2nx.

The phase-offset fit minimises g(phi) = sum_n ||I_n - |A_n e^{j phi}|^2||^2
(Eq. optphase), A_n = K2^H P diag(h) K1 diag(c_n), with the gradient of
Eq. phasederive, by L-BFGS with Armijo backtracking (the same optimiser
reading as the same-grid fit: memory m, first and restarted directions
-grad / max|grad|, c1 = 1e-4, at most 30 halvings), then the free constant of
phi is removed: arg sum_r w_r e^{j phi_r} = 0.
"""
from __future__ import annotations

import numpy as np


def signed_freq(n: int) -> np.ndarray:
    """Signed FFT-order integer frequencies of n points: k for k < n/2, k - n after."""
    k = np.arange(n)
    return np.where(2 * k < n, k, k - n)


def transfer(ny: int, nx: int, wavelength: float, na: float, z_d: float, pixel: float) -> np.ndarray:
    """h[ky][kx] on the half grid's frequencies (Eq. angularspectrum with the pupil)."""
    v = signed_freq(ny)[:, None] / (ny * pixel)
    u = signed_freq(nx)[None, :] / (nx * pixel)
    rho2 = (wavelength * u) ** 2 + (wavelength * v) ** 2
    inside = np.sqrt(rho2) <= na
    arg = np.sqrt(np.clip(1.0 - rho2, 0.0, None))
    h = np.exp(1j * 2.0 * np.pi / wavelength * arg * z_d)
    return np.where(inside, h, 0.0)


def pad_spectrum(X: np.ndarray) -> np.ndarray:
    """P: the ny x nx spectrum placed on the 2ny x 2nx grid at signed indices."""
    ny, nx = X.shape
    out = np.zeros((2 * ny, 2 * nx), dtype=complex)
    ry = signed_freq(ny) % (2 * ny)
    rx = signed_freq(nx) % (2 * nx)
    out[np.ix_(ry, rx)] = X
    return out


def crop_spectrum(V: np.ndarray) -> np.ndarray:
    """P^T: the entries of the 2ny x 2nx spectrum at the half grid's signed indices."""
    ny, nx = V.shape[0] // 2, V.shape[1] // 2
    ry = signed_freq(ny) % (2 * ny)
    rx = signed_freq(nx) % (2 * nx)
    return V[np.ix_(ry, rx)]


def apply(x: np.ndarray, h: np.ndarray) -> np.ndarray:
    """A x = K2^H P diag(h) K1 x: ny x nx field -> 2ny x 2nx field."""
    ny, nx = h.shape
    X = np.fft.fft2(np.asarray(x, dtype=complex).reshape(ny, nx)) * h
    # numpy's ifft2 divides by 4 ny nx; K2^H divides by ny nx
    return np.fft.ifft2(pad_spectrum(X)) * 4.0


def apply_adjoint(v: np.ndarray, h: np.ndarray) -> np.ndarray:
    """A^H v = K1^H diag(conj h) P^T K2 v / (ny nx): 2ny x 2nx -> ny x nx."""
    ny, nx = h.shape
    V = np.fft.fft2(np.asarray(v, dtype=complex).reshape(2 * ny, 2 * nx))
    # K1^H = ny nx ifft2, and the 1 / (ny nx) of K2^H
    return np.fft.ifft2(np.conj(h) * crop_spectrum(V))


def fields(T: np.ndarray, incident: np.ndarray) -> np.ndarray:
    """c_n = TM_est e^{j theta_n}: C[n][r] = sum_k T[r][k] incident[n][k]."""
    return (np.asarray(incident, dtype=complex) @ np.asarray(T, dtype=complex).T)


def forward(C: np.ndarray, h: np.ndarray, phi=None) -> np.ndarray:
    """I[n] = |A (c_n e^{j phi})|^2 as rows of 4 ny nx pixels (row-major 2ny x 2nx)."""
    C = np.asarray(C, dtype=complex)
    u = np.ones(C.shape[1]) if phi is None else np.exp(1j * np.asarray(phi, dtype=float))
    return np.stack([np.abs(apply(c * u, h)).reshape(-1) ** 2 for c in C])


def loss_grad(phi, C, I, h):
    """g(phi) (Eq. optphase) and dg/dphi (Eq. phasederive):
    dg/dphi = sum_n -4 Im(conj(u) conj(c_n) A^H(w_n G_n)), w_n = A(c_n u), G_n = I_n - |w_n|^2."""
    ny, nx = h.shape
    phi = np.asarray(phi, dtype=float)
    u = np.exp(1j * phi)
    g, grad = 0.0, np.zeros_like(phi)
    for c, In in zip(np.asarray(C, dtype=complex), np.asarray(I, dtype=float)):
        w = apply(c * u, h)
        G = In.reshape(2 * ny, 2 * nx) - np.abs(w) ** 2
        g += float(np.sum(G * G))
        v = np.conj(c) * apply_adjoint(w * G, h).reshape(-1)
        grad += -4.0 * np.imag(np.conj(u) * v)
    return g, grad


def fit(C, I, h, iters: int = 100, m: int = 5, weights=None, tol: float = 0.0):
    """L-BFGS over phi from 0 with Armijo backtracking; phi shifted so that
    arg sum_r w_r e^{j phi_r} = 0.  tol > 0: stop after an accepted step that
    lowers g by at most tol of its value.  Returns (phi, g, iterations)."""
    M = np.asarray(C).shape[1]
    phi = np.zeros(M)
    f, g = loss_grad(phi, C, I, h)
    S, Y = [], []
    done = 0
    for it in range(iters):
        gmax = np.max(np.abs(g))
        if not gmax > 0:
            break
        if S:  # two-loop recursion
            q = g.copy()
            al = []
            for s, y in reversed(list(zip(S, Y))):
                a = np.dot(s, q) / np.dot(y, s)
                al.append(a)
                q -= a * y
            q *= np.dot(S[-1], Y[-1]) / np.dot(Y[-1], Y[-1])
            for (s, y), a in zip(zip(S, Y), reversed(al)):
                b = np.dot(y, q) / np.dot(y, s)
                q += (a - b) * s
            p = -q
            if not np.dot(p, g) < 0:
                S, Y = [], []
                p = -g / gmax
        else:
            p = -g / gmax
        gp = np.dot(p, g)
        a, accepted = 1.0, False
        for _ in range(31):
            ft, gt = loss_grad(phi + a * p, C, I, h)
            if ft <= f + 1e-4 * a * gp:
                accepted = True
                break
            a *= 0.5
        if not accepted:
            break
        s, y = a * p, gt - g
        if np.dot(s, y) > 1e-10 * np.linalg.norm(s) * np.linalg.norm(y):
            S.append(s)
            Y.append(y)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
        decrease = f - ft
        phi, f, g = phi + s, ft, gt
        done = it + 1
        if tol > 0 and decrease <= tol * (f + decrease):
            break
    w = np.ones(M) if weights is None else np.asarray(weights, dtype=float)
    phi = phi - np.angle(np.sum(w * np.exp(1j * phi)))
    return phi, f, done
