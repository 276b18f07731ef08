"""FP64 CPU oracle for reference-less TM retrieval (arXiv 2302.13524).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the CUDA library
never calls it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, FP64, naive O(N^2) DFT); this
module only loads the compiled library and marshals numpy arrays.  The
pipeline helper ``retrieve_tm`` strings the C steps together in the order of
the paper: per-row retrieval (Algorithm 1), then the defocus phase-offset fit
(Sec. 2.3, Eq. optphase) and its application TM_true = diag(e^{i phi}) TM_est
(Eq. phaseoffset).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")

INIT = {"random": 0, "bp": 1, "spectral": 2, "given": 3, "lanczos": 4}
ROW_MAXITER, ROW_CONVERGED, ROW_ZERO, ROW_NUMERIC = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, FP64, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        c_int, c_dbl, c_u64 = ctypes.c_int, ctypes.c_double, ctypes.c_uint64
        sig = {
            "orc_num_threads": ([], c_int),
            "orc_dft": ([dp, dp, c_int, c_int], c_int),
            "orc_forward": ([dp, dp, c_int, c_int, c_int, dp, dp], c_int),
            "orc_adjoint": ([dp, dp, c_int, c_int, c_int, dp], c_int),
            "orc_loss_grad": ([dp, dp, dp, c_int, c_int, c_int, dp, dp], c_int),
            "orc_philox4x32_10": ([u32p, u32p, u32p], None),
            "orc_random_cnormal": ([c_u64, c_int, c_int, dp], c_int),
            "orc_init": ([dp, dp, c_int, c_int, c_int, ip, c_int, c_u64, c_int, c_dbl, dp], c_int),
            "orc_quartic_argmin": ([dp], c_dbl),
            "orc_lbfgs_direction": ([c_int, dp, dp, dp, c_int, dp], c_int),
            "orc_retrieve": ([dp, dp, c_int, c_int, c_int, ip, c_int, c_int, c_int, c_u64, c_int,
                              c_dbl, c_dbl, dp, dp, ip, ip], c_int),
            "orc_lbfgs_step": ([dp, dp, c_int, c_int, dp, dp, dp, c_int, dp, dp, dp, dp, dp, dp],
                               c_int),
            "orc_defocus_apply": ([dp, c_int, c_int, dp, c_dbl, c_int, dp], c_int),
            "orc_defocus_forward": ([dp, c_int, c_int, c_int, dp, c_dbl, dp, dp], c_int),
            "orc_phase_loss_grad": ([dp, dp, dp, c_int, c_int, c_int, dp, c_dbl, dp, dp], c_int),
            "orc_phase_fit": ([dp, dp, c_int, c_int, c_int, dp, c_dbl, c_int, c_int, dp, dp, ip,
                               dp, c_dbl], c_int),
            "orc_fidelity_rows": ([dp, dp, c_int, c_int, dp], c_int),
            "orc_set_probe_2d": ([c_int, c_int], c_int),
            "orc_set_cost": ([c_int], c_int),
            "orc_amp_step": ([dp, dp, dp, ctypes.c_size_t], c_dbl),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def num_threads() -> int:
    return lib().orc_num_threads()


def dft(x, sign: int = -1) -> np.ndarray:
    """Unnormalised DFT, X[k] = sum_n x[n] exp(sign 2 pi i k n / N)."""
    x = _c128(x)
    X = np.empty_like(x)
    assert lib().orc_dft(_p(x), _p(X), x.size, sign) == 0
    return X


class probe_2d:
    """Context in which the probing DFT K of every oracle call for rows of
    length N is the 2D DFT of the row read as an n1 x (N / n1) array (paper:
    "the 2D Fourier transform matrix for N_kx x 2N_ky"), its spectrum stored
    column by column (pattern k1 + n1 k2).  Outside it K is the 1D DFT."""

    def __init__(self, n1: int, N: int):
        self.n1, self.N = int(n1), int(N)

    def __enter__(self):
        if lib().orc_set_probe_2d(self.n1, self.N) != 0:
            raise ValueError("n1 must divide N")
        return self

    def __exit__(self, *a):
        lib().orc_set_probe_2d(0, 0)


class amplitude_cost:
    """Context in which every oracle call uses the amplitude cost
    f = sum (sqrt(y) - |Qt|)^2 (the Discussion's alternative for Poisson
    noise) with its gradient 2 Q^H((|z| - a) z / |z|) and its line search
    (orc_amp_step); outside it the paper's intensity cost (Eq. optTMsmall2)."""

    def __enter__(self):
        lib().orc_set_cost(1)
        return self

    def __exit__(self, *a):
        lib().orc_set_cost(0)


def amp_step(z, w, y) -> float:
    """The amplitude cost's step along a line with fields z + alpha w."""
    z = _c128(z).ravel()
    w = _c128(w).ravel()
    y = _f64(y).ravel()
    return lib().orc_amp_step(_p(z), _p(w), _p(y), y.size)


def forward(T, masks, return_fields: bool = False):
    """Y[m, j, k] = |F(d_j * t_m)[k]|^2 (Eq. optTMsmall2); optionally Z = Q t too."""
    T = _c128(T)
    masks = _c128(masks)
    M, N = T.shape
    J = masks.shape[0]
    Y = np.empty((M, J, N))
    Z = np.empty((M, J, N), np.complex128) if return_fields else None
    assert lib().orc_forward(_p(T), _p(masks), M, N, J, _p(Z), _p(Y)) == 0
    return (Y, Z) if return_fields else Y


def adjoint(V, masks) -> np.ndarray:
    """(Q^H v)[n] = sum_j conj(d_j[n]) sum_k exp(+2 pi i k n/N) v[j, k], per row."""
    V = _c128(V)
    masks = _c128(masks)
    M, J, N = V.shape
    out = np.empty((M, N), np.complex128)
    assert lib().orc_adjoint(_p(V), _p(masks), M, N, J, _p(out)) == 0
    return out


def loss_grad(T, masks, Y):
    """f = ||y - |Qt|^2||^2 and g = -4 Q^H diag(Qt)(y - |Qt|^2) per row (Eq. derivative)."""
    T = _c128(T)
    masks = _c128(masks)
    Y = _f64(Y)
    M, N = T.shape
    J = masks.shape[0]
    loss = np.empty(M)
    G = np.empty((M, N), np.complex128)
    assert lib().orc_loss_grad(_p(T), _p(masks), _p(Y), M, N, J, _p(loss), _p(G)) == 0
    return loss, G


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.empty(4, np.uint32)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib().orc_philox4x32_10(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p), o.ctypes.data_as(u32p))
    return o


def random_cnormal(seed: int, row: int, N: int) -> np.ndarray:
    out = np.empty(N, np.complex128)
    lib().orc_random_cnormal(seed, row, N, _p(out))
    return out


def init(Y, masks, init: str = "spectral", seed: int = 0, power_iters: int = 100,
         clip: float = 2.0, row_ids=None) -> np.ndarray:
    Y = _f64(Y)
    masks = _c128(masks)
    M, J, N = Y.shape
    rid = None if row_ids is None else np.ascontiguousarray(row_ids, dtype=np.int32)
    T0 = np.empty((M, N), np.complex128)
    assert lib().orc_init(_p(Y), _p(masks), M, N, J, _ip(rid), INIT[init], seed, power_iters,
                          clip, _p(T0)) == 0
    return T0


def quartic_argmin(c) -> float:
    c = _f64(c)
    return lib().orc_quartic_argmin(_p(c))


def lbfgs_direction(g, S, Y) -> np.ndarray:
    """p = -H g by the two-loop recursion; S, Y: [np][n] pairs, oldest first."""
    g = _f64(g)
    S = _f64(S).reshape(-1, g.size)
    Y = _f64(Y).reshape(-1, g.size)
    p = np.empty_like(g)
    lib().orc_lbfgs_direction(g.size, _p(g), _p(S), _p(Y), S.shape[0], _p(p))
    return p


def retrieve_rows(Y, masks, iters: int, m: int = 5, init: str = "spectral", seed: int = 0,
                  power_iters: int = 100, clip: float = 2.0, tol: float = 0.0, T_init=None,
                  row_ids=None):
    """Algorithm 1 on every row; returns (T, loss, iters_done, status)."""
    Y = _f64(Y)
    masks = _c128(masks)
    M, J, N = Y.shape
    rid = None if row_ids is None else np.ascontiguousarray(row_ids, dtype=np.int32)
    if T_init is not None:
        T = _c128(T_init).copy()
        init = "given"
    else:
        T = np.zeros((M, N), np.complex128)
    loss = np.empty(M)
    it = np.empty(M, np.int32)
    st = np.empty(M, np.int32)
    assert lib().orc_retrieve(_p(Y), _p(masks), M, N, J, _ip(rid), iters, m, INIT[init], seed,
                              power_iters, clip, tol, _p(T), _p(loss), _ip(it), _ip(st)) == 0
    return T, loss, it, st


def lbfgs_step(y, masks, t, S=None, Yh=None):
    """One iteration of Algorithm 1 from state (t, pairs); see orc_lbfgs_step."""
    y = _f64(y)
    masks = _c128(masks)
    t = _c128(t)
    N = t.size
    J = masks.shape[0]
    if S is None:
        S = np.zeros((0, 2 * N))
        Yh = np.zeros((0, 2 * N))
    S = _f64(S).reshape(-1, 2 * N)
    Yh = _f64(Yh).reshape(-1, 2 * N)
    p = np.empty(N, np.complex128)
    coef = np.empty(5)
    alpha = ctypes.c_double()
    tn = np.empty(N, np.complex128)
    loss = ctypes.c_double()
    g = np.empty(N, np.complex128)
    lib().orc_lbfgs_step(_p(y), _p(masks), N, J, _p(t), _p(S), _p(Yh), S.shape[0], _p(p),
                         _p(coef), ctypes.byref(alpha), _p(tn), ctypes.byref(loss), _p(g))
    return dict(p=p, coef=coef, alpha=alpha.value, t=tn, loss=loss.value, g=g)


def defocus_apply(x, H=None, coef: float = 0.05, adjoint: bool = False) -> np.ndarray:
    """D x = ifft2(H .* fft2(x)) (adjoint: conj(H)) on a 2D field x."""
    x = _c128(x)
    ny, nx = x.shape
    Hc = None if H is None else _c128(H)
    out = np.empty_like(x)
    assert lib().orc_defocus_apply(_p(x), ny, nx, _p(Hc), coef, int(adjoint), _p(out)) == 0
    return out


def defocus_forward(C, grid, H=None, coef: float = 0.05, phi=None) -> np.ndarray:
    """I_n = |D(c_n * e^{i phi})|^2 for fields C [Nd, ny*nx]."""
    C = _c128(C)
    Nd = C.shape[0]
    ny, nx = grid
    Hc = None if H is None else _c128(H)
    ph = None if phi is None else _f64(phi)
    out = np.empty((Nd, ny * nx))
    assert lib().orc_defocus_forward(_p(C), Nd, ny, nx, _p(Hc), coef, _p(ph), _p(out)) == 0
    return out


def phase_loss_grad(phi, C, Ydef, grid, H=None, coef: float = 0.05):
    """g(phi) of Eq. optphase and its gradient, Eq. phasederive."""
    phi = _f64(phi)
    C = _c128(C)
    Ydef = _f64(Ydef)
    ny, nx = grid
    Hc = None if H is None else _c128(H)
    loss = np.zeros(1)
    grad = np.empty(ny * nx)
    assert lib().orc_phase_loss_grad(_p(phi), _p(C), _p(Ydef), C.shape[0], ny, nx, _p(Hc), coef,
                                     _p(loss), _p(grad)) == 0
    return loss[0], grad


def phase_fit(C, Ydef, grid, H=None, coef: float = 0.05, iters: int = 100, m: int = 5,
              weights=None, tol: float = 0.0):
    """L-BFGS/Armijo fit of phi from phi = 0; returns (phi, iters_done, loss).
    tol > 0: stop after an accepted step that lowers the loss by at most tol
    of its value."""
    C = _c128(C)
    Ydef = _f64(Ydef)
    ny, nx = grid
    Hc = None if H is None else _c128(H)
    w = None if weights is None else _f64(weights)
    phi = np.empty(ny * nx)
    done = np.zeros(1, np.int32)
    loss = np.zeros(1)
    assert lib().orc_phase_fit(_p(C), _p(Ydef), C.shape[0], ny, nx, _p(Hc), coef, iters, m,
                               _p(w), _p(phi), _ip(done), _p(loss), float(tol)) == 0
    return phi, int(done[0]), loss[0]


def fidelity_rows(A, B) -> np.ndarray:
    """|<a_r, b_r>| / (||a_r|| ||b_r||) per row (0 for a zero row)."""
    A = _c128(A)
    B = _c128(B)
    out = np.empty(A.shape[0])
    lib().orc_fidelity_rows(_p(A), _p(B), A.shape[0], A.shape[1], _p(out))
    return out


def matrix_fidelity(A, B) -> float:
    """|sum_r <a_r, b_r>| / (||A||_F ||B||_F): one global phase allowed."""
    A = _c128(A)
    B = _c128(B)
    num = abs(np.vdot(A.ravel(), B.ravel()))
    den = np.linalg.norm(A) * np.linalg.norm(B)
    return float(num / den) if den > 0 else 0.0


def defocus_fields(T, masks, n_defocus: int) -> np.ndarray:
    """c_n = column n of Z = Q t over all rows, for the first n_defocus patterns: [Nd, M]."""
    _, Z = forward(T, masks, return_fields=True)
    M = Z.shape[0]
    return np.ascontiguousarray(Z.reshape(M, -1)[:, :n_defocus].T)


def retrieve_tm(Y, masks, Ydef, grid, iters: int, m: int = 5, init: str = "spectral",
                seed: int = 0, power_iters: int = 100, clip: float = 2.0, tol: float = 0.0,
                H=None, coef: float = 0.05, phase_iters: int = 100, T_init=None):
    """The whole path: rows by Algorithm 1, then (if Ydef is given) the phase
    offset fit on the first Ydef.shape[0] patterns and T_out = diag(e^{i phi}) T_est.
    Returns dict(T, T_est, phi, loss, iters, status)."""
    T_est, loss, it, st = retrieve_rows(Y, masks, iters, m, init, seed, power_iters, clip, tol,
                                        T_init=T_init)
    out = dict(T_est=T_est, loss=loss, iters=it, status=st, phi=None, T=T_est)
    if Ydef is not None:
        Nd = Ydef.shape[0]
        C = defocus_fields(T_est, masks, Nd)
        wts = np.sum(np.abs(T_est) ** 2, axis=1)
        phi, pit, ploss = phase_fit(C, Ydef, grid, H, coef, phase_iters, m, weights=wts)
        out.update(phi=phi, phase_iters=pit, phase_loss=ploss,
                   T=np.exp(1j * phi)[:, None] * T_est)
    return out
