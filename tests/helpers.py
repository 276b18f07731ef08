"""Shared helpers for the GPU tests: seeded inputs rounded to the precision the
library takes, and the error measures the parity bars are stated in."""
import numpy as np

import oracle
import synth


def rel_l2_rows(a, b):
    """max over rows of ||a_r - b_r|| / ||b_r|| (rows of b that are zero: absolute)."""
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    num = np.linalg.norm(a - b, axis=1)
    den = np.linalg.norm(b, axis=1)
    return float(np.max(np.where(den > 0, num / np.where(den > 0, den, 1), num)))


def max_rel_elem_rows(a, b):
    """max over rows r and entries i of |a_ri - b_ri| / max_i |b_ri| (complex
    modulus; rows of b that are zero: absolute).  Unlike rel_l2_rows, one
    wrong entry (a bad bin of one mask, a wrong twiddle at one index) shows at
    its full size instead of being diluted by the row's norm."""
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    num = np.max(np.abs(a - b), axis=1)
    den = np.max(np.abs(b), axis=1)
    return float(np.max(np.where(den > 0, num / np.where(den > 0, den, 1), num)))


def assert_rows_close(a, b, tol):
    """Both measures at the same bar: per-row relative L2 and per-entry error
    relative to the row's largest entry."""
    e2, em = rel_l2_rows(a, b), max_rel_elem_rows(a, b)
    assert e2 <= tol and em <= tol, f"rel L2 {e2:.3e}, max entry {em:.3e}, bar {tol:.1e}"


def c64(x):
    return np.ascontiguousarray(x, dtype=np.complex64)


def f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


def problem(N, M, J, seed=0, tm="iid", R=None, photons=None):
    """Ground truth T (complex64-rounded), masks (complex64-rounded) and
    intensities made by the oracle from them, rounded to float32: the exact
    inputs both implementations see."""
    if tm == "iid":
        T = synth.tm_iid(M, N, seed)
    else:
        T = synth.tm_modes(M, N, R, seed)
    _, d = synth.mask_phases(J, N, seed)
    T = c64(T)
    d = c64(d)
    Y = oracle.forward(T.astype(np.complex128), d.astype(np.complex128))
    if photons is not None:
        Y = synth.shot_noise(Y, synth.photon_scale(Y.mean(), photons), seed)
    return T, d, f32(Y)


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def to_np(t):
    return t.detach().cpu().numpy()
