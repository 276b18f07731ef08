"""Seeded synthetic inputs for TM retrieval (arXiv 2302.13524), shared by the
oracle tests, the GPU tests and the benchmark.

This module draws random numbers and nothing else: ground-truth transmission
matrices, mask phases and shot noise.  It holds none of the retrieval
method's arithmetic (no probing operator, no loss, no solver); intensities are
made by whichever implementation is under test (the oracle's forward model
for oracle inputs, the library's for GPU inputs).

The paper's own data (a holography-measured TM, a Maxwell-solved TM and camera
images) is not available; these generators stand in for it with the shapes of
the paper's workloads:

* ``tm_iid``   -- rows i.i.d. CN(0, 1/N) (the tiny parity configuration);
* ``tm_modes`` -- a fiber-like mode model T = U diag(e^{i theta}) V with R
  guided modes, U (M x R) and V^H (N x R) orthonormalised complex Gaussians
  and theta uniform: every row lies in the same R-dimensional input subspace,
  as the rows of a multimode fiber's TM do;
* ``mask_phases`` -- the J random phase vectors psi_j of Eq. probingmatrix,
  uniform in [0, 2 pi), and d_j = exp(i psi_j);
* ``shot_noise`` -- Poisson counts at a photon scale, divided back;
* ``fiber_disc`` / ``camera_frames`` -- the fiber core on a pixel grid, and
  camera-count speckle images of it (the raw input of the preprocessing).

Seeds: each draw uses ``numpy.random.default_rng([seed, stream, ...])`` with a
fixed stream number per kind (0 = TM, 1 = masks, 2 = noise, 3 = row photon
levels, 4 = camera frames), so one part can be regenerated without the others, and noise for a
single row depends only on (seed, row).
"""
from __future__ import annotations

import numpy as np

STREAM_TM, STREAM_MASK, STREAM_NOISE, STREAM_PHOTONS, STREAM_CAMERA = 0, 1, 2, 3, 4

# Workloads.  N input modes, M output pixels on an ny x nx grid (row = a*nx + b),
# J masks, K = J*N intensities per row.
CONFIGS = {
    "tiny": dict(N=64, M=128, grid=(16, 8), J=4, tm="iid", R=None, photons=None,
                 n_defocus=256, iters=200, init="random", defocus_coef=0.05),
    "plain": dict(N=2048, M=8192, grid=(128, 64), J=4, tm="modes", R=1100, photons=1e4,
                  n_defocus=50, iters=100, init="spectral", defocus_coef=0.05),
    "batching": dict(N=2286, M=8192, grid=(128, 64), J=4, tm="modes", R=1100,
                     photons=(1e3, 1e5), n_defocus=50, iters=300, init="spectral",
                     defocus_coef=0.05, tol=1e-7),
    "precision": dict(N=4096, M=16384, grid=(128, 128), J=4, tm="modes", R=2200, photons=1e4,
                      n_defocus=50, iters=100, init="spectral", defocus_coef=0.05),
    "learned": dict(N=2048, M=8192, grid=(128, 64), J=4, tm="family", R=1100, photons=1e4,
                    n_defocus=50, iters=100, init="learned", defocus_coef=0.05,
                    train_fibers=list(range(1, 26)), test_fibers=list(range(101, 106)),
                    widths=(1024, 1024)),
}


def mask_phases(J: int, N: int, seed: int = 0):
    """psi [J, N] uniform in [0, 2 pi) and masks d = exp(i psi) (complex128)."""
    rng = np.random.default_rng([seed, STREAM_MASK])
    psi = rng.uniform(0.0, 2.0 * np.pi, size=(J, N))
    return psi, np.exp(1j * psi)


def tm_iid(M: int, N: int, seed: int = 0) -> np.ndarray:
    """Rows i.i.d. complex Gaussian CN(0, 1/N), complex128 [M, N]."""
    rng = np.random.default_rng([seed, STREAM_TM])
    re = rng.standard_normal((M, N))
    im = rng.standard_normal((M, N))
    return (re + 1j * im) / np.sqrt(2.0 * N)


def tm_modes(M: int, N: int, R: int, seed: int = 0, dtype=np.complex128) -> np.ndarray:
    """Mode model T = U diag(e^{i theta}) V, U: Q-factor of an M x R complex
    Gaussian, V: conjugate transpose of the Q-factor of an N x R complex
    Gaussian, theta uniform in [0, 2 pi).  Scaled so that E||row||^2 = 1."""
    rng = np.random.default_rng([seed, STREAM_TM])
    R = min(R, M, N)
    U = np.linalg.qr(rng.standard_normal((M, R)) + 1j * rng.standard_normal((M, R)))[0]
    V = np.linalg.qr(rng.standard_normal((N, R)) + 1j * rng.standard_normal((N, R)))[0].conj().T
    theta = rng.uniform(0.0, 2.0 * np.pi, size=R)
    T = (U * np.exp(1j * theta)) @ V
    return (T * np.sqrt(M / R)).astype(dtype)


def tm_family(M: int, N: int, R: int, fiber_seed: int, basis_seed: int = 0,
              dtype=np.complex64) -> np.ndarray:
    """A fiber of a family: the input mode basis V (the guided modes seen from
    the input plane, fixed by the fiber type) comes from basis_seed; the mode
    coupling U and phases theta come from fiber_seed.  Scaled so E||row||^2 = 1."""
    rb = np.random.default_rng([basis_seed, STREAM_TM, 1])
    rf = np.random.default_rng([fiber_seed, STREAM_TM, 2])
    R = min(R, M, N)
    V = np.linalg.qr(rb.standard_normal((N, R)) + 1j * rb.standard_normal((N, R)))[0].conj().T
    U = np.linalg.qr(rf.standard_normal((M, R)) + 1j * rf.standard_normal((M, R)))[0]
    theta = rf.uniform(0.0, 2.0 * np.pi, size=R)
    T = (U * np.exp(1j * theta)) @ V
    return (T * np.sqrt(M / R)).astype(dtype)


def tm_family_device(M: int, N: int, R: int, fiber_seed: int, basis_seed: int = 0, device: str = "cuda"):
    """The fiber family of tm_family drawn on a GPU with torch's seeded
    generator (the same distribution -- shared input basis V per basis_seed,
    coupling U and phases theta per fiber_seed, E||row||^2 = 1 -- but not the
    same numbers as the numpy version).  For workloads too large to draw on
    the host in reasonable time (25 training fibers of 8192 x 2048); returns
    a complex64 torch tensor on `device`."""
    import torch

    def gen(seed, stream, sub):
        g = torch.Generator(device=device)
        g.manual_seed(int(seed) * 1_000_003 + stream * 1009 + sub)
        return g

    R = min(R, M, N)

    def cgauss(g, rows, cols):
        re = torch.randn((rows, cols), generator=g, device=device, dtype=torch.float64)
        im = torch.randn((rows, cols), generator=g, device=device, dtype=torch.float64)
        return torch.complex(re, im)

    V = torch.linalg.qr(cgauss(gen(basis_seed, STREAM_TM, 1), N, R))[0].conj().T
    gf = gen(fiber_seed, STREAM_TM, 2)
    U = torch.linalg.qr(cgauss(gf, M, R))[0]
    theta = torch.rand(R, generator=gf, device=device, dtype=torch.float64) * (2.0 * np.pi)
    T = (U * torch.exp(1j * theta)) @ V
    return (T * np.sqrt(M / R)).to(torch.complex64)


def make_tm(cfg: dict, seed: int = 0, M: int | None = None) -> np.ndarray:
    M = cfg["M"] if M is None else M
    if cfg["tm"] == "iid":
        return tm_iid(M, cfg["N"], seed)
    return tm_modes(M, cfg["N"], cfg["R"], seed)


def row_photons(cfg: dict, M: int, seed: int = 0) -> np.ndarray | None:
    """Mean photon count per pixel for each row: a constant, or log-uniform
    between two levels (uneven noise across rows)."""
    ph = cfg.get("photons")
    if ph is None:
        return None
    if isinstance(ph, tuple):
        rng = np.random.default_rng([seed, STREAM_PHOTONS])
        return np.exp(rng.uniform(np.log(ph[0]), np.log(ph[1]), size=M))
    return np.full(M, float(ph))


def shot_noise(Y: np.ndarray, scale, seed: int = 0, row_ids=None) -> np.ndarray:
    """Poisson shot noise: y_noisy = Poisson(s y) / s row by row, where s is the
    photon scale of the row (scalar or per-row array of photons per unit
    intensity).  Row r uses default_rng([seed, 2, row_ids[r]])."""
    Y = np.asarray(Y, dtype=np.float64)
    M = Y.shape[0]
    rows = np.arange(M) if row_ids is None else np.asarray(row_ids)
    s = np.broadcast_to(np.asarray(scale, dtype=np.float64), (M,))
    out = np.empty_like(Y)
    for i in range(M):
        rng = np.random.default_rng([seed, STREAM_NOISE, int(rows[i])])
        out[i] = rng.poisson(np.maximum(Y[i], 0.0) * s[i]) / s[i]
    return out


def photon_scale(Y_mean: float, photons) -> np.ndarray:
    """Photons per unit intensity so that a row of mean intensity Y_mean
    collects `photons` per pixel on average."""
    return np.asarray(photons, dtype=np.float64) / Y_mean


def fiber_disc(ny: int, nx: int, radius: float = 0.45) -> np.ndarray:
    """Pixels of an ny x nx grid (p = a*nx + b) inside the fiber core, a disc
    centred on the grid of radius `radius` times the smaller side: bool [ny*nx]."""
    a, b = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    r = radius * min(ny, nx)
    return (((a - (ny - 1) / 2) ** 2 + (b - (nx - 1) / 2) ** 2) <= r * r).ravel()


def camera_frames(K: int, H: int, W: int, photons: float = 2000.0, dark: float = 2.0,
                  radius: float = 0.45, seed: int = 0, dtype=np.uint16) -> np.ndarray:
    """K speckle images [K, H, W] of a fiber's distal end as a camera records
    them: exponential speckle of mean `photons` counts inside a centred disc,
    Poisson counts plus a Poisson dark level outside.  uint16 frames are
    clipped at 65535; float32 frames keep the counts as floats."""
    rng = np.random.default_rng([seed, STREAM_CAMERA])
    core = fiber_disc(H, W, radius).reshape(H, W)
    out = np.empty((K, H, W), dtype=dtype)
    for k0 in range(0, K, 256):  # frame blocks bound the temporaries
        k1 = min(K, k0 + 256)
        lam = rng.exponential(photons, size=(k1 - k0, H, W)) * core + dark
        counts = rng.poisson(lam)
        out[k0:k1] = np.minimum(counts, 65535) if np.dtype(dtype) == np.uint16 else counts
    return out


def sample_rows(M: int, n: int, seed: int = 0) -> np.ndarray:
    """n distinct row indices in [0, M), sorted, seeded."""
    rng = np.random.default_rng([seed, 99])
    return np.sort(rng.choice(M, size=min(n, M), replace=False))
