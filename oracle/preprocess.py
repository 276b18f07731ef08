"""Camera preprocessing before the per-row solves (Sec. 2.2, the procedure that
follows Algorithm 1), in plain numpy.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the CUDA library never
calls it and shares no code with it.

The paper reduces the number of row problems in two steps before solving them:

1. half-sampling: only every other pixel of each intensity image is kept, in
   both directions, so the kept grid samples the transmitted field at twice
   the camera pixel size (still above Nyquist for the fiber's NA);
2. a binary fiber mask on the half-sampled grid whose one-region holds 99.9 %
   of the total intensity; rows outside it are set to zero without being
   solved.

Readings (the paper gives the two steps in words only):

* "odd indexes" counts from one, so 0-based rows and columns
  ``offset, offset + 2, ...`` are kept with ``offset = 0`` by default;
  ``offset = 1`` keeps the other phase.  The kept grid has
  ``(H - offset + 1) // 2`` rows and ``(W - offset + 1) // 2`` columns; pixel
  ``p = a * nx + b`` of the grid is camera pixel ``(2a + offset, 2b + offset)``.
* the intensity a pixel contributes is its sum over all K probe images,
  ``E[p] = sum_i I_i[p]``;
* the mask is the smallest set of pixels, brightest first, whose energies sum
  to at least ``frac * sum(E)``; pixels tied with the last one taken are
  included (so the set is a threshold set ``E >= tau``); a set of all-dark
  frames gives an empty mask;
* integer (camera count) frames are summed exactly in 64-bit integers; float
  frames in FP64.  The comparison with ``frac * total`` is made in FP64.
* the rows handed to the solver are pixel-major, ``y[p, i] = I_i[p]`` with the
  pattern index ``i = j * N + k`` of the probing stack, and all-zero outside
  the mask (a zero row is returned as zero by the solver without iterating).
"""
from __future__ import annotations

import numpy as np


def half_grid(H: int, W: int, offset: int = 0) -> tuple[int, int]:
    """(ny, nx) of the half-sampled grid of an H x W image."""
    return (H - offset + 1) // 2, (W - offset + 1) // 2


def half_sample(frames, offset: int = 0) -> np.ndarray:
    """Keep rows and columns offset, offset + 2, ... of every frame [..., H, W]."""
    if offset not in (0, 1):
        raise ValueError("offset must be 0 or 1")
    return np.asarray(frames)[..., offset::2, offset::2]


def pixel_energy(hs) -> np.ndarray:
    """E[p] = sum over the K frames of the half-sampled intensity at pixel p;
    uint64 for integer frames (exact), float64 otherwise.  hs: [K, ny, nx]."""
    hs = np.asarray(hs)
    flat = hs.reshape(hs.shape[0], -1)
    if np.issubdtype(flat.dtype, np.integer):
        return flat.astype(np.uint64).sum(axis=0)
    return flat.astype(np.float64).sum(axis=0)


def fiber_mask(E, frac: float = 0.999) -> np.ndarray:
    """Boolean mask of the smallest brightest-first pixel set holding at least
    frac of the total energy, ties with its last pixel included."""
    if not 0.0 < frac <= 1.0:
        raise ValueError("frac must be in (0, 1]")
    E = np.asarray(E)
    total = float(E.sum())
    if E.size == 0 or total == 0.0:
        return np.zeros(E.shape, dtype=bool)
    desc = np.sort(E)[::-1]
    running = np.cumsum(desc).astype(np.float64)
    reached = running >= frac * total
    c = int(np.argmax(reached)) + 1 if reached.any() else desc.size
    tau = desc[c - 1]
    return E >= tau


def camera_rows(frames, offset: int = 0, frac: float = 0.999):
    """Camera frames [K, H, W] -> (y [M, K] float32, mask [M] bool, E [M]).

    y[p, i] is frame i at grid pixel p, zero for pixels outside the mask."""
    hs = half_sample(frames, offset)
    K = hs.shape[0]
    E = pixel_energy(hs)
    mask = fiber_mask(E, frac)
    y = np.ascontiguousarray(hs.reshape(K, -1).T, dtype=np.float32)
    y[~mask] = 0.0
    return y, mask, E
