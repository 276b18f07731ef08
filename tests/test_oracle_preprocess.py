"""Pins for the camera preprocessing oracle (half-sampling, fiber mask, rows):
index-coded frames, closed-form masks, brute force over pixel subsets on tiny
inputs, and exact integer energies."""
import itertools

import numpy as np
import pytest

from oracle import preprocess as pp


def coded_frames(K, H, W):
    """frames[k, r, c] = k * 10^6 + r * 10^3 + c: every value names its own position."""
    k, r, c = np.meshgrid(np.arange(K), np.arange(H), np.arange(W), indexing="ij")
    return (k * 1_000_000 + r * 1_000 + c).astype(np.int64)


@pytest.mark.parametrize("H,W", [(7, 6), (6, 7), (1, 5), (8, 8)])
@pytest.mark.parametrize("offset", [0, 1])
def test_half_sample_keeps_every_other_pixel(H, W, offset):
    K = 3
    hs = pp.half_sample(coded_frames(K, H, W), offset)
    ny, nx = pp.half_grid(H, W, offset)
    assert hs.shape == (K, ny, nx)
    # the kept grid is every in-range index of the form 2a + offset
    assert ny == len([r for r in range(H) if r % 2 == offset])
    assert nx == len([c for c in range(W) if c % 2 == offset])
    for k in range(K):
        for a in range(ny):
            for b in range(nx):
                v = int(hs[k, a, b])
                assert (v // 1_000_000, (v // 1_000) % 1_000, v % 1_000) == (k, 2 * a + offset, 2 * b + offset)


def test_half_sample_rejects_other_offsets():
    with pytest.raises(ValueError):
        pp.half_sample(np.zeros((1, 4, 4)), 2)


@pytest.mark.parametrize("frac", [0.3, 0.5, 0.999, 1.0])
def test_mask_of_a_uniform_disc_is_the_disc(frac):
    """Equal energies inside a disc, none outside: every threshold set that
    reaches any fraction of the total is the whole disc (ties included)."""
    ny, nx = 24, 17
    a, b = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    disc = (a - 11.5) ** 2 + (b - 8.0) ** 2 <= 7.5 ** 2
    E = np.where(disc, 5, 0).astype(np.uint64).ravel()
    np.testing.assert_array_equal(pp.fiber_mask(E, frac), disc.ravel())


def test_mask_of_powers_of_two():
    """E = 2^i, i < 20, total 2^20 - 1.  The top c pixels hold 2^20 - 2^(20-c),
    which reaches 0.999 * (2^20 - 1) first at c = 10 (2^10 = 1024 <= 1049.6 < 2^11),
    and 0.5 * (2^20 - 1) already at c = 1."""
    rng = np.random.default_rng(3)
    i = rng.permutation(20)
    E = (np.uint64(1) << i.astype(np.uint64))
    m = pp.fiber_mask(E, 0.999)
    assert m.sum() == 10 and set(i[m]) == set(range(10, 20))
    m = pp.fiber_mask(E, 0.5)
    assert m.sum() == 1 and i[m][0] == 19


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("frac", [0.5, 0.9, 0.999])
def test_mask_is_the_smallest_subset_brute_force(seed, frac):
    """Over all subsets of 11 distinct energies: the mask has the smallest
    cardinality of any subset reaching frac of the total, reaches it, and
    every pixel in it is brighter than every pixel outside."""
    rng = np.random.default_rng(seed)
    E = rng.choice(10_000, size=11, replace=False).astype(np.uint64)
    total = float(E.sum())
    best = min(len(s) for r in range(12) for s in itertools.combinations(range(11), r)
               if float(sum(int(E[j]) for j in s)) >= frac * total)
    m = pp.fiber_mask(E, frac)
    assert m.sum() == best
    assert float(E[m].sum()) >= frac * total
    if not m.all():
        assert E[m].min() > E[~m].max()


def test_mask_frac_one_keeps_the_lit_pixels():
    E = np.array([0, 3, 0, 1, 7, 0], dtype=np.uint64)
    np.testing.assert_array_equal(pp.fiber_mask(E, 1.0), E > 0)


def test_mask_of_dark_frames_is_empty():
    assert not pp.fiber_mask(np.zeros(9, np.uint64), 0.999).any()
    assert not pp.fiber_mask(np.zeros(9), 0.999).any()


@pytest.mark.parametrize("frac", [0.0, -0.1, 1.5])
def test_mask_rejects_fractions_outside_the_unit_interval(frac):
    with pytest.raises(ValueError):
        pp.fiber_mask(np.ones(3), frac)


def test_integer_energy_is_exact():
    """4097 saturated uint16 frames: E = 4097 * 65535 per pixel exactly."""
    fr = np.full((4097, 2, 4), 65535, dtype=np.uint16)
    E = pp.pixel_energy(pp.half_sample(fr))
    assert E.dtype == np.uint64 and (E == 4097 * 65535).all()


@pytest.mark.parametrize("offset", [0, 1])
def test_camera_rows_are_the_kept_pixels_pixel_major(offset):
    """y[p, i] = frame i at camera pixel (2a + offset, 2b + offset) for p = a*nx + b
    inside the mask, zero outside, checked entry by entry."""
    K, H, W = 5, 9, 8
    rng = np.random.default_rng(offset)
    fr = rng.integers(0, 50, size=(K, H, W)).astype(np.uint16)
    fr[:, :, : 3] = 0  # a dark band: those pixels fall outside the mask
    y, mask, E = pp.camera_rows(fr, offset, 0.95)
    ny, nx = pp.half_grid(H, W, offset)
    assert y.shape == (ny * nx, K) and y.dtype == np.float32
    for a in range(ny):
        for b in range(nx):
            p = a * nx + b
            r, c = 2 * a + offset, 2 * b + offset
            assert E[p] == sum(int(fr[i, r, c]) for i in range(K))
            for i in range(K):
                assert y[p, i] == (fr[i, r, c] if mask[p] else 0)
    assert mask.any() and not mask.all()


def test_camera_frames_generator():
    """Seeded, shaped and structured as stated: the same seed gives the same
    frames, the disc is bright and the outside holds only the dark level."""
    import synth
    a = synth.camera_frames(300, 20, 30, seed=9)
    b = synth.camera_frames(300, 20, 30, seed=9)
    c = synth.camera_frames(300, 20, 30, seed=10)
    assert a.dtype == np.uint16 and a.shape == (300, 20, 30)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    core = synth.fiber_disc(20, 30, 0.45).reshape(20, 30)
    assert core.sum() > 0 and (~core).sum() > 0
    assert a[:, core].mean() > 1000 and a[:, ~core].mean() < 5
    f = synth.camera_frames(8, 6, 6, seed=1, dtype=np.float32)
    assert f.dtype == np.float32 and (f >= 0).all() and np.array_equal(f, np.round(f))
