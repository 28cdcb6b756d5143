"""The synthetic inputs follow their stated recipe (CPU).

The paper's part data is not available, so every input is a seeded synthetic
scan at the paper's process scales (Tables 5 and 6).  These tests check each
generator against its recipe: seeds, sizes, parameter ranges, serpentine
geometry (track j + 1 starts where and when track j ends), layer surfaces and
times, and the branch coverage of the random states.
"""
import math

import numpy as np
import pytest

import workloads as wl

TR_X0, TR_Y0, TR_UX, TR_UY, TR_V, TR_P, TR_TS, TR_LAYER = range(8)


def _check_serpentine(tracks, length_of):
    """Consecutive tracks of a layer: the next starts where and when the
    previous ends, in the opposite direction (no jump time)."""
    for a, b in zip(tracks[:-1], tracks[1:]):
        if a[TR_LAYER] != b[TR_LAYER]:
            continue
        L = length_of(a)
        assert b[TR_TS] == pytest.approx(a[TR_TS] + L / a[TR_V], rel=1e-12)
        assert a[TR_UX] * b[TR_UX] + a[TR_UY] * b[TR_UY] == pytest.approx(-1.0, abs=1e-12)


def test_line_4096():
    w = wl.line_4096()
    g = w.specimens[0].grid
    assert g.dims == (4096, 1, 1) and g.spacing[0] == 1e-5
    assert w.n_steps == 2000 and w.dt == 1e-5 and w.T_thr == 0.0
    tr = w.specimens[0].source.tracks
    assert tr.shape == (1, 8) and tr[0, TR_P] == 200.0 and tr[0, TR_V] == 1.0
    assert w.point_updates == 4096 * 2000


def test_block_256():
    w = wl.block_256()
    assert w.meta["seed"] == wl.SEED_BASE + 2
    g = w.specimens[0].grid
    assert g.dims == (256, 256, 64) and g.spacing == (1e-5, 1e-5, -1e-5)
    assert w.n_steps == 20000 and w.T_thr == 600.0
    assert w.point_updates == 256 * 256 * 64 * 20000
    tr = w.specimens[0].source.tracks
    assert tr.shape == (20, 8)
    assert np.all((tr[:, TR_P] >= 150) & (tr[:, TR_P] <= 250))
    assert np.all((tr[:, TR_V] >= 0.8) & (tr[:, TR_V] <= 1.2))
    # centred lines 100 um apart: 0.325 mm + j 0.1 mm across the 2.55 mm width
    np.testing.assert_allclose(tr[:, TR_Y0], 0.325e-3 + 1e-4 * np.arange(20), rtol=0, atol=1e-15)
    L = 255 * 1e-5
    assert np.all(np.isin(tr[:, TR_X0], [0.0, L]))
    _check_serpentine(tr, lambda a: L)
    # seeded: the same arrays every time, another seed gives others
    np.testing.assert_array_equal(tr, wl.block_256().specimens[0].source.tracks)
    assert not np.array_equal(tr, wl.block_256(seed=1).specimens[0].source.tracks)


def test_batch_64():
    w = wl.batch_64()
    assert w.meta["seed"] == wl.SEED_BASE + 3 and len(w.specimens) == 64
    sizes = []
    for sp in w.specimens:
        nx, ny, nz = sp.grid.dims
        assert nx == ny and nz == 16
        sizes.append(sp.grid.n)
        src = sp.source
        assert 0.0 <= src.t_offset <= 5e-3
        tr = src.tracks
        assert np.all(tr[:, TR_P] == tr[0, TR_P]) and 150 <= tr[0, TR_P] <= 300
        assert np.all(tr[:, TR_V] == tr[0, TR_V]) and 0.5 <= tr[0, TR_V] <= 1.5
        if len(tr) > 1:
            hatch = np.diff(tr[:, TR_Y0])
            assert np.allclose(hatch, hatch[0], rtol=1e-9) and 80e-6 <= hatch[0] <= 120e-6
        width = (nx - 1) * 1e-5
        _check_serpentine(tr, lambda a: width)
    sizes = np.array(sizes)
    # n ~ logU[1e4, 2e6] rounded to a square of 16 layers
    assert sizes.min() >= 0.8e4 and sizes.max() <= 2.1e6
    # 64 draws of mean (2e6 - 1e4) / ln 200 = 3.8e5; the seeded set holds 1.51e7
    assert sizes.sum() == 15136960
    assert np.median(np.log(sizes)) == pytest.approx(0.5 * (math.log(1e4) + math.log(2e6)), abs=1.0)


def test_part_512():
    w = wl.part_512()
    g = w.specimens[0].grid
    assert g.dims == (512, 512, 256) and w.n_steps == 250000 and w.dt == 1e-5
    src = w.specimens[0].source
    L = src.layers
    assert L.shape == (5, 4)
    # surfaces 30 um apart, the last at 0; 0.5 s per layer
    np.testing.assert_allclose(L[:, 0], [-120e-6, -90e-6, -60e-6, -30e-6, 0.0], atol=1e-15)
    np.testing.assert_allclose(L[:, 1], 0.5 * np.arange(5), atol=1e-12)
    np.testing.assert_allclose(L[:, 3], 0.5 * np.arange(1, 6), atol=1e-12)
    assert np.all(L[:, 2] < L[:, 3]) and np.all(L[:, 2] > L[:, 1])
    tr = src.tracks
    half = 0.5 * 511e-5
    for l in range(5):
        t = tr[tr[:, TR_LAYER] == l]
        assert 0 < len(t) <= 50
        th = math.radians(67.0 * l)
        # every track runs along the layer's direction (either way) ...
        cross = t[:, TR_UX] * math.sin(th) - t[:, TR_UY] * math.cos(th)
        np.testing.assert_allclose(cross, 0.0, atol=1e-12)
        # ... from a point of the square's boundary
        dx, dy = np.abs(t[:, TR_X0] - half), np.abs(t[:, TR_Y0] - half)
        assert np.all(np.maximum(dx, dy) == pytest.approx(half, rel=1e-9))
        assert t[0, TR_TS] == pytest.approx(L[l, 1])
        assert np.all(np.diff(t[:, TR_TS]) > 0)
    assert np.all(tr[:, TR_P] == 200.0) and np.all(tr[:, TR_V] == 1.0)
    # the first layer's scan: 50 lines of 5.11 mm at 1 m/s
    assert L[0, 2] - L[0, 1] == pytest.approx(50 * 511e-5, rel=1e-9)


def test_surrogate_lines():
    w = wl.surrogate_lines()
    assert w.meta["seed"] == wl.SEED_BASE + 4 and len(w.specimens) == 128
    for sp in w.specimens:
        assert sp.grid.dims == (512, 1, 1)
        ox, oy, oz = sp.grid.origin
        assert 0.0 <= -oz <= 1e-4 and 0.0 <= oy <= 3e-4
        tr = sp.source.tracks
        assert tr.shape == (3, 8)
        assert np.all((tr[:, TR_P] >= 150) & (tr[:, TR_P] <= 250))
        assert np.all((tr[:, TR_V] >= 0.8) & (tr[:, TR_V] <= 1.2))
        _check_serpentine(tr, lambda a: 511e-5)


@pytest.mark.parametrize("block", [1, 10, 100])
def test_random_states_cover_every_branch_region(block):
    n = 20000
    xas, xam, T0, T1 = wl.random_states(n, seed=5, block=block)
    assert np.all(xas >= 0) and np.all(xam >= 0) and np.all(xas + xam <= 0.9)
    gap = 0.9 - (xas + xam)
    assert not np.any((gap > 0) & (gap < 1e-5))
    # the App. A selectors: pure beta, full alpha_s, alpha_s only, alpha_m only
    assert np.any((xas == 0) & (xam == 0)) and np.any((xas == 0.9) & (xam == 0))
    assert np.any((xam == 0) & (xas > 0) & (xas < 0.9)) and np.any((xas == 0) & (xam > 0))
    # every temperature band at both levels
    for lo, hi in wl.T_BANDS:
        assert np.any((T0 >= lo) & (T0 < hi)) and np.any((T1 >= lo) & (T1 < hi))
    # blocks of identical band choices
    band = lambda T: np.searchsorted([b[1] for b in wl.T_BANDS], T, side="right")
    b0 = band(T0)[: (n // block) * block].reshape(-1, block)
    assert np.all(b0 == b0[:, :1])
