"""Pins of the phase-aware coarsening reference (oracle/coarsen.py) against
what fixes it without the reference itself: octant counts of the octree,
uniform fields, one perturbed point (the octants that hold it, counted in
closed form), linear ramps (an octant's range is slope x its width),
octants exactly at the tolerance, flat axes, and the hierarchy (a
coarsenable octant's children are coarsenable).  Sec. 3, the adaptive-mesh
passage: an octant of eight sibling cells is coarsened only where every
phase's values agree."""
import itertools

import numpy as np
import pytest

from oracle import coarsen as oc


def fields(dims, f):
    nx, ny, nz = dims
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return f(i, j, k).astype(np.float64).ravel()


@pytest.mark.parametrize("dims,level,expect", [
    ((33, 17, 9), 1, (16, 8, 4)), ((33, 17, 9), 3, (4, 2, 1)), ((33, 17, 9), 4, (2, 1, 0)),
    ((256, 256, 64), 1, (127, 127, 31)), ((256, 256, 64), 7, (1, 1, 0)),
    ((4096, 1, 1), 5, (127, 1, 1)), ((2, 2, 2), 1, (0, 0, 0))])
def test_octant_counts(dims, level, expect):
    """Octant i of level l spans points i 2^l .. (i + 1) 2^l, so an axis of n
    points holds floor((n - 1) / 2^l) of them; a flat axis holds one."""
    assert oc.level_shape(dims, level) == expect


def test_uniform_fields_coarsen_everywhere():
    dims = (17, 9, 5)
    n = 17 * 9 * 5
    ms = oc.coarsen_masks(np.full(n, 0.3), np.full(n, 0.2), np.full(n, 0.5), dims, 0.0, 3)
    for l, m in enumerate(ms, start=1):
        assert m.shape == oc.level_shape(dims, l)[::-1]
        assert m.all()


@pytest.mark.parametrize("phase", [0, 1, 2])
@pytest.mark.parametrize("p0", [(8, 4, 2), (5, 3, 1), (0, 0, 0), (16, 8, 4)])
def test_one_perturbed_point_blocks_exactly_its_octants(phase, p0):
    """A point raised by more than tol in any one phase blocks the octants
    whose span holds it: along each axis the i with i 2^l <= p <= (i + 1) 2^l
    (two of them where p sits on an interior multiple of 2^l)."""
    dims = (17, 9, 5)
    n = 17 * 9 * 5
    base = [np.full(n, 0.3), np.full(n, 0.1), np.full(n, 0.6)]
    i0, j0, k0 = p0
    base[phase][i0 + 17 * (j0 + 9 * k0)] += 2e-3
    ms = oc.coarsen_masks(*base, dims, 1e-3, 3)
    for l, m in enumerate(ms, start=1):
        w = 1 << l
        cz, cy, cx = m.shape
        holders = [[i for i in range(c) if i * w <= p <= (i + 1) * w]
                   for c, p in ((cx, i0), (cy, j0), (cz, k0))]
        blocked = set(itertools.product(*holders))
        for k, j, i in itertools.product(range(cz), range(cy), range(cx)):
            assert m[k, j, i] == (0 if (i, j, k) in blocked else 1), (l, i, j, k)
        assert (m == 0).sum() == len(blocked)


def test_ramp_coarsens_up_to_the_level_its_slope_allows():
    """X_as = a i (a ramp along x): every octant of level l spans 2^l points
    steps, so its range is a 2^l, coarsenable exactly while a 2^l <= tol;
    the other phases are uniform."""
    dims = (65, 9, 9)
    a = 1.0 / 1024          # exact in binary: the ranges are exact
    xas = fields(dims, lambda i, j, k: a * i)
    n = xas.size
    for tol, top in ((a * 4, 2), (a * 8, 3), (a * 8 - 1e-12, 2), (a * 0.5, 0)):
        ms = oc.coarsen_masks(xas, np.zeros(n), 1.0 - xas, dims, tol, 3)
        for l, m in enumerate(ms, start=1):
            assert m.size > 0
            assert m.all() == (l <= top) and (m.any() == (l <= top)), (tol, l)


def test_range_equal_to_tol_coarsens():
    dims = (9, 9, 9)
    n = 729
    xam = np.zeros(n)
    xam[0] = 0.25
    ms = oc.coarsen_masks(np.zeros(n), xam, np.ones(n) - xam, dims, 0.25, 1)
    assert ms[0].all()
    ms = oc.coarsen_masks(np.zeros(n), xam, np.ones(n) - xam, dims, np.nextafter(0.25, 0), 1)
    assert ms[0][0, 0, 0] == 0 and ms[0].sum() == ms[0].size - 1


def test_flat_axes_make_a_binary_tree_on_a_line():
    """A line of points (ny = nz = 1) coarsens pairs of segments: octant i of
    level l spans points i 2^l .. (i + 1) 2^l of the line."""
    x = np.zeros(33)
    x[20] = 1.0
    ms = oc.coarsen_masks(x, np.zeros(33), 1.0 - x, (33, 1, 1), 0.5, 4)
    for l, m in enumerate(ms, start=1):
        w = 1 << l
        assert m.shape == (1, 1, 32 // w)
        got = np.nonzero(m[0, 0] == 0)[0].tolist()
        assert got == [i for i in range(32 // w) if i * w <= 20 <= (i + 1) * w]


def test_children_of_a_coarsenable_octant_are_coarsenable():
    """The hierarchy: octant (i, j, k) of level l holds the points of its
    children (2i + a, 2j + b, 2k + c) of level l - 1, so its ranges bound
    theirs; on a random field with structure every level-l 1 has level-(l-1)
    children that are all 1."""
    rng = np.random.default_rng(3)
    dims = (37, 21, 13)
    xas = fields(dims, lambda i, j, k: 0.45 + 0.45 * np.tanh((i - 18.0) / 3.0))
    xas = np.clip(xas + rng.normal(0, 1e-3, xas.size) * (rng.random(xas.size) < 0.02), 0, 0.9)
    xam = fields(dims, lambda i, j, k: np.where(k > 6, 0.3, 0.0)) * (0.9 - xas) / 0.9
    ms = oc.coarsen_masks(xas, xam, 1 - xas - xam, dims, 5e-3, 4)
    assert 0 < ms[0].sum() < ms[0].size
    for l in range(1, len(ms)):
        p, c = ms[l], ms[l - 1]
        for k, j, i in zip(*np.nonzero(p)):
            assert c[2 * k:2 * k + 2, 2 * j:2 * j + 2, 2 * i:2 * i + 2].all()


def test_mask_sizes():
    assert oc.mask_sizes((33, 17, 9), 3) == [16 * 8 * 4, 8 * 4 * 2, 4 * 2 * 1]
