"""GPU parity of the phase-aware coarsening criterion (ms_coarsen_mask,
ms_coarsen_ctx) against oracle/coarsen.py.

The decision is integer work on exact operations (minima, maxima and one FP64
subtraction per phase), so the masks must be bit-identical to the oracle's on
the same inputs.  Inputs are seeded synthetic phase fields with the structure
of a scanned part: a transformed band under the tracks, a sharp front, a
martensite layer, small noise, and values on a dyadic grid in some cases so
that ranges fall exactly on the tolerance.  On a context after a run, the
GPU's fractions and the oracle's differ by up to the run tolerance, so the
masks are compared on the octants whose decision that difference cannot
change.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import coarsen as oc
from tests._util import gpu_workload, oracle_workload

pytestmark = pytest.mark.gpu

RUN_TOL = 1e-4


@pytest.fixture(scope="module")
def ms():
    import paper_2402_17580_gb300 as m
    m.load()
    return m


def synthetic_phases(dims, seed, dyadic=False):
    """Seeded phase fields of a scanned block: alpha_s dissolved in a band
    along x with a sharp logistic front across y, martensite in the band
    below a depth, noise on 2 % of the points; with dyadic=True every value
    is a multiple of 2^-10."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    yc = rng.uniform(0.3, 0.7) * max(ny - 1, 1)
    hw = 0.2 * max(ny - 1, 1)
    w = rng.uniform(0.3, 0.6)
    xas = 0.9 - 0.8 / (1.0 + np.exp((np.abs(j - yc) - hw) / w))
    xam = np.where(k < rng.integers(1, max(nz, 2)), 0.0, 0.35) * (0.9 - xas) / 0.9
    noise = (rng.random(xas.shape) < 0.02) * rng.normal(0.0, 3e-3, xas.shape)
    xas = np.clip(xas + noise, 0.0, 0.9 - xam)
    if dyadic:
        xas = np.round(xas * 1024) / 1024
        xam = np.round(xam * 1024) / 1024
        xam = np.minimum(xam, 0.9 - xas)
    xb = 1.0 - xas - xam
    return xas.ravel(), xam.ravel(), xb.ravel()


CASES = [((33, 17, 9), 4, 1e-2, False), ((40, 24, 10), 4, 3e-3, False),
         ((65, 33, 17), 5, 8.0 / 1024, True), ((257, 33, 1), 7, 4.0 / 1024, True),
         ((130, 1, 1), 6, 0.0, True), ((5, 5, 5), 3, 1e-3, False)]


@pytest.mark.parametrize("dims,n_levels,tol,dyadic", CASES)
def test_masks_match_the_oracle_bit_for_bit(ms, dims, n_levels, tol, dyadic):
    """Host arrays through ms_coarsen_mask: every level's mask equals the
    oracle's, the counts equal the masks' sums, and the sizes match the
    octree's octant counts (ragged dims, flat axes, levels that run out)."""
    from paper_2402_17580_gb300 import _binding as B
    xas, xam, xb = synthetic_phases(dims, seed=sum(dims), dyadic=dyadic)
    got, counts = B.coarsen_mask(xas, xam, xb, dims, tol, n_levels)
    ref = oc.coarsen_masks(xas, xam, xb, dims, tol, n_levels)
    assert B.coarsen_sizes(dims, n_levels) == oc.mask_sizes(dims, n_levels)
    for l, (g, r) in enumerate(zip(got, ref), start=1):
        assert g.shape == r.shape, l
        np.testing.assert_array_equal(g, r, err_msg=f"level {l}")
        assert counts[l - 1] == int(r.sum())
    # a structured field leaves both kinds of octant on the first level
    if got[0].size > 8 and tol > 0:
        assert 0 < counts[0] < got[0].size


def test_negative_zero_and_nan_values(ms):
    """The kernels order the values through integer keys of the doubles:
    -0 and +0 (range 0), negative values, and a NaN, which reaches the
    ranges of the octants that hold it (range <= tol is false there, as in
    the oracle), must all give the oracle's masks."""
    from paper_2402_17580_gb300 import _binding as B
    dims, n_levels, tol = (37, 19, 11), 4, 1e-2
    xas, xam, xb = synthetic_phases(dims, seed=5)
    xam = xam.copy()
    xam[::7] = -0.0
    xb = xb - 1.5                      # negative values
    xas = xas.copy()
    xas[int(np.prod(dims)) // 2 + 3] = np.nan
    got, counts = B.coarsen_mask(xas, xam, xb, dims, tol, n_levels)
    ref = oc.coarsen_masks(xas, xam, xb, dims, tol, n_levels)
    for l, (g, r) in enumerate(zip(got, ref), start=1):
        np.testing.assert_array_equal(g, r, err_msg=f"level {l}")
        assert counts[l - 1] == int(r.sum())
    assert int(got[0].size - got[0].sum()) > 0


def test_device_pointers_on_a_torch_stream(ms):
    torch = pytest.importorskip("torch")
    from paper_2402_17580_gb300 import _binding as B
    dims, n_levels, tol = (48, 20, 12), 4, 5e-3
    xas, xam, xb = synthetic_phases(dims, seed=5)
    ref = oc.coarsen_masks(xas, xam, xb, dims, tol, n_levels)
    d = [torch.from_numpy(v).cuda() for v in (xas, xam, xb)]
    mask = torch.full((sum(oc.mask_sizes(dims, n_levels)),), 7, dtype=torch.uint8, device="cuda")
    _, sbytes = B.coarsen_sizes(dims, n_levels, with_scratch=True)
    scratch = torch.empty(sbytes, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    for sp, sb in ((0, 0), (scratch.data_ptr(), sbytes)):   # own scratch, then the caller's
        mask.fill_(7)
        torch.cuda.synchronize()
        counts = B.coarsen_mask_device(d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), dims,
                                       tol, n_levels, mask.data_ptr(), s.cuda_stream, sp, sb)
        flat = mask.cpu().numpy()
        np.testing.assert_array_equal(flat, np.concatenate([r.ravel() for r in ref]))
        assert counts == [int(r.sum()) for r in ref]
    with pytest.raises(ms.MSError, match="INVALID_ARG"):
        B.coarsen_mask_device(d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), dims, tol,
                              n_levels, mask.data_ptr(), s.cuda_stream, scratch.data_ptr(),
                              sbytes - 8)


def test_full_size_grid_sampled(ms):
    """The 256 x 256 x 64 grid (4.19M points, 7 levels): sampled octants of
    every level against the oracle's per-octant definition, and the masks
    nest (a coarsenable octant's children are coarsenable)."""
    from paper_2402_17580_gb300 import _binding as B
    dims, n_levels, tol = (256, 256, 64), 5, 4e-3
    xas, xam, xb = synthetic_phases(dims, seed=11)
    got, counts = B.coarsen_mask(xas, xam, xb, dims, tol, n_levels)
    fields = oc.phase_fields(xas, xam, xb, dims)
    rng = np.random.default_rng(12)
    for l, g in enumerate(got, start=1):
        cz, cy, cx = g.shape
        assert (cx, cy, cz) == oc.level_shape(dims, l)
        n = min(600, g.size)
        for o in rng.choice(g.size, n, replace=False):
            k, j, i = np.unravel_index(o, g.shape)
            ok = all(r <= tol for r in oc.octant_ranges(fields, l, i, j, k))
            assert g[k, j, i] == (1 if ok else 0), (l, i, j, k)
        assert counts[l - 1] == int(g.sum())
        if l > 1:
            c = got[l - 2]
            for k, j, i in zip(*np.nonzero(g)):
                assert c[2 * k:2 * k + 2, 2 * j:2 * j + 2, 2 * i:2 * i + 2].all()


def test_context_state_after_a_run(ms):
    """ms_coarsen_ctx on a block after its tracks: the same masks as
    ms_coarsen_mask on the context's own fractions, and, against the oracle's
    run of the same workload, the same decision on every octant whose ranges
    sit more than twice the run tolerance away from tol."""
    from paper_2402_17580_gb300 import _binding as B
    w = wl.block_256(dims=(48, 24, 10), n_tracks=3, n_steps=1200, T_thr=0.0)
    dims, n_levels, tol = w.specimens[0].grid.dims, 3, 1e-2
    ctx, g = gpu_workload(w)
    masks, counts = ctx.coarsen(tol, n_levels, dims)
    same, _ = B.coarsen_mask(g[0], g[1], g[2], dims, tol, n_levels)
    for a, b in zip(masks, same):
        np.testing.assert_array_equal(a, b)
    o = oracle_workload(w)
    fields = oc.phase_fields(o[0], o[1], o[2], dims)
    robust = 0
    for l, m in enumerate(masks, start=1):
        cz, cy, cx = m.shape
        for k in range(cz):
            for j in range(cy):
                for i in range(cx):
                    r = oc.octant_ranges(fields, l, i, j, k)
                    if all(v <= tol - 2 * RUN_TOL for v in r):
                        assert m[k, j, i] == 1, (l, i, j, k)
                        robust += 1
                    elif any(v > tol + 2 * RUN_TOL for v in r):
                        assert m[k, j, i] == 0, (l, i, j, k)
                        robust += 1
    assert robust >= 0.95 * sum(m.size for m in masks)
    assert 0 < counts[0] < masks[0].size
    ctx.close()


def test_errors(ms):
    from paper_2402_17580_gb300 import _binding as B
    x = np.zeros(27)
    for dims, lv, tol in (((0, 3, 3), 1, 0.0), ((3, 3, 3), 0, 0.0), ((3, 3, 3), 31, 0.0),
                          ((3, 3, 3), 1, -1.0), ((3, 3, 3), 1, float("nan"))):
        with pytest.raises(ms.MSError, match="INVALID_ARG"):
            B.coarsen_mask(x, x, x, dims, tol, lv) if dims[0] else B.coarsen_sizes(dims, lv)
    c = ms.Context(27)
    with pytest.raises(ms.MSError, match="STATE"):
        c.coarsen(0.0, 1, (3, 3, 3))
    c.close()
