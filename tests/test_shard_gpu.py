"""Sharded runs of the CUDA path on one GPU (the multi-GPU partition, Sec. 3:
the ODEs are independent per point, so a partition needs no exchange).

One workload is split the way several GPUs would split it: a block into
z-slabs (shard.shard_slabs; each slab a grid of its own with the parent's
coordinates, ms_grid.k_offset), a batch into size-balanced groups of
specimens (shard.shard_specimens).  Every shard is a context on its own
stream; all shards are queued before any result is read, so their kernels
run concurrently.  The merged fractions and App. A state must equal the
unsharded run's bit for bit: the tiles, their active-set decisions and their
arithmetic are the same.
"""
import numpy as np
import pytest

import workloads as wl
from paper_2402_17580_gb300 import shard

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ms():
    import paper_2402_17580_gb300 as m
    m.load()
    return m


def _state(ctx):
    return np.stack(ctx.fractions()), ctx.aux()


def _run(ms, grids, sources, w, params):
    ctx = ms.Context(sum(g.n for g in grids), params)
    ctx.set_points(grids)
    ctx.fill_state(w.init_xas, w.init_xam)
    ctx.run_track(sources, w.n_steps, w.dt)
    return ctx


@pytest.mark.parametrize("case", ["small", "block_256"])
def test_z_slab_shards_merge_to_the_whole_run(ms, case):
    if case == "small":
        w = wl.block_256(dims=(256, 64, 16), n_tracks=6, n_steps=3000)
        parts, over = 3, dict(steps_per_launch=128)
    else:   # the bench's workload and launch configuration
        w = wl.block_256()
        parts, over = 4, dict(steps_per_launch=256, block_threads=256,
                              flags=ms._binding.MS_FLAG_GRAPH)
    sp = w.specimens[0]
    p = ms.default_params(T_thr=w.T_thr, **over)
    whole = _run(ms, [sp.grid], [sp.source], w, p)
    ref = _state(whole)
    whole.close()
    nx, ny, nz = sp.grid.dims
    slabs = shard.shard_slabs(nz, parts)
    ctxs = []
    for k0, k1 in slabs:
        assert (nx * ny * k0) % 128 == 0
        ctxs.append(_run(ms, [shard.slab_grid(sp.grid, k0, k1)], [sp.source], w, p))
    got_f = np.empty_like(ref[0])
    got_a = np.empty_like(ref[1])
    for (k0, k1), c in zip(slabs, ctxs):
        a, b = shard.slab_range(sp.grid, k0, k1)
        f, aux = _state(c)
        got_f[:, a:b] = f
        got_a[a:b] = aux
        c.close()
    np.testing.assert_array_equal(got_f, ref[0])
    np.testing.assert_array_equal(got_a, ref[1])
    assert np.min(ref[0][0]) < 0.5   # the tracks transformed the block


def test_specimen_shards_merge_to_the_whole_batch(ms):
    w = wl.batch_64(n_specimens=12, n_lo=2e3, n_hi=8e4, n_steps=2000)
    grids = [s.grid for s in w.specimens]
    srcs = [s.source for s in w.specimens]
    p = ms.default_params(T_thr=w.T_thr, steps_per_launch=128)
    whole = _run(ms, grids, srcs, w, p)
    ref = _state(whole)
    whole.close()
    sizes = [g.n for g in grids]
    offs = np.cumsum([0] + sizes)
    parts = shard.shard_specimens(sizes, 3)
    assert shard.imbalance(sizes, parts) < 1.5
    ctxs = [_run(ms, [grids[i] for i in part], [srcs[i] for i in part], w, p) for part in parts]
    got_f = np.empty_like(ref[0])
    got_a = np.empty_like(ref[1])
    for part, c in zip(parts, ctxs):
        f, aux = _state(c)
        o = 0
        for i in part:
            got_f[:, offs[i]:offs[i + 1]] = f[:, o:o + sizes[i]]
            got_a[offs[i]:offs[i + 1]] = aux[o:o + sizes[i]]
            o += sizes[i]
        c.close()
    np.testing.assert_array_equal(got_f, ref[0])
    np.testing.assert_array_equal(got_a, ref[1])
