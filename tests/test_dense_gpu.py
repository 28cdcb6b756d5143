"""The dense one-step launch (k_track_dense): ms_run_track with no active set
(T_thr = 0), one step per launch, in the FP32 explicit path.

It is k_track's arithmetic per tile, organised for streaming the state (fixed
tile chunks per warp, the grid data of a warp's specimen kept in shared
memory, row coordinates from the tile's first point, L2 prefetch ahead).  So
its results must equal, bit for bit, those of the general kernel on the same
launches, and its work counters must agree; the results must also equal
those of two steps per launch.  The grids
below reach every branch of its set-up: row tiles with the far field (tracks
along x), tiles that cross grid rows, a ragged last tile, several specimens
of uneven sizes, subset specimens and a long line.
"""
import numpy as np
import pytest

import workloads as wl
from tests._util import gpu_workload, max_abs_diff, oracle_workload

pytestmark = pytest.mark.gpu

RUN_TOL = 1e-4


@pytest.fixture(scope="module")
def ms():
    import paper_2402_17580_gb300 as m
    m.load()
    return m


def _counters(st):
    return (st.source_evaluations, st.model_point_steps, st.farfield_node_evaluations,
            st.farfield_point_sources, st.tile_steps_active, st.launches)


def _dense_vs_general(w, **kw):
    """S = 1 through the dense launch, against S = 1 with MS_FLAG_COUNT_OPS
    (which keeps k_track: it counts the model's transcendentals per branch)
    and against S = 2 (k_track, two steps per launch)."""
    from paper_2402_17580_gb300._binding import MS_FLAG_COUNT_OPS
    c1, g1 = gpu_workload(w, steps_per_launch=1, T_thr=0.0, **kw)
    cg, gg = gpu_workload(w, steps_per_launch=1, T_thr=0.0, flags=MS_FLAG_COUNT_OPS, **kw)
    c2, g2 = gpu_workload(w, steps_per_launch=2, T_thr=0.0, **kw)
    for a, b, c in zip(g1, gg, g2):
        assert np.array_equal(a, b)
        assert np.array_equal(a, c)
    assert np.array_equal(c1.aux(), cg.aux())
    assert np.array_equal(c1.aux(), c2.aux())
    s1, sg = c1.stats(), cg.stats()
    assert sg.model_sfu_ex2 > 0 and s1.model_sfu_ex2 == 0   # the two kernels ran
    assert _counters(s1) == _counters(sg)
    for c in (c1, cg, c2):
        c.close()
    return g1, s1


@pytest.mark.parametrize("dims", [(256, 8, 4), (200, 7, 3), (129, 5, 2)])
def test_dense_launch_equals_general_kernel(ms, dims):
    """Row tiles (nx a multiple of 128), tiles across rows and a ragged tail;
    four serpentine tracks along x whose receding sources reach the far
    field on the 256-wide block."""
    w = wl.block_256(dims=dims, n_tracks=4, n_steps=3000, T_thr=0.0)
    g, st = _dense_vs_general(w)
    if dims[0] == 256:
        assert st.farfield_point_sources > 0
    o = oracle_workload(w)
    assert max_abs_diff(g, o) <= RUN_TOL


def test_dense_launch_equals_general_kernel_direct_sum(ms):
    w = wl.block_256(dims=(256, 8, 4), n_tracks=4, n_steps=1500, T_thr=0.0)
    _, st = _dense_vs_general(w, farfield_dist=0.0)
    assert st.farfield_point_sources == 0


def test_dense_launch_several_specimens(ms):
    """Specimens of uneven sizes in one context: a warp's chunks cross
    specimen boundaries."""
    w = wl.batch_64(n_specimens=5, n_lo=300, n_hi=6000, n_steps=1200, T_thr=0.0)
    _dense_vs_general(w)


def test_dense_launch_long_line(ms):
    w = wl.line_4096(n_points=4096, n_steps=2000)
    g, st = _dense_vs_general(w)
    assert st.farfield_point_sources > 0
    o = oracle_workload(w)
    assert max_abs_diff(g, o) <= RUN_TOL


def test_dense_launch_subset_specimen(ms):
    """A subset specimen (ms_set_points_subset) takes the per-point
    coordinates of point_coords4."""
    w = wl.block_256(dims=(64, 16, 8), n_tracks=3, n_steps=600, T_thr=0.0)
    sp = w.specimens[0]
    idx = np.sort(np.random.default_rng(5).choice(sp.grid.n, 777, replace=False))
    out = []
    for S in (1, 2):
        ctx = ms.Context(idx.size, T_thr=0.0, steps_per_launch=S)
        ctx.set_points_subset(sp.grid, idx)
        ctx.fill_state(w.init_xas, w.init_xam)
        ctx.run_track([sp.source], w.n_steps, w.dt)
        out.append((ctx.fractions(), ctx.aux()))
        ctx.close()
    for a, b in zip(out[0][0], out[1][0]):
        assert np.array_equal(a, b)
    assert np.array_equal(out[0][1], out[1][1])
