"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances.  The kernels compute in FP32 with SFU transcendentals (relative
error ~2^-22) and store the fractions in FP32 (half an ulp of 0.9 is 3e-8).
One step therefore agrees with the oracle to ~1e-7 absolute; 2e-6 leaves room
for the temperature-dependent thresholds.  Long runs accumulate one rounding
per step, so whole runs are held to the target max|dX| <= 1e-4 and the sum of
the four fractions to 1 +- 1e-6.
"""
import numpy as np
import pytest

import oracle as orc
import workloads as wl
from tests._util import (gpu_workload, max_abs_diff, oracle_params, oracle_view,
                         oracle_workload)

pytestmark = pytest.mark.gpu

RUN_TOL = 1e-4      # max|dX| for whole runs (FP32 path vs FP64 oracle)
SUM_TOL = 1e-6      # |sum of the four fractions - 1|
STEP_TOL = 2e-6     # one step


@pytest.fixture(scope="module")
def ms():
    import paper_2402_17580_gb300 as m
    m.load()
    return m


def check_sum(fr):
    s = fr[0] + fr[1] + fr[2] + fr[3]
    assert np.max(np.abs(s - 1.0)) <= SUM_TOL
    for a in fr:
        assert np.all(a >= -1e-7) and np.all(a <= 1 + 1e-7)


# ------------------------------------------------------------ single step
@pytest.mark.parametrize("dt,block", [(1e-5, 1), (1e-3, 1), (1e-3, 10)])
def test_single_step_every_branch(ms, dt, block):
    """Brute force over random states x random (T^n, T^{n+1}) in every branch
    region (ragged count), one step via ms_step with host temperature arrays."""
    n = 6 * 128 + 37
    xas, xam, T0, T1 = wl.random_states(n, seed=11 + block, block=block)
    T0, T1 = T0.astype(np.float32), T1.astype(np.float32)
    ctx = ms.Context(n)
    ctx.set_state(xas, xam)
    ctx.step(T0, T1, dt)
    g = ctx.fractions()
    st = orc.State.make(oracle_view(xas), oracle_view(xam))
    orc.step(st, T0.astype(np.float64), T1.astype(np.float64), dt)
    o = orc.fractions(st, T1.astype(np.float64))
    assert max_abs_diff(g, np.stack(o)) <= STEP_TOL
    check_sum(g)
    gaux = ctx.aux()
    agree = np.mean((gaux > 0) == (st.mode == orc.MODE_AS_TO_B))  # ABI: aux = X~_beta > 0
    assert agree >= 0.999


def test_appendix_a_initiation_below_fp32_range(ms):
    """App. A at 1200 K from (0.9, 0, 0.1): the first step's X~_beta ~ 3.6e-70
    is far below the FP32 range; the kernel carries it in log2 form."""
    ctx = ms.Context(1)
    ctx.set_state([0.9], [0.0])
    ctx.step(np.float32([1200.0]), np.float32([1200.0]), 1e-5)
    st = orc.State.make([0.9], [0.0])
    orc.step(st, 1200.0, 1200.0, 1e-5)
    assert st.mode[0] == orc.MODE_AS_TO_B
    assert ctx.aux()[0] == pytest.approx(st.xt[0], rel=1e-4)
    for _ in range(20):
        ctx.step(np.float32([1200.0]), np.float32([1200.0]), 1e-5)
    orc.run_temps(st, np.full(21, 1200.0), 1e-5)
    assert ctx.aux()[0] == pytest.approx(st.xt[0], rel=1e-4)


def test_random_temperature_histories(ms):
    """Many steps of random temperature walks through every branch."""
    rng = np.random.default_rng(5)
    n, steps, dt = 3 * 128 + 5, 300, 1e-4
    T = np.empty((steps + 1, n), dtype=np.float32)
    T[0] = rng.uniform(300, 2100, n)
    for s in range(steps):
        T[s + 1] = np.clip(T[s] + rng.normal(0, 25, n), 280, 2600)
    xas, xam, _, _ = wl.random_states(n, seed=3)
    ctx = ms.Context(n)
    ctx.set_state(xas, xam)
    for s in range(steps):
        ctx.step(T[s], T[s + 1], dt)
    g = ctx.fractions()
    st = orc.State.make(oracle_view(xas), oracle_view(xam))
    orc.run_temps(st, T.astype(np.float64), dt)
    o = np.stack(orc.fractions(st, T[-1].astype(np.float64)))
    assert max_abs_diff(g, o) <= RUN_TOL
    check_sum(g)


@pytest.mark.parametrize("flags", [{"martensite_literal": 1}, {"init_ba_steps": 1}])
def test_reading_switches_match_the_oracle(ms, flags):
    """The readings' switches (A3: martensite set to its equilibrium below
    T_am,start; A6: the beta -> alpha_s initiation kept until the App. A exit
    rule) on random temperature walks through ms_step and on a moving-source
    line through ms_run_track, against the oracle with the same switches."""
    rng = np.random.default_rng(21)
    n, steps, dt = 2 * 128 + 9, 200, 1e-4
    T = np.empty((steps + 1, n), dtype=np.float32)
    T[0] = rng.uniform(300, 2100, n)
    for s in range(steps):
        T[s + 1] = np.clip(T[s] + rng.normal(0, 25, n), 280, 2600)
    xas, xam, _, _ = wl.random_states(n, seed=8)
    ctx = ms.Context(n, **flags)
    p = oracle_params(ctx.params)
    ctx.set_state(xas, xam)
    for s in range(steps):
        ctx.step(T[s], T[s + 1], dt)
    st = orc.State.make(oracle_view(xas), oracle_view(xam))
    orc.run_temps(st, T.astype(np.float64), dt, p)
    o = np.stack(orc.fractions(st, T[-1].astype(np.float64), p))
    assert max_abs_diff(ctx.fractions(), o) <= RUN_TOL
    w = wl.line_4096(n_points=1024, n_steps=1500)
    _, g = gpu_workload(w, **flags)
    assert max_abs_diff(g, oracle_workload(w, p=p)) <= RUN_TOL
    check_sum(g)


# ------------------------------------------------------- moving source runs
def test_line_4096_full(ms):
    """4096 points on a line under one moving source, 2000 steps of 1e-5 s,
    every point against the oracle (max|dX| <= 1e-4)."""
    w = wl.line_4096()
    _, g = gpu_workload(w)
    o = oracle_workload(w)
    assert max_abs_diff(g, o) <= RUN_TOL
    check_sum(g)
    assert np.max(g[3]) > 0.99        # the melt pool is there
    assert np.max(g[1]) > 0.5         # martensite formed behind it


def test_small_block_all_points_ragged(ms):
    """3D block with a ragged tile tail, serpentine tracks, every point."""
    w = wl.block_256(dims=(40, 24, 10), n_tracks=4, n_steps=1500, T_thr=0.0)
    _, g = gpu_workload(w)
    o = oracle_workload(w)
    assert max_abs_diff(g, o) <= RUN_TOL
    check_sum(g)


@pytest.mark.parametrize("case", ["line_4096", "small_block", "two_layers"])
def test_fp32_path_against_the_literal_appendix_a_exit(ms, case):
    """App. A leaves the alpha_s -> beta initiation once X~_beta dt > 1e-15.
    The library (and the default oracle) also wait for X~_beta >= 1e-3
    (reading A5: below that an FP32 state cannot hold 0.9 - X~_beta).  Here
    the FP32 path with its default exit rule runs against the oracle with the
    literal rule (init_exit_floor = 0) on the line, a small block and two
    layers with interlayer cooling, at the workloads' dt = 1e-5 s, every
    point: the floor moves no result there (a heating point crosses the
    alpha_s -> beta band in milliseconds, while X~_beta needs seconds to reach
    1e-10)."""
    if case == "line_4096":
        w = wl.line_4096()
    elif case == "small_block":
        w = wl.block_256(dims=(40, 24, 10), n_tracks=4, n_steps=1500, T_thr=0.0)
    else:
        w = wl.part_512(dims=(24, 20, 8), n_layers=2, tracks_per_layer=4, t_layer=2e-3,
                        hatch=5e-5)
    _, g = gpu_workload(w)
    o = oracle_workload(w, p=orc.params(init_exit_floor=0.0))
    assert max_abs_diff(g, o) <= RUN_TOL
    check_sum(g)


def test_batched_specimens_with_offsets(ms):
    """Several specimens of uneven sizes and start offsets in one context."""
    w = wl.batch_64(n_specimens=5, n_lo=200, n_hi=3000, n_steps=1200, T_thr=0.0)
    _, g = gpu_workload(w)
    o = oracle_workload(w)
    assert max_abs_diff(g, o) <= RUN_TOL
    check_sum(g)


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_layers_and_interlayer_cooling(ms, precision):
    """Two layers: inactive points above the first surface, interlayer
    cool-down to T0, rotated tracks of the second layer; every precision
    (and with the active set on)."""
    w = wl.part_512(dims=(24, 20, 8), n_layers=2, tracks_per_layer=4, t_layer=2e-3, hatch=5e-5)
    _, g = gpu_workload(w, precision=precision)
    o = oracle_workload(w)
    assert max_abs_diff(g, o) <= (1e-6 if precision == 3 else RUN_TOL)
    check_sum(g)


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_initiation_cooling_through_the_plateau(ms, precision):
    """Points in App. A alpha_s -> beta initiation (X_alpha = 0.9 above
    T_as,end) that cool through T_as,end: the initiation ends where
    X_alpha^eq returns to the plateau 0.9, in every fraction type (a state set
    to 0.9 and the plateau must compare equal when the fraction type is wider
    than the arithmetic)."""
    n = 128 + 7
    T = np.concatenate([np.full(60, 1150.0), np.linspace(1150.0, 900.0, 80), np.full(40, 353.0)])
    hist = np.tile(T[:, None], (1, n)).astype(np.float32)
    ctx = ms.Context(n, precision=precision)
    ctx.set_state(np.full(n, 0.9), np.zeros(n))
    for k in range(len(T) - 1):
        ctx.step(hist[k], hist[k + 1], 1e-5)
    g = ctx.fractions()
    s = orc.State.uniform(n, 0.9, 0.0)
    orc.run_temps(s, hist.astype(np.float64), 1e-5)
    o = np.stack(orc.fractions(s, hist[-1].astype(np.float64)))
    assert max_abs_diff(g, o) <= (1e-6 if precision in (1, 3) else RUN_TOL)
    assert np.all(np.stack(g)[0] > 0.89)


def test_block_256_full_size_sampled(ms):
    """The full 256x256x64 block, 20 tracks, 20000 steps, in the bench's launch
    configuration (active set on); 192 seeded sample points against the oracle."""
    w = wl.block_256()
    _, g = gpu_workload(w)
    idx = np.random.default_rng(9).choice(w.n_points, 192, replace=False)
    o = oracle_workload(w, idx)
    assert max_abs_diff(g, o, idx) <= RUN_TOL
    check_sum(g)


def test_batch_64_full_size_sampled(ms):
    """The full batched workload: 64 specimens of log-uniform sizes in
    [1e4, 2e6] points (1.5e7 in all), each with its own power, speed, hatch and start
    offset, 10000 steps in one context with the active set on; 256 seeded
    sample points against the oracle."""
    w = wl.batch_64()
    _, g = gpu_workload(w)
    idx = np.random.default_rng(13).choice(w.n_points, 256, replace=False)
    o = oracle_workload(w, idx)
    assert max_abs_diff(g, o, idx) <= RUN_TOL
    check_sum(g)


def test_part_512_full_size_sampled_compensated(ms):
    """The part-scale workload at full size: 512 x 512 x 256 points, 5 layers
    of 50 rotated serpentine tracks, 250000 steps, with the compensated
    fraction accumulator its length needs (plain FP32 accumulates ~2e-4 over
    the 250000 steps); 64 seeded sample points, half of them in the top 60 um
    the tracks melt, against the oracle."""
    w = wl.part_512()
    _, g = gpu_workload(w, precision=ms.MS_KAHAN)
    nx, ny, nz = w.specimens[0].grid.dims
    rng = np.random.default_rng(17)
    top = rng.integers(0, nx * ny * 6, 32)            # the six top layers of points
    rest = rng.integers(0, w.n_points, 32)
    idx = np.unique(np.concatenate([top, rest]))
    o = oracle_workload(w, idx)
    assert max_abs_diff(g, o, idx) <= RUN_TOL
    check_sum(g)


# ------------------------------------------------------------- properties
def test_steps_per_launch_is_bit_invariant(ms):
    """Temporal blocking changes no arithmetic: S = 1, 7, 32, 96 and a run
    split over several calls give identical bits."""
    w = wl.block_256(dims=(33, 9, 5), n_tracks=3, n_steps=250, T_thr=0.0)
    ref = None
    for S, chunks in ((1, 1), (7, 1), (32, 3), (96, 2)):
        _, g = gpu_workload(w, steps_per_launch=S, chunks=chunks)
        if ref is None:
            ref = g
        else:
            for a, b in zip(ref, g):
                assert np.array_equal(a, b)


def test_checkpoint_roundtrip_bit_exact(ms):
    """run(2N) == run(N); checkpoint; restore into a fresh context; run(N)."""
    w = wl.line_4096(n_points=700, n_steps=600)
    _, full = gpu_workload(w)
    ctx, _ = gpu_workload(w, n_steps=300)
    blob = ctx.checkpoint()
    ctx2 = ms.Context(w.n_points, T_thr=w.T_thr)
    ctx2.set_points([s.grid for s in w.specimens])
    ctx2.restore(blob)
    ctx2.run_track([s.source for s in w.specimens], 300, w.dt)
    for a, b in zip(full, ctx2.fractions()):
        assert np.array_equal(a, b)


def test_active_set_skip_error_is_bounded(ms):
    """Reading A9: skipping cold, saturated steps changes results by less than
    the neglected diffusion (k(600 K) * t, ~1e-5 here)."""
    w = wl.block_256(dims=(64, 16, 8), n_tracks=3, n_steps=3000, T_thr=0.0)
    _, a = gpu_workload(w, T_thr=0.0)
    _, b = gpu_workload(w, T_thr=600.0)
    assert max(float(np.max(np.abs(x - y))) for x, y in zip(a, b)) <= 2e-5


def test_active_set_skips_cold_tiles_line(ms):
    """Reading A9 with the tile bound: on the line, tiles well ahead of the
    source are cold and saturated and skip whole launches; results stay within
    the oracle budget and within the skip bound of the dense run."""
    w = wl.line_4096()
    _, dense = gpu_workload(w, T_thr=0.0)
    ctx, g = gpu_workload(w, T_thr=600.0, steps_per_launch=32)
    st = ctx.stats()
    assert st.tile_steps_active < 0.75 * st.tile_steps_total
    assert st.tile_steps_active > 0
    assert max(float(np.max(np.abs(x - y))) for x, y in zip(dense, g)) <= 2e-5
    assert max_abs_diff(g, oracle_workload(w)) <= RUN_TOL


def test_active_set_full_block_against_dense_run(ms):
    """The tile bound must never drop a tile that gets hot: on the whole
    256 x 256 x 64 block (every point compared), the run with T_thr = 600 K
    stays within the reading-A9 skip bound of the run without any skipping,
    while the bound removes a large part of the tile-steps."""
    w = wl.block_256()
    dctx, dense = gpu_workload(w, T_thr=0.0, steps_per_launch=256)
    dctx.close()
    ctx, g = gpu_workload(w, T_thr=600.0, steps_per_launch=256)
    st = ctx.stats()
    print("active tile-steps", st.tile_steps_active / st.tile_steps_total)
    assert st.tile_steps_active < 0.8 * st.tile_steps_total
    assert max(float(np.max(np.abs(x - y))) for x, y in zip(dense, g)) <= 2e-5
    ctx.close()


def test_tile_order_does_not_change_results(ms):
    """The persistent warps take the active tiles heaviest first (by the
    cycles the previous launch spent on them) or in index order
    (ms_params.tile_order); tiles are independent, so the two give the same
    bits, over several launches whose active sets and classes change."""
    w = wl.block_256(dims=(128, 48, 12), n_tracks=4, n_steps=2400)
    out = []
    for order in (0, 1):
        ctx, g = gpu_workload(w, steps_per_launch=64, tile_order=order)
        st = ctx.stats()
        assert st.tile_steps_active < st.tile_steps_total
        out.append((np.stack(g), ctx.aux()))
        ctx.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


def test_fixed_point_tiles_skip_exactly(ms):
    """A tile whose points all sit on the alpha_s plateau's fixed point
    (X_as = 0.9, X_am = 0, the untouched room-temperature state) stays out of
    the active set while the rigorous temperature bound keeps it below
    T_as,end: there every step is the identity.  With T_thr just above T0 the
    cold skip of reading A9 has nothing to act on (the receding sources keep
    the block above it), so the run must equal the dense run, and it skips
    tile-steps."""
    w = wl.block_256(dims=(128, 64, 48), n_tracks=3, n_steps=3000, T_thr=354.0)
    ctx, g = gpu_workload(w)
    st = ctx.stats()
    dctx, dense = gpu_workload(w, T_thr=0.0)
    assert st.tile_steps_active < 0.8 * st.tile_steps_total
    assert max_abs_diff(g, np.stack(dense)) == 0.0
    # the App. A variable too: points heated past T_as,end start the alpha_s
    # -> beta initiation while X_as still rounds to 0.9
    np.testing.assert_array_equal(ctx.aux(), dctx.aux())
    check_sum(g)


def test_active_set_batched_offsets(ms):
    """Specimens that have not started yet are skipped until their start."""
    w = wl.batch_64(n_specimens=6, n_lo=300, n_hi=4000, n_steps=800, T_thr=600.0)
    ctx, g = gpu_workload(w, steps_per_launch=16)
    st = ctx.stats()
    assert st.tile_steps_active < st.tile_steps_total
    assert max_abs_diff(g, oracle_workload(w)) <= RUN_TOL
    check_sum(g)


def test_f64_accumulation_parity(ms):
    """MS_F64ACC: FP64 fractions, FP32 rates; tighter agreement on the line."""
    w = wl.line_4096(n_points=1024, n_steps=2000)
    _, g = gpu_workload(w, precision=ms.MS_F64ACC)
    o = oracle_workload(w)
    assert max_abs_diff(g, o) <= 3e-5
    check_sum(g)


def test_full_fp64_path_parity(ms):
    """MS_F64: temperatures, rates and fractions in FP64 on the GPU (the
    spot-check path) agree with the FP64 oracle far below the FP32 budget."""
    w = wl.block_256(dims=(24, 10, 6), n_tracks=3, n_steps=1200, T_thr=0.0)
    _, g = gpu_workload(w, precision=ms.MS_F64)
    o = oracle_workload(w)
    assert max_abs_diff(g, o) <= 1e-6
    check_sum(g)


def test_point_subset_matches_the_full_grid(ms):
    """ms_set_points_subset: a seeded subset of the block advances exactly as
    those points do in the full-grid run (same coordinates, same arithmetic)."""
    w = wl.block_256(dims=(40, 24, 10), n_tracks=4, n_steps=700, T_thr=0.0)
    sp = w.specimens[0]
    # a subset's warps hold points of several rows, so it sums every source
    # point by point: compare with the full grid's direct sum
    _, full = gpu_workload(w, farfield_dist=0.0)
    idx = np.sort(np.random.default_rng(4).choice(sp.grid.n, 1000, replace=False))
    ctx = ms.Context(idx.size, T_thr=0.0, farfield_dist=0.0)
    ctx.set_points_subset(sp.grid, idx)
    ctx.fill_state()
    ctx.run_track([sp.source], w.n_steps, w.dt)
    sub = ctx.fractions()
    for a, b in zip(full, sub):
        assert np.array_equal(a[idx], b)


@pytest.mark.parametrize("case", ["axis", "rotated", "axis_skip", "hybrid"])
def test_row_tiles_match_the_general_form(ms, case):
    """Tiles inside one grid row (rows of 128 points here) compute the
    x-independent parts of every source's offsets once per source, and for
    levels whose sources all move along +-x the whole perpendicular distance;
    a subset specimen holding the same points takes the per-point form.  Both
    must give identical bits: serpentine along x, a second layer rotated by
    67 degrees (mixed levels), the active set on, and the hybrid kernel with a
    zero network."""
    if case == "rotated":
        w = wl.part_512(dims=(128, 10, 6), n_layers=2, tracks_per_layer=3, t_layer=5e-3,
                        hatch=3e-5)
    else:
        w = wl.block_256(dims=(128, 6, 5), n_tracks=3, n_steps=600)
    T_thr = 600.0 if case == "axis_skip" else 0.0
    sp = w.specimens[0]
    idx = np.arange(sp.grid.n, dtype=np.int64)
    zero = ms.Surrogate(np.zeros(5187, dtype=np.float32)) if case == "hybrid" else None
    out = []
    for subset in (False, True):
        ctx = ms.Context(sp.grid.n, T_thr=T_thr, steps_per_launch=128, farfield_dist=0.0)
        if subset:
            ctx.set_points_subset(sp.grid, idx)
        else:
            ctx.set_points([sp.grid])
        ctx.fill_state(w.init_xas, w.init_xam)
        if zero is not None:
            ctx.set_surrogate(zero, 0.0)
        ctx.run_track([sp.source], w.n_steps, w.dt)
        out.append((np.stack(ctx.fractions()), ctx.aux(), ctx.temperature()))
        ctx.close()
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)
    assert np.max(np.abs(out[0][0][0] - 0.9)) > 0.5   # the tracks transformed alpha_s
    if zero is not None:
        zero.close()


@pytest.mark.parametrize("T,xas,xam,ex2,slow", [
    # 900 K: X_alpha^eq on its 0.9 plateau (no exp), k_as (exp + rcp), r1 and
    # r2 (lg2 X_as shared, lg2 of each second factor, one exp each); g at
    # 900 K: no exponential (plateau, above T_am,start)
    (900.0, 0.5, 0.2, 3, 4),
    # 1000 K: X_alpha^eq = 1 - exp(.) at T^n and again in g at T^{n+1}; k_as;
    # r1 only (X_am = 0)
    (1000.0, 0.5, 0.0, 4, 3),
    # 700 K: plateau, k_as, r1 and r2, and X_am,0^eq = 1 - exp(.) in g below
    # T_am,start
    (700.0, 0.3, 0.1, 4, 4),
])
def test_model_transcendental_counts(ms, T, xas, xam, ex2, slow):
    """The roofline's per-branch count of the model's transcendentals, pinned
    by hand from the formulas of Sec. 2.2 on isothermal points (the source
    starts after the run, so T = T0 everywhere and no source is evaluated)."""
    n, steps = 3 * 128 + 5, 40
    grid = wl.Grid((0.0, 0.0, 0.0), (1e-5, 1e-5, -1e-5), (n, 1, 1))
    tracks = np.array([[0.0, 0.0, 1.0, 0.0, 1.0, 200.0, 1.0, 0]], dtype=np.float64)
    src = wl.HeatSource(tracks, np.array([[0.0, 0.0, 1e9, 1e9]]), T0=T)
    ctx = ms.Context(n, T_thr=0.0, flags=ms._binding.MS_FLAG_COUNT_OPS)
    ctx.set_points([grid])
    ctx.set_state(np.full(n, xas), np.full(n, xam))
    ctx.reset_stats()
    ctx.run_track([src], steps, 1e-5)
    st = ctx.stats()
    assert st.source_evaluations == 0
    assert st.model_point_steps == n * steps
    assert st.model_sfu_ex2 == ex2 * n * steps
    assert st.model_sfu_slow == slow * n * steps
    # without MS_FLAG_COUNT_OPS the kernel counts nothing and runs the same steps
    plain = ms.Context(n, T_thr=0.0)
    plain.set_points([grid])
    plain.set_state(np.full(n, xas), np.full(n, xam))
    plain.run_track([src], steps, 1e-5)
    assert plain.stats().model_sfu_ex2 == 0
    np.testing.assert_array_equal(np.stack(plain.fractions()), np.stack(ctx.fractions()))
    plain.close()


@pytest.mark.parametrize("dims", [(200, 7, 3), (250, 8, 4), (300, 5, 3)])
def test_farfield_on_a_ragged_row_tile(ms, dims):
    """The last tile of these grids lies inside one row but holds fewer than
    128 points, so some lanes hold no point of the specimen.  The far field
    sums the receding sources at the nodes of the tile's range in every lane
    and adds the lanes' sums across the warp, all at the row's y and z: the
    run must stay within 1e-5 of the direct sum and within the run tolerance
    of the oracle (1800 steps: the receding sources of the first tracks are
    far by then)."""
    w = wl.block_256(dims=dims, n_tracks=4, n_steps=1800, T_thr=0.0)
    assert w.n_points % 128 != 0
    _, direct = gpu_workload(w, farfield_dist=0.0)
    ctx, far = gpu_workload(w, farfield_dist=5e-3)
    assert ctx.stats().farfield_point_sources > 0
    assert max_abs_diff(far, np.stack(direct)) <= 1e-5
    assert max_abs_diff(far, oracle_workload(w)) <= RUN_TOL


@pytest.mark.parametrize("dims", [(200, 9, 4), (100, 12, 3), (160, 7, 3)])
def test_farfield_on_tiles_across_two_rows(ms, dims):
    """Rows of fewer than 256 points, not a multiple of 128: most 128-point
    tiles hold the end of one grid row and the start of the next.  The far
    field serves them over both rows' x-ranges (8 nodes each, each point
    interpolating from its own row's nodes); tiles across three rows sum
    point by point.  The run must stay within 1e-5 of the direct sum and
    within the run tolerance of the oracle, with the far field taking a
    large share of the point-source pairs."""
    w = wl.block_256(dims=dims, n_tracks=4, n_steps=3000, T_thr=0.0)
    _, direct = gpu_workload(w, farfield_dist=0.0)
    ctx, far = gpu_workload(w, farfield_dist=5e-3)
    st = ctx.stats()
    assert st.farfield_point_sources > 0.3 * (st.farfield_point_sources + st.source_evaluations)
    assert max_abs_diff(far, np.stack(direct)) <= 1e-5
    assert max_abs_diff(far, oracle_workload(w)) <= RUN_TOL


def test_farfield_matches_the_direct_sum(ms):
    """ms_params.farfield_dist: in row tiles, sources at least 5 mm behind
    every point are summed at 8 Chebyshev nodes of the tile's x-range and
    interpolated.  Four serpentine tracks over a 256 x 8 x 4 block, then
    their receding sources: the run stays within 1e-5 of the direct sum's run
    and within the run tolerance of the oracle, most point-source pairs come
    from the interpolation, and the paths it does not serve refuse it."""
    w = wl.block_256(dims=(256, 8, 4), n_tracks=4, n_steps=3000, T_thr=0.0)
    _, direct = gpu_workload(w, farfield_dist=0.0)
    ctx, far = gpu_workload(w, farfield_dist=5e-3)
    st = ctx.stats()
    assert st.farfield_node_evaluations > 0
    assert st.farfield_point_sources > 0.5 * (st.farfield_point_sources + st.source_evaluations)
    assert max_abs_diff(far, np.stack(direct)) <= 1e-5
    o = oracle_workload(w)
    assert max_abs_diff(far, o) <= RUN_TOL
    check_sum(far)
    with pytest.raises(ms.MSError):
        ms.Context(16, farfield_dist=-1.0)
    # every path with FP32 arithmetic takes it (the default); the full-FP64
    # path sums every source point by point
    for prec, tol in ((ms.MS_F64ACC, 3e-5), (ms.MS_KAHAN, 3e-5)):
        c, g = gpu_workload(w, precision=prec)
        assert c.stats().farfield_point_sources == st.farfield_point_sources
        assert max_abs_diff(g, o) <= tol
        c.close()
    c, g = gpu_workload(w, precision=ms.MS_F64)
    assert c.stats().farfield_node_evaluations == 0
    c.close()


def test_farfield_in_the_implicit_scheme(ms):
    """The implicit scheme's hot kernel takes the far field like the explicit
    one: the same temperatures to within the interpolation error, so a run
    with steps of 1e-4 s stays within 1e-5 of its direct-sum run and within
    the run tolerance of the implicit oracle."""
    w = wl.block_256(dims=(256, 8, 4), n_tracks=4, n_steps=300, T_thr=0.0)
    w.dt = 1e-4
    _, direct = gpu_workload(w, integrator=ms.MS_IMPLICIT, farfield_dist=0.0)
    ctx, far = gpu_workload(w, integrator=ms.MS_IMPLICIT)
    p = oracle_params(ctx.params)
    assert ctx.stats().farfield_point_sources > 0
    assert max_abs_diff(far, np.stack(direct)) <= 1e-5
    assert max_abs_diff(far, oracle_workload(w, p=p)) <= RUN_TOL


@pytest.mark.parametrize("case", ["batch", "layers"])
def test_farfield_batched_and_layered(ms, case):
    """The far field on specimens of uneven sizes with start offsets (every
    specimen's own tiles, x-range and sources) and on two layers whose second
    one is rotated by 67 degrees (only the first layer's levels run along x):
    within 1e-5 of the direct sum's run and within the run tolerance of the
    oracle."""
    if case == "batch":
        a = wl.block_256(seed=11, dims=(256, 6, 4), n_tracks=3, n_steps=2500, T_thr=0.0)
        b = wl.block_256(seed=12, dims=(384, 4, 3), n_tracks=2, n_steps=2500, T_thr=0.0)
        b.specimens[0].source.t_offset = 3e-3
        w = wl.Workload("two_specimens", a.specimens + b.specimens, 2500, 1e-5, T_thr=0.0)
    else:
        w = wl.part_512(dims=(256, 12, 6), n_layers=2, tracks_per_layer=3, t_layer=1e-2,
                        hatch=4e-5)
    dist = 3e-3   # below the 4-range guard (5.08 mm at 10 um): the guard decides
    _, direct = gpu_workload(w, farfield_dist=0.0)
    ctx, far = gpu_workload(w, farfield_dist=dist)
    st = ctx.stats()
    assert st.farfield_node_evaluations > 0
    assert max_abs_diff(far, np.stack(direct)) <= 1e-5
    assert max_abs_diff(far, oracle_workload(w)) <= RUN_TOL
    check_sum(far)


def test_temperature_query_matches_the_source(ms):
    w = wl.block_256(dims=(30, 20, 5), n_tracks=2, n_steps=150, T_thr=0.0)
    sp = w.specimens[0]
    ctx, _ = gpu_workload(w)
    T = ctx.temperature()
    x, y, z = sp.grid.coords()
    To, _ = orc.temperature(sp.source, x, y, z, w.n_steps * w.dt)
    assert np.max(np.abs(T - To) / To) <= 2e-5


def test_kahan_compensated_parity(ms):
    """MS_KAHAN: double-float fractions, FP32 rates; as tight as FP64
    accumulation on the line."""
    w = wl.line_4096(n_points=1024, n_steps=2000)
    _, g = gpu_workload(w, precision=ms.MS_KAHAN)
    o = oracle_workload(w)
    assert max_abs_diff(g, o) <= 3e-5
    check_sum(g)


def test_graph_replay_is_bit_identical(ms):
    """MS_FLAG_GRAPH: the captured launch sequence (with the active set) gives
    the same bits as direct launches, on the first (capture) and a replayed
    pass, and counts the same launches."""
    from paper_2402_17580_gb300._binding import MS_FLAG_GRAPH, MS_FLAG_TIME_KERNELS
    w = wl.batch_64(n_specimens=4, n_lo=300, n_hi=3000, n_steps=500, T_thr=600.0)
    _, ref = gpu_workload(w, steps_per_launch=32)
    ctx = ms.Context(w.n_points, T_thr=w.T_thr, steps_per_launch=32,
                     flags=MS_FLAG_GRAPH | MS_FLAG_TIME_KERNELS)
    ctx.set_points([s.grid for s in w.specimens])
    for _ in range(2):
        ctx.fill_state(0.9, 0.0)
        ctx.run_track([s.source for s in w.specimens], w.n_steps, w.dt)
        g = ctx.fractions()
        for a, b in zip(ref, g):
            assert np.array_equal(a, b)
    st = ctx.stats()
    assert st.hot_kernel_launches == 2 * 16 and st.hot_kernel_ms > 0


def test_autotuner_picks_a_measured_configuration(ms):
    from paper_2402_17580_gb300.autotune import autotune
    w = wl.line_4096(n_points=2048, n_steps=400)
    res = autotune([s.grid for s in w.specimens], [s.source for s in w.specimens], w.n_points,
                   w.dt, trial_steps=256, repeats=1,
                   candidates={"steps_per_launch": (32, 128), "block_threads": (128,)})
    assert len(res.table) == 4 and res.ms == min(t for _, t in res.table) and res.ms > 0
    ctx = ms.Context(w.n_points, **res.params)
    ctx.set_points([s.grid for s in w.specimens])
    ctx.fill_state()
    ctx.run_track([s.source for s in w.specimens], w.n_steps, w.dt)
    _, dense = gpu_workload(w)
    for a, b in zip(dense, ctx.fractions()):
        assert np.array_equal(a, b)


def test_device_pointers_on_a_torch_stream(ms):
    """ms_step with device temperature arrays on the caller's stream."""
    torch = pytest.importorskip("torch")
    n = 1000
    xas, xam, T0, T1 = wl.random_states(n, seed=21)
    ctx = ms.Context(n)
    s = torch.cuda.Stream()
    ctx.set_stream(s.cuda_stream)
    ctx.set_state(xas, xam)
    t0 = torch.tensor(T0, dtype=torch.float32, device="cuda")
    t1 = torch.tensor(T1, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    ctx.step_device(t0.data_ptr(), t1.data_ptr(), 1e-4)
    g = ctx.fractions()
    ref = ms.Context(n)
    ref.set_state(xas, xam)
    ref.step(T0.astype(np.float32), T1.astype(np.float32), 1e-4)
    for a, b in zip(g, ref.fractions()):
        assert np.array_equal(a, b)
    ctx.set_stream(None)


# ------------------------------------------------------------ error paths
def test_error_paths(ms):
    ctx = ms.Context(10)
    with pytest.raises(ms.MSError) as e:
        ctx.set_state(np.full(10, np.nan), np.zeros(10))
    assert e.value.code == -5
    with pytest.raises(ms.MSError) as e:
        ctx.set_state(np.full(10, 0.6), np.full(10, 0.6))
    assert e.value.code == -1
    with pytest.raises(ms.MSError) as e:
        ctx.fractions()
    assert e.value.code == -6
    with pytest.raises(ms.MSError) as e:
        ctx.run_track([wl.line_4096().specimens[0].source], 1, 1e-5)
    assert e.value.code == -6
    with pytest.raises(ms.MSError) as e:
        ctx.step(np.zeros(10, np.float32), np.zeros(10, np.float32), -1.0)
    assert e.value.code == -1
    with pytest.raises(ms.MSError):
        ms.Context(10, precision=7)
    w = wl.line_4096(n_points=10)
    with pytest.raises(ms.MSError) as e:
        ctx.set_points([wl.Grid(dims=(11, 1, 1))])
    assert e.value.code == -1
    ctx.set_points([s.grid for s in w.specimens])
    bad = wl.HeatSource(np.array([[0, 0, 1.0, 1.0, 1.0, 200.0, 0.0, 0]]), w.specimens[0].source.layers)
    with pytest.raises(ms.MSError) as e:
        ctx.run_track([bad], 1, 1e-5)
    assert e.value.code == -1


def test_edge_cases(ms):
    """Degenerate and extreme inputs: zero steps, one point (a tile of 127
    padding lanes), the largest launch (512 steps), large explicit steps
    (invariants of P6 hold: every fraction in [0, 1], the sum 1)."""
    w = wl.line_4096(n_points=1, n_steps=300)
    ctx, g0 = gpu_workload(w, n_steps=0)
    assert np.allclose(np.stack(g0)[:2, 0], [0.9, 0.0])
    ctx, g = gpu_workload(w)
    assert max_abs_diff(g, oracle_workload(w)) <= RUN_TOL
    w = wl.line_4096(n_points=700, n_steps=1100)
    _, a = gpu_workload(w, steps_per_launch=512)
    _, b = gpu_workload(w, steps_per_launch=128)
    assert max_abs_diff(a, np.stack(b)) == 0.0
    xas, xam, T0, T1 = wl.random_states(4 * 128 + 3, seed=21)
    c = ms.Context(xas.size)
    c.set_state(xas, xam)
    for _ in range(20):
        c.step(T0.astype(np.float32), T1.astype(np.float32), 0.05)
    check_sum(c.fractions())


def test_verify_matches_host_reductions(ms):
    """ms_verify (device reductions) against the same reductions on the host:
    FP32 block against an MS_F64 subset context of the same grid."""
    w = wl.block_256(dims=(64, 64, 8), n_tracks=3, n_steps=600)
    ctx, g = gpu_workload(w)
    g = np.stack(g)
    idx = np.sort(np.random.default_rng(4).choice(w.n_points, 3000, replace=False))
    ref = ms.Context(idx.size, precision=ms.MS_F64, T_thr=0.0)
    ref.set_points_subset(w.specimens[0].grid, idx)
    ref.fill_state(w.init_xas, w.init_xam)
    ref.run_track([w.specimens[0].source], w.n_steps, w.dt)
    r = np.stack(ref.fractions())
    d, s1, s2 = ctx.verify(ref, idx)
    assert d == np.max(np.abs(g[:, idx] - r))
    assert abs(s1 - np.max(np.abs(g.sum(axis=0) - 1.0))) <= 1e-15
    assert abs(s2 - np.max(np.abs(r.sum(axis=0) - 1.0))) <= 1e-15
    assert 0 < d <= RUN_TOL and s1 <= SUM_TOL
    # without a map: a context against itself
    assert ctx.verify(ctx) == (0.0, s1, s1)
    with pytest.raises(ms.MSError, match="INVALID_ARG"):
        ctx.verify(ref, np.array([w.n_points], dtype=np.int64))
    ref.close()
    ctx.close()


# ------------------------------------------------ implicit scheme (Sec. 3)
IMPL_STEP_TOL = 1e-5   # one implicit step: FP32 rounding over the iterations and substeps


@pytest.mark.parametrize("dt", [1e-5, 1e-3, 0.05])
def test_implicit_single_step_every_branch(ms, dt):
    """MS_IMPLICIT through ms_step against the oracle's Crank-Nicolson step on
    random states and temperature pairs of every branch (dt = 0.05 s takes 5
    substeps of 0.01 s).  Both sides stop on the same WRMS rule; they can
    differ in the stop only when the norm lands within rounding of 1."""
    n = 6 * 128 + 37
    xas, xam, T0, T1 = wl.random_states(n, seed=91, block=1)
    T0, T1 = T0.astype(np.float32), T1.astype(np.float32)
    ctx = ms.Context(n, integrator=ms.MS_IMPLICIT)
    ctx.set_state(xas, xam)
    ctx.step(T0, T1, dt)
    g = ctx.fractions()
    st = ctx.stats()
    p = oracle_params(ctx.params)
    s = orc.State.make(oracle_view(xas), oracle_view(xam))
    orc.step(s, T0.astype(np.float64), T1.astype(np.float64), dt, p)
    o = orc.fractions(s, T1.astype(np.float64), p)
    assert max_abs_diff(g, np.stack(o)) <= IMPL_STEP_TOL
    check_sum(g)
    assert st.fp_iterations > 0 and st.fp_unconverged == 0


def test_implicit_line_run(ms):
    """The 4096-point line, 2000 steps, Crank-Nicolson in the hot kernel."""
    w = wl.line_4096()
    ctx, g = gpu_workload(w, integrator=1)
    p = oracle_params(ctx.params)
    assert max_abs_diff(g, oracle_workload(w, p=p)) <= RUN_TOL
    check_sum(g)
    st = ctx.stats()
    assert st.fp_iterations > 0 and st.fp_unconverged == 0


def test_implicit_full_fp64_path(ms):
    """MS_F64 with MS_IMPLICIT against the oracle on a small block."""
    w = wl.block_256(dims=(48, 16, 6), n_tracks=2, n_steps=900)
    ctx, g = gpu_workload(w, integrator=1, precision=ms.MS_F64)
    p = oracle_params(ctx.params)
    assert max_abs_diff(g, oracle_workload(w, p=p)) <= 1e-6


def test_implicit_cooldown_with_large_steps(ms):
    """The paper's use: cool-down steps of 0.05 s (5 substeps each) through
    ms_step with external temperatures, 40 steps on random histories."""
    n = 3 * 128 + 11
    rng = np.random.default_rng(5)
    xas, xam, _, _ = wl.random_states(n, seed=93, block=1)
    T = np.empty((41, n))
    T[0] = rng.uniform(900, 1500, n)
    for k in range(40):
        T[k + 1] = np.maximum(353.0, T[k] - rng.uniform(0, 40, n))
    T = T.astype(np.float32)
    ctx = ms.Context(n, integrator=ms.MS_IMPLICIT)
    ctx.set_state(xas, xam)
    for k in range(40):
        ctx.step(T[k], T[k + 1], 0.05)
    g = ctx.fractions()
    p = oracle_params(ctx.params)
    s = orc.State.make(oracle_view(xas), oracle_view(xam))
    orc.run_temps(s, T.astype(np.float64), 0.05, p)
    o = orc.fractions(s, T[-1].astype(np.float64), p)
    assert max_abs_diff(g, np.stack(o)) <= RUN_TOL
    assert ctx.stats().fp_unconverged == 0


def test_implicit_unsupported_combinations(ms):
    with pytest.raises(ms.MSError, match="UNSUPPORTED"):
        ms.Context(1000, integrator=ms.MS_IMPLICIT, precision=ms.MS_KAHAN)
    with pytest.raises(ms.MSError, match="INVALID_ARG"):
        ms.Context(1000, integrator=7)
    ctx = ms.Context(1000, integrator=ms.MS_IMPLICIT)
    s = ms.Surrogate(np.zeros(5187, dtype=np.float32))
    with pytest.raises(ms.MSError, match="UNSUPPORTED"):
        ctx.set_surrogate(s, 0.0)
    s.close()
    ctx.close()
