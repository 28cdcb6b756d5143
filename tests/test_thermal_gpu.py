"""GPU tests of the grid thermal solver and of its coupling to the phase model.

Tolerances.  The solver runs in FP32: one substep rounds each node's update
to ~6e-8 relative (2.5e-4 K at the 4130 K cap); diffusion damps these
errors, so after a few hundred substeps the field is held to 0.1 K of the
FP64 reference, and r_c (the running maximum of (T - T_s) / 50 K) to 0.1/50 =
2e-3.  The coupling is checked apart from that: the phase model's oracle is
driven by the GPU's own temperature history, so the coupled run is held to
the phase model's run tolerance (1e-4)."""
import numpy as np
import pytest

import oracle as orc
from oracle import thermal as oth
import workloads as wl
from tests._util import max_abs_diff, oracle_params

pytestmark = pytest.mark.gpu

T_TOL = 0.1
RC_TOL = 2e-3
RUN_TOL = 1e-4


@pytest.fixture(scope="module")
def ms():
    import paper_2402_17580_gb300 as m
    m.load()
    return m


def _case(nx=40, ny=24, nz=12):
    grid = wl.Grid((0.0, 0.0, 0.0), (1e-5, 1e-5, -1e-5), (nx, ny, nz))
    # one track along x through the middle, then the laser is off
    tracks = np.array([[0.0, 120e-6, 1.0, 0.0, 1.0, 180.0, 0.0, 0]])
    layers = np.array([[0.0, 0.0, 0.39e-3, 1.0]])
    src = wl.HeatSource(tracks, layers)
    return grid, src


def _oracle_params(tp):
    return oth.ThermalParams(rho=tp.rho, c=tp.c, k_ms=tp.k_ms, k_p=tp.k_p, T_s=tp.T_s, T_l=tp.T_l,
                             T0=tp.T0, T_inf=tp.T_inf, emissivity=tp.emissivity, T_max=tp.T_max,
                             beam_radius=tp.beam_radius, h_powder=tp.h_powder,
                             radiation=bool(tp.radiation), dirichlet_bottom=bool(tp.dirichlet_bottom),
                             cap=bool(tp.cap))


def _oracle_run(grid, src, tp, n_steps, dt):
    g = oth.Grid3(grid.origin, grid.spacing, grid.dims)
    p = _oracle_params(tp)
    T, rc = oth.initial_state(p, g)
    for s in range(n_steps):
        T, rc = oth.step(p, g, T, rc, src.tracks, src.layers, s * dt, dt)
    return T.ravel(), rc.ravel()


@pytest.mark.parametrize("n_steps", [20, 120])
def test_thermal_matches_the_oracle(ms, n_steps):
    """The laser crossing the grid (20 steps: under the beam; 120: cooling
    after the track) with powder, radiation, Dirichlet bottom and the cap."""
    grid, src = _case()
    th = ms.Thermal(grid)
    th.set_source(src)
    for _ in range(n_steps):
        th.step(1e-5)
    T, rc = th.get()
    To, rco = _oracle_run(grid, src, th.params, n_steps, 1e-5)
    assert rco.reshape(grid.dims[::-1])[0].max() == 1.0   # the laser melted powder
    assert np.max(np.abs(T - To)) <= T_TOL
    assert np.max(np.abs(rc - rco)) <= RC_TOL
    st = th.stats()
    assert st["substeps"] == n_steps * oth.n_substeps(_oracle_params(th.params), grid.spacing, 1e-5)
    th.close()


def test_thermal_energy_balance(ms):
    """Adiabatic box, no radiation, no cap: the heat gained equals the laser's
    energy W t (FP32 sums: 1e-4)."""
    grid, src = _case(40, 24, 16)
    tp = ms.thermal_params(radiation=0, dirichlet_bottom=0, cap=0)
    th = ms.Thermal(grid, tp)
    th.set_source(src)
    for _ in range(20):
        th.step(1e-5)
    T, _ = th.get()
    V = 1e-15
    gained = np.sum(tp.rho * tp.c * V * (T - tp.T0))
    g = oth.Grid3(grid.origin, grid.spacing, grid.dims)
    p = _oracle_params(tp)
    h = 1e-5 / oth.n_substeps(p, grid.spacing, 1e-5)
    n = int(round(20 * 1e-5 / h))
    expect = sum(h * np.sum(oth.source_field(p, g, oth.laser_position(src.tracks, src.layers, s * h))) * V
                 for s in range(n))
    assert gained == pytest.approx(expect, rel=1e-4)
    th.close()


def test_coupled_run_matches_the_phase_oracle(ms):
    """ms_thermal_run_coupled one step at a time: the phase model on the
    device against the oracle driven by the same temperature history."""
    grid, src = _case()
    n = grid.n
    th = ms.Thermal(grid)
    th.set_source(src)
    ctx = ms.Context(n)
    ctx.set_state(np.full(n, 0.9), np.zeros(n))
    ctx.set_stream(None)
    hist = [np.full(n, th.params.T0)]
    for _ in range(150):
        th.run_coupled(ctx, 1, 1e-5)
        hist.append(th.get()[0].astype(np.float32).astype(np.float64))
    g = ctx.fractions()
    s = orc.State.uniform(n, 0.9, 0.0)
    p = oracle_params()
    orc.run_temps(s, np.stack(hist), 1e-5, p)
    o = np.stack(orc.fractions(s, hist[-1], p))
    assert max_abs_diff(g, o) <= RUN_TOL
    assert np.stack(g)[1].max() > 0.1                  # martensite formed behind the pool
    th.close()
    ctx.close()


def test_coupled_many_steps_without_sync(ms):
    """The same coupled run in one call (no host round trip per step) ends in
    the same state as the step-by-step run."""
    grid, src = _case()
    n = grid.n
    out = []
    for chunks in (1, 150):
        th = ms.Thermal(grid)
        th.set_source(src)
        ctx = ms.Context(n)
        ctx.fill_state(0.9, 0.0)
        for _ in range(chunks):
            th.run_coupled(ctx, 150 // chunks, 1e-5)
        out.append(np.stack(ctx.fractions()))
        th.close()
        ctx.close()
    np.testing.assert_array_equal(out[0], out[1])


def test_thermal_errors(ms):
    grid, src = _case()
    with pytest.raises(ms.MSError, match="INVALID_ARG"):
        ms.Thermal(grid, rho=-1.0)
    th = ms.Thermal(grid)
    ctx = ms.Context(grid.n + 1)
    with pytest.raises(ms.MSError, match="INVALID_ARG"):
        th.run_coupled(ctx, 1, 1e-5)
    with pytest.raises(ms.MSError, match="INVALID_ARG"):
        th.step(-1.0)
    unsorted = wl.HeatSource(np.array([[0.0, 0.0, 1.0, 0.0, 1.0, 180.0, 2e-4, 0],
                                       [0.0, 1e-4, 1.0, 0.0, 1.0, 180.0, 1e-4, 0]]), src.layers)
    with pytest.raises(ms.MSError, match="INVALID_ARG"):
        th.set_source(unsorted)
    th.close()
    ctx.close()
