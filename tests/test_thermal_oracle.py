"""Pins of the FP64 thermal reference (oracle/thermal.py) on the CPU: energy
conservation of the finite volumes, the source's normalisation, diffusion of
a Gaussian bump against its closed form, radiative cooling against an ODE
solver, the running maximum r_c and the laser path."""
import math

import numpy as np
import pytest

from oracle import thermal as th


def _grid(n=(24, 20, 10), h=10e-6):
    return th.Grid3((0.0, 0.0, 0.0), (h, h, -h), n)


def test_finite_volumes_conserve_energy():
    """Adiabatic box, no cap, no radiation: the heat in the box grows by the
    source's energy exactly (to rounding), whatever the conductivity field."""
    p = th.ThermalParams(radiation=False, dirichlet_bottom=False, cap=False)
    g = _grid()
    rng = np.random.default_rng(1)
    T = 353.0 + 900.0 * rng.random((10, 20, 24))
    rc = rng.random((10, 20, 24))
    dx, dy, dz = 10e-6, 10e-6, 10e-6
    V = dx * dy * dz
    e0 = np.sum(p.rho * p.c * V * T)
    added = 0.0
    h = 2e-7
    for s in range(30):
        q = th.source_field(p, g, (120e-6 + 2e-6 * s, 100e-6, 150.0))
        added += h * np.sum(q) * V
        T, rc = th.substep(p, g, T, rc, q, h)
    e1 = np.sum(p.rho * p.c * V * T)
    assert abs((e1 - e0) - added) <= 1e-10 * e0


def test_source_integrates_to_the_effective_power():
    """eq:heat_soruce_cylindrical over the powder layer: sum q V = W_eff when
    the Gaussian is resolved (R / dx = 6) and h_p is a whole number of node
    layers."""
    p = th.ThermalParams()
    g = th.Grid3((-0.4e-3, -0.4e-3, 0.0), (10e-6, 10e-6, -10e-6), (81, 81, 6))
    q = th.source_field(p, g, (0.0, 0.0, 180.0))
    assert np.sum(q) * 1e-15 == pytest.approx(180.0, rel=1e-6)
    assert np.count_nonzero(q.reshape(6, -1).any(axis=1)) == 3   # 30 um of 10 um layers


def test_gaussian_bump_diffuses_like_the_closed_form():
    """Uniform k (all consolidated), no source: a Gaussian bump spreads as
    A (s0^2 / (s0^2 + 2 a t))^(3/2) exp(-r^2 / (2 (s0^2 + 2 a t))); the
    error falls by ~4 when the spacing halves (second order)."""
    p = th.ThermalParams(radiation=False, dirichlet_bottom=False, cap=False, k_p=28.6)
    a = p.k_ms / (p.rho * p.c)
    s0, A, t_end, L = 40e-6, 500.0, 2e-4, 200e-6
    errs = []
    for h in (20e-6, 10e-6):
        n = int(round(2 * L / h)) + 1
        g = th.Grid3((-L, -L, L), (h, h, -h), (n, n, n))
        X, Y, Z = np.meshgrid(g.x, g.y, g.z, indexing="xy")
        r2 = (X ** 2 + Y ** 2 + Z ** 2).transpose(2, 0, 1)
        T = p.T0 + A * np.exp(-r2 / (2 * s0 ** 2))
        rc = np.ones_like(T)
        steps = th.n_substeps(p, g.spacing, t_end) * 4
        for _ in range(steps):
            T, rc = th.substep(p, g, T, rc, 0.0, t_end / steps)
        s2 = s0 ** 2 + 2 * a * t_end
        exact = p.T0 + A * (s0 ** 2 / s2) ** 1.5 * np.exp(-r2 / (2 * s2))
        errs.append(np.max(np.abs(T - exact)))
    assert errs[1] < 0.02 * A
    assert 3.0 < errs[0] / errs[1] < 5.0, errs


def test_radiative_cooling_matches_the_ode():
    """A single layer of nodes at a uniform temperature loses
    eps sigma (T^4 - T_inf^4) per unit area: dT/dt = -that / (rho c |dz|);
    compared with an adaptive Runge-Kutta solution."""
    from scipy.integrate import solve_ivp
    p = th.ThermalParams(dirichlet_bottom=False, cap=False)
    g = th.Grid3((0.0, 0.0, 0.0), (10e-6, 10e-6, -10e-6), (4, 4, 1))
    T = np.full((1, 4, 4), 2500.0)
    rc = np.ones_like(T)
    t_end, n = 0.02, 2000
    for _ in range(n):
        T, rc = th.substep(p, g, T, rc, 0.0, t_end / n)
    f = lambda t, y: [-p.emissivity * th.SIGMA_SB * (y[0] ** 4 - p.T_inf ** 4) / (p.rho * p.c * 10e-6)]
    ref = solve_ivp(f, (0, t_end), [2500.0], rtol=1e-10, atol=1e-8).y[0, -1]
    assert np.allclose(T, ref, rtol=2e-4)
    assert T[0, 0, 0] < 2500.0


def test_consolidated_fraction_is_a_running_maximum():
    """eq:consolidated_fraction: powder melted once stays consolidated, and
    its conductivity becomes k_ms."""
    p = th.ThermalParams(radiation=False, dirichlet_bottom=False, cap=False)
    g = _grid((3, 3, 5))                           # 3 powder layers (30 um), 2 solid
    T, rc = th.initial_state(p, g)
    assert rc[:3].max() == 0.0 and rc[3:].min() == 1.0
    T[0] = 2000.0                                  # above T_l
    T, rc = th.substep(p, g, T, rc, 0.0, 1e-9)
    assert np.all(rc[0] == 1.0)
    T[0] = 400.0
    T, rc = th.substep(p, g, T, rc, 0.0, 1e-9)
    assert np.all(rc[0] == 1.0)
    assert np.all(th.conductivity(p, rc[0]) == p.k_ms)
    mid = th.liquid_fraction(p, np.array([1903.0]))[0]
    assert mid == pytest.approx(0.5)


def test_laser_path_follows_the_tracks():
    """On from a track's start to the next track's start (the last one to the
    layer's scan end), moving at v along u; off before and after."""
    tracks = np.array([[0.0, 0.0, 1.0, 0.0, 1.0, 180.0, 0.0, 0],
                       [1e-3, 1e-4, -1.0, 0.0, 1.0, 180.0, 1e-3, 0]])
    layers = np.array([[0.0, 0.0, 2e-3, 5e-3]])
    assert th.laser_position(tracks, layers, -1e-6) is None
    x, y, W = th.laser_position(tracks, layers, 0.5e-3)
    assert (x, y, W) == pytest.approx((0.5e-3, 0.0, 180.0))
    x, y, _ = th.laser_position(tracks, layers, 1.5e-3)
    assert (x, y) == pytest.approx((0.5e-3, 1e-4))
    assert th.laser_position(tracks, layers, 2e-3) is None
