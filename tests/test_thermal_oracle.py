"""Pins of the FP64 thermal reference (oracle/thermal.py) on the CPU: energy
conservation of the finite volumes, the source's normalisation, diffusion of
a Gaussian bump against its closed form, radiative cooling against an ODE
solver, the running maximum r_c, the laser path, the face conductance of two
materials in series, the discrete eigenmodes of each axis (Dirichlet bottom,
adiabatic sides and top), radiative equilibrium, the T_max cap, the maximum
principle of step() and the time at which it takes the source."""
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
    # a node exactly at depth h_p is below the layer (depth in [0, h_p)): with
    # binary spacings the boundary is exact and 2 node layers carry W
    p2 = th.ThermalParams(h_powder=2.0 ** -15)
    g2 = th.Grid3((-0.4e-3, -0.4e-3, 0.0), (10e-6, 10e-6, -2.0 ** -16), (81, 81, 6))
    q2 = th.source_field(p2, g2, (0.0, 0.0, 180.0))
    assert np.sum(q2) * 1e-10 * 2.0 ** -16 == pytest.approx(180.0, rel=1e-6)
    assert np.count_nonzero(q2.reshape(6, -1).any(axis=1)) == 2


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


def test_face_conductance_is_two_half_cells_in_series():
    """Two volumes of different conductivity side by side: by Fourier's law
    the heat crossing their common face per unit time is the temperature
    difference over the series resistance of the two half-cells,
    (d / 2) / (k_a A) + (d / 2) / (k_b A); one explicit substep moves exactly
    h times that (in both directions of each axis)."""
    p = th.ThermalParams(radiation=False, dirichlet_bottom=False, cap=False)
    dx, dy, dz = 20e-6, 15e-6, 10e-6
    for axis in range(3):
        dims = [1, 1, 1]
        dims[axis] = 2
        g = th.Grid3((0.0, 0.0, 0.0), (dx, dy, -dz), tuple(dims))
        shape = (dims[2], dims[1], dims[0])
        d = (dx, dy, dz)[axis]
        A = dx * dy * dz / d
        rc = np.array([1.0, 0.0]).reshape(shape)       # k_ms | k_p
        T = np.array([1500.0, 400.0]).reshape(shape)
        h = 1e-9
        T1, _ = th.substep(p, g, T, rc, 0.0, h)
        q = (1500.0 - 400.0) / ((d / 2) / (p.k_ms * A) + (d / 2) / (p.k_p * A))
        moved = p.rho * p.c * dx * dy * dz * (T.ravel() - T1.ravel())
        assert moved[0] == pytest.approx(h * q, rel=1e-12), axis
        assert moved[1] == pytest.approx(-h * q, rel=1e-12), axis


def _mode_decay(p, g, T0_field, n, h):
    rc = np.ones_like(T0_field)
    T = T0_field.copy()
    for _ in range(n):
        T, rc = th.substep(p, g, T, rc, 0.0, h)
    return T


def test_discrete_eigenmodes_decay_at_their_closed_form_rates():
    """Explicit Euler on the finite volumes is linear; its eigenvectors on a
    row of n volumes are known in closed form.  With adiabatic ends (x, y)
    the mode cos(theta (i + 1/2)), theta = m pi / n, and with the bottom held
    at T0 and an adiabatic top (z, bottom node j = 0) the mode
    sin(theta j), theta = (2m + 1) pi / (2n - 1), are each multiplied per
    substep by 1 - 4 a h sin^2(theta / 2) / d^2, a = k / (rho c).  This fixes
    every face's area over distance on a non-cubic grid, the Dirichlet bottom
    and the adiabatic top."""
    p = th.ThermalParams(radiation=False, cap=False)
    sp = (20e-6, 15e-6, 10e-6)
    a = p.k_ms / (p.rho * p.c)
    n, A, steps = 12, 200.0, 400
    for axis in range(3):
        dims = [1, 1, 1]
        dims[axis] = n
        g = th.Grid3((0.0, 0.0, 0.0), (sp[0], sp[1], -sp[2]), tuple(dims))
        d = sp[axis]
        h = 0.3 * d * d / (4 * a)                   # stable for a single axis
        shape = (dims[2], dims[1], dims[0])
        i = np.arange(n)
        for m in (1, 3):
            if axis < 2:
                pq = th.ThermalParams(radiation=False, cap=False, dirichlet_bottom=False)
                theta = m * np.pi / n
                v = np.cos(theta * (i + 0.5))
            else:
                pq = p
                theta = (2 * m + 1) * np.pi / (2 * n - 1)
                j = (n - 1) - i                     # z[0] is the top, z[n - 1] the bottom
                v = np.sin(theta * j)
            T = _mode_decay(pq, g, (p.T0 + A * v).reshape(shape), steps, h)
            lam = (1.0 - 4.0 * a * h * np.sin(theta / 2) ** 2 / d ** 2) ** steps
            np.testing.assert_allclose(T.ravel() - p.T0, lam * A * v, rtol=0, atol=1e-9 * A)
            assert lam < 0.9, (axis, m)


def test_radiation_vanishes_at_the_ambient_temperature():
    """The top surface exchanges eps sigma (T^4 - T_inf^4): a surface at T_inf
    stays there exactly, one below it warms, one above it cools; in a uniform
    column only the top layer changes in the first substep."""
    p = th.ThermalParams(dirichlet_bottom=False, cap=False)
    g = th.Grid3((0.0, 0.0, 0.0), (10e-6, 10e-6, -10e-6), (2, 2, 3))
    for T_start, sign in ((p.T_inf, 0), (250.0, 1), (400.0, -1)):
        T = np.full((3, 2, 2), T_start)
        T1, _ = th.substep(p, g, T, np.ones_like(T), 0.0, 1e-6)
        assert np.all(np.sign(T1[0] - T[0]) == sign), T_start
        assert np.array_equal(T1[1:], T[1:]), T_start


def test_temperature_is_capped_at_T_max():
    """Sec. 2.1 limits the temperature at T_v + 1000 K = 4130 K: under a
    source strong enough to pass it in one substep the hottest nodes sit at
    exactly T_max and none above."""
    p = th.ThermalParams(radiation=False, dirichlet_bottom=False)
    g = _grid((9, 9, 4))
    T, rc = th.initial_state(p, g)
    q = th.source_field(p, g, (40e-6, 40e-6, 5000.0))
    T1, rc1 = th.substep(p, g, T, rc, q, 1e-5)
    assert T1.max() == p.T_max
    assert np.count_nonzero(T1 == p.T_max) >= 3
    assert np.all(rc1[T1 == p.T_max] == 1.0)


def test_step_keeps_the_maximum_principle():
    """Below the explicit scheme's stability limit every node's new value is
    a convex combination of its own and its neighbours' old values, so with
    no source, radiation or boundary value the minimum never falls and the
    maximum never rises, whatever the conductivity field; step() picks its
    substeps to stay below that limit, h <= rho c / (k_max sum 2 / d^2)."""
    p = th.ThermalParams(radiation=False, dirichlet_bottom=False, cap=False)
    g = th.Grid3((0.0, 0.0, 0.0), (20e-6, 15e-6, -10e-6), (9, 8, 7))
    rng = np.random.default_rng(5)
    T = 353.0 + 1500.0 * (rng.random((7, 8, 9)) > 0.5)      # a rough field
    rc = np.ones_like(T)
    dt = 2e-5
    n = th.n_substeps(p, g.spacing, dt)
    limit = p.rho * p.c / (p.k_ms * (2 / 20e-6 ** 2 + 2 / 15e-6 ** 2 + 2 / 10e-6 ** 2))
    assert dt / n <= limit and dt / (n - 1) > 0.9 * limit
    lo, hi = T.min(), T.max()
    for _ in range(3):
        T, rc = th.step(p, g, T, rc, np.zeros((0, 8)), np.zeros((0, 4)), 0.0, dt)
        assert T.min() >= lo - 1e-9 and T.max() <= hi + 1e-9
        lo, hi = T.min(), T.max()
    assert hi - lo < 1500.0


def test_step_evaluates_the_source_at_each_substep_start():
    """Explicit Euler takes the source at the start of each substep: a step
    that ends the moment the laser turns on adds no heat, and the step that
    starts then adds P dt (the Gaussian resolved, the layer whole)."""
    p = th.ThermalParams(radiation=False, dirichlet_bottom=False, cap=False)
    g = th.Grid3((-0.3e-3, -0.3e-3, 0.0), (10e-6, 10e-6, -10e-6), (61, 61, 5))
    tracks = np.array([[0.0, 0.0, 1.0, 0.0, 0.0, 150.0, 1e-6, 0]])    # v = 0: stays put
    layers = np.array([[0.0, 0.0, 1.0, 1.0]])
    T, rc = th.initial_state(p, g)
    V = 1e-15
    T1, rc1 = th.step(p, g, T, rc, tracks, layers, 0.0, 1e-6)
    assert np.array_equal(T1, T)
    T2, _ = th.step(p, g, T1, rc1, tracks, layers, 1e-6, 1e-6)
    e = p.rho * p.c * V * (T2 - T1).sum()
    assert e == pytest.approx(150.0 * 1e-6, rel=1e-6)
