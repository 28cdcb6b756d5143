"""FP64 reference of the grid thermal solver (test infrastructure only: tests/,
``__graft_entry__.smoke()`` and bench.py's baseline legs may import it; the
product never does).

The paper's thermal model (Sec. 2.1) is the heat equation
    rho c dT/dt = div(k grad T) + q_vol
with a conductivity that depends on the material state (eq:material_parameter_
interp): k = r_p k_p + r_m k_m + r_s k_s, where the consolidated fraction r_c
is the running maximum of the liquid fraction g(T) for initially powdery
material (eq:consolidated_fraction) and r_p = 1 - r_c, r_m = g(T),
r_s = r_c - g(T); with k_m = k_s = k_ms this is k = (1 - r_c) k_p + r_c k_ms.
The laser is the cylindrical volumetric source eq:heat_soruce_cylindrical,
q = 2 W / (pi R^2 h_p) exp(-2 (x^2 + y^2) / R^2) within the powder layer.

Discretisation written out here (the readings are listed in the design notes):

* one finite volume per grid node, V = dx dy |dz|; between neighbours the
  conductance G = k_f A / d with the harmonic mean k_f = 2 k_a k_b / (k_a + k_b)
  (0 when both are 0) and A the shared face, d the node distance;
* explicit Euler substeps, n = ceil(dt / (0.9 dt_stab)) with
  dt_stab = rho c / (k_ms (2/dx^2 + 2/dy^2 + 2/dz^2));
* in a substep from t: the source at t (the laser on track j from its start
  to the next track's start, the last track until the layer's scan end,
  position (x0, y0) + u v (t - t_start)); nodes within h_p below the top
  surface receive it;
* the top layer of nodes loses eps sigma (T^4 - T_inf^4) per unit area;
  the bottom layer is held at T0 (Dirichlet); the sides are adiabatic;
* after the update T is capped at T_max (the paper limits [T] at T_v + 1000 K)
  and r_c <- max(r_c, g(T)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SIGMA_SB = 5.670374419e-8   # Stefan-Boltzmann constant, W/(m^2 K^4)


@dataclass
class ThermalParams:
    """Table 1 (Ti-6Al-4V) and Table 5 (process) values by default."""
    rho: float = 4090.0
    c: float = 1130.0
    k_ms: float = 28.6
    k_p: float = 0.286
    T_s: float = 1878.0
    T_l: float = 1928.0
    T0: float = 353.0
    T_inf: float = 293.0
    emissivity: float = 0.7
    T_max: float = 4130.0
    beam_radius: float = 0.06e-3
    h_powder: float = 30e-6
    radiation: bool = True
    dirichlet_bottom: bool = True
    cap: bool = True


def liquid_fraction(p: ThermalParams, T):
    return np.clip((T - p.T_s) / (p.T_l - p.T_s), 0.0, 1.0)


def conductivity(p: ThermalParams, rc):
    return (1.0 - rc) * p.k_p + rc * p.k_ms


def n_substeps(p: ThermalParams, spacing, dt):
    dx, dy, dz = (abs(s) for s in spacing)
    dt_stab = p.rho * p.c / (p.k_ms * (2 / dx ** 2 + 2 / dy ** 2 + 2 / dz ** 2))
    return max(1, int(math.ceil(dt / (0.9 * dt_stab) - 1e-9)))


def laser_position(tracks, layers, t):
    """(x, y, W) of the laser at time t, or None when it is off.  tracks:
    rows x0, y0, ux, uy, v, P, t_start, layer (sorted by t_start per layer);
    layers: rows z_surface, t_begin, t_scan_end, t_end."""
    tracks = np.asarray(tracks, dtype=np.float64).reshape(-1, 8)
    layers = np.asarray(layers, dtype=np.float64).reshape(-1, 4)
    for j, tr in enumerate(tracks):
        lay = int(tr[7])
        t_end = layers[lay, 2]
        if j + 1 < len(tracks) and int(tracks[j + 1, 7]) == lay:
            t_end = tracks[j + 1, 6]
        if tr[6] <= t < t_end:
            d = tr[4] * (t - tr[6])
            return tr[0] + tr[2] * d, tr[1] + tr[3] * d, tr[5]
    return None


class Grid3:
    """Node coordinates of an (nx, ny, nz) grid; arrays are [k, j, i]."""

    def __init__(self, origin, spacing, dims):
        self.origin, self.spacing, self.dims = origin, spacing, dims
        nx, ny, nz = dims
        ox, oy, oz = origin
        dx, dy, dz = spacing
        self.x = ox + dx * np.arange(nx)
        self.y = oy + dy * np.arange(ny)
        self.z = oz + dz * np.arange(nz)
        self.top = int(np.argmax(self.z))
        self.bottom = int(np.argmin(self.z))


def source_field(p: ThermalParams, g: Grid3, pos):
    """q_vol [W/m^3] on the grid for the laser at pos = (x, y, W) or None."""
    nx, ny, nz = g.dims
    q = np.zeros((nz, ny, nx))
    if pos is None:
        return q
    sx, sy, W = pos
    r2 = (g.x[None, :] - sx) ** 2 + (g.y[:, None] - sy) ** 2
    plane = 2.0 * W / (math.pi * p.beam_radius ** 2 * p.h_powder) * np.exp(-2.0 * r2 / p.beam_radius ** 2)
    depth = g.z[g.top] - g.z
    inside = (depth >= 0.0) & (depth < p.h_powder)
    q[inside] = plane
    return q


def substep(p: ThermalParams, g: Grid3, T, rc, q, h):
    """One explicit Euler substep of length h; returns (T', rc')."""
    dx, dy, dz = (abs(s) for s in g.spacing)
    k = conductivity(p, rc)

    def harm(a, b):
        s = a + b
        return np.where(s > 0.0, 2.0 * a * b / np.where(s > 0.0, s, 1.0), 0.0)

    flux = np.zeros_like(T)                      # W into each node
    # x faces
    kf = harm(k[:, :, 1:], k[:, :, :-1])
    f = kf * (dy * dz / dx) * (T[:, :, 1:] - T[:, :, :-1])
    flux[:, :, :-1] += f
    flux[:, :, 1:] -= f
    # y faces
    kf = harm(k[:, 1:, :], k[:, :-1, :])
    f = kf * (dx * dz / dy) * (T[:, 1:, :] - T[:, :-1, :])
    flux[:, :-1, :] += f
    flux[:, 1:, :] -= f
    # z faces
    kf = harm(k[1:, :, :], k[:-1, :, :])
    f = kf * (dx * dy / dz) * (T[1:, :, :] - T[:-1, :, :])
    flux[:-1, :, :] += f
    flux[1:, :, :] -= f
    V = dx * dy * dz
    flux += q * V
    if p.radiation:
        Tt = T[g.top]
        flux[g.top] -= p.emissivity * SIGMA_SB * (Tt ** 4 - p.T_inf ** 4) * dx * dy
    Tn = T + h * flux / (p.rho * p.c * V)
    if p.dirichlet_bottom:
        Tn[g.bottom] = p.T0
    if p.cap:
        Tn = np.minimum(Tn, p.T_max)
    rcn = np.maximum(rc, liquid_fraction(p, Tn))
    return Tn, rcn


def initial_state(p: ThermalParams, g: Grid3):
    """T = T0 everywhere; r_c = 0 (powder) within h_p of the top surface,
    1 below."""
    nx, ny, nz = g.dims
    T = np.full((nz, ny, nx), p.T0)
    depth = g.z[g.top] - g.z
    rc = np.ones((nz, ny, nx))
    rc[(depth >= 0.0) & (depth < p.h_powder)] = 0.0
    return T, rc


def step(p: ThermalParams, g: Grid3, T, rc, tracks, layers, t, dt):
    """Advance from t to t + dt with the substeps of n_substeps."""
    n = n_substeps(p, g.spacing, dt)
    h = dt / n
    for s in range(n):
        ts = t + s * h
        q = source_field(p, g, laser_position(tracks, layers, ts))
        T, rc = substep(p, g, T, rc, q, h)
    return T, rc
