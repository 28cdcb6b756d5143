"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This module holds NO arithmetic of the phase model or of the temperature
formula: it only lays out grids, scan tracks (start points, directions,
speeds, powers, start times) and random initial states.  Both the CUDA path
and the oracle receive its outputs as plain inputs.

Workloads (the paper's FEM part data is not available; these synthetic,
Rosenthal-driven inputs take the paper's process scales, Tables 5 and 6:
v ~ 1 m/s, P ~ 200 W, hatch 80-120 um, layer 30 um):

* ``line_4096``   4096 points on a line (10 um spacing) at depth 0, one track
                  along it (P = 200 W, v = 1 m/s), 2000 steps of 1e-5 s.
* ``block_256``   256 x 256 x 64 block at 10 um spacing, 20 serpentine tracks
                  along x with hatch 100 um, P ~ U(150, 250) W, v ~ U(0.8, 1.2)
                  m/s drawn from the seed, 20000 steps of 1e-5 s.
* ``batch_64``    64 specimens, point counts log-uniform in [1e4, 2e6]
                  (nx = ny = round(sqrt(n / 16)), nz = 16), each with its own
                  P ~ U(150, 300) W, v ~ U(0.5, 1.5) m/s, hatch ~ U(80, 120) um
                  and start-time offset ~ U(0, 5 ms), 10000 steps.
* ``part_512``    512 x 512 x 256 block, 5 layers of 30 um, 50 serpentine
                  tracks per layer (P = 200 W, v = 1 m/s, hatch 100 um),
                  rotated by 67 degrees per layer, 0.5 s per layer (scan, then
                  linear interlayer cool-down to T0).

* ``surrogate_lines``  training histories of the window surrogate: short
                  serpentines over lines at random depth and lateral offset.

Seeds default to 2402175800 + the workload number (1 .. 5).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2402175800

# material / source constants of the synthetic driver (Ti-6Al-4V half-space)
ABSORPTIVITY = 0.35
CONDUCTIVITY = 7.0         # W/(m K)
DIFFUSIVITY = 3e-6         # m^2/s
T_PREHEAT = 353.0          # K
T_MAX = 3130.0 + 1000.0    # K, boiling temperature + 1000 K (Sec. 2.1)
NEVER = 1e30               # "no end" time


@dataclass
class Grid:
    """Points x = ox + i*dx, y = oy + j*dy, z = oz + (k + k_offset)*dz; i
    fastest.  k_offset > 0: the z-planes k_offset .. k_offset + nz - 1 of a
    larger grid with the same origin and spacing (a z-slab shard)."""
    origin: tuple = (0.0, 0.0, 0.0)
    spacing: tuple = (1e-5, 1e-5, -1e-5)
    dims: tuple = (1, 1, 1)
    k_offset: int = 0

    @property
    def n(self) -> int:
        nx, ny, nz = self.dims
        return nx * ny * nz

    def ijk(self, idx):
        idx = np.asarray(idx, dtype=np.int64)
        nx, ny, _ = self.dims
        return idx % nx, (idx // nx) % ny, idx // (nx * ny)

    def coords(self, idx=None):
        """Coordinates (float64) of the points with natural indices ``idx``."""
        if idx is None:
            idx = np.arange(self.n, dtype=np.int64)
        i, j, k = self.ijk(idx)
        ox, oy, oz = self.origin
        dx, dy, dz = self.spacing
        return ox + i * dx, oy + j * dy, oz + (k + self.k_offset) * dz


@dataclass
class HeatSource:
    """Superposed moving point sources.

    tracks: (n, 8) float64 rows  x0, y0, ux, uy, v, P, t_start, layer
    layers: (m, 4) float64 rows  z_surface, t_begin, t_scan_end, t_end
    """
    tracks: np.ndarray
    layers: np.ndarray
    A: float = ABSORPTIVITY
    k: float = CONDUCTIVITY
    alpha: float = DIFFUSIVITY
    T0: float = T_PREHEAT
    T_max: float = T_MAX
    t_offset: float = 0.0
    z_tol: float = 5e-6


@dataclass
class Specimen:
    grid: Grid
    source: HeatSource


@dataclass
class Workload:
    name: str
    specimens: list
    n_steps: int
    dt: float
    T_thr: float = 0.0
    init_xas: float = 0.9   # room-temperature equilibrium (0.9, 0, 0.1), App. A
    init_xam: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def n_points(self) -> int:
        return sum(s.grid.n for s in self.specimens)

    @property
    def point_updates(self) -> int:
        return self.n_points * self.n_steps


def _one_layer(t_begin=0.0):
    return np.array([[0.0, t_begin, NEVER, NEVER]])


def serpentine_x(y_lines, x_lo, x_hi, v, P, t0=0.0, layer=0):
    """Serpentine tracks along x between x_lo and x_hi at the given y values;
    track j+1 starts where and when track j ends (no jump time)."""
    rows, t = [], t0
    length = x_hi - x_lo
    for j, y in enumerate(y_lines):
        fwd = j % 2 == 0
        x0, ux = (x_lo, 1.0) if fwd else (x_hi, -1.0)
        rows.append([x0, y, ux, 0.0, v[j], P[j], t, layer])
        t += length / v[j]
    return np.array(rows, dtype=np.float64), t


def line_4096(n_points=4096, n_steps=2000, dt=1e-5) -> Workload:
    grid = Grid((0.0, 0.0, 0.0), (1e-5, 1e-5, -1e-5), (n_points, 1, 1))
    tracks = np.array([[0.0, 0.0, 1.0, 0.0, 1.0, 200.0, 0.0, 0]], dtype=np.float64)
    src = HeatSource(tracks, _one_layer())
    return Workload("line_4096", [Specimen(grid, src)], n_steps, dt, T_thr=0.0)


def block_256(seed=None, dims=(256, 256, 64), n_tracks=20, n_steps=20000, dt=1e-5,
              T_thr=600.0) -> Workload:
    seed = SEED_BASE + 2 if seed is None else seed
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    P = rng.uniform(150.0, 250.0, n_tracks)
    v = rng.uniform(0.8, 1.2, n_tracks)
    width = (ny - 1) * 1e-5
    hatch = 1e-4
    y0 = 0.5 * (width - (n_tracks - 1) * hatch)
    tracks, t_end = serpentine_x([y0 + j * hatch for j in range(n_tracks)], 0.0,
                                 (nx - 1) * 1e-5, v, P)
    grid = Grid((0.0, 0.0, 0.0), (1e-5, 1e-5, -1e-5), dims)
    w = Workload("block_256", [Specimen(grid, HeatSource(tracks, _one_layer()))], n_steps, dt,
                 T_thr=T_thr)
    w.meta.update(seed=seed, scan_end_s=t_end)
    return w


def batch_64(seed=None, n_specimens=64, n_lo=1e4, n_hi=2e6, n_steps=10000, dt=1e-5,
             T_thr=600.0) -> Workload:
    seed = SEED_BASE + 3 if seed is None else seed
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(n_specimens):
        n_s = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        nxy = max(4, int(round(math.sqrt(n_s / 16.0))))
        P = rng.uniform(150.0, 300.0)
        v = rng.uniform(0.5, 1.5)
        hatch = rng.uniform(80e-6, 120e-6)
        offset = rng.uniform(0.0, 5e-3)
        width = (nxy - 1) * 1e-5
        n_tr = max(1, int(width // hatch))
        ys = [0.5 * (width - (n_tr - 1) * hatch) + j * hatch for j in range(n_tr)]
        tracks, _ = serpentine_x(ys, 0.0, width, [v] * n_tr, [P] * n_tr)
        src = HeatSource(tracks, _one_layer(), t_offset=offset)
        specs.append(Specimen(Grid((0.0, 0.0, 0.0), (1e-5, 1e-5, -1e-5), (nxy, nxy, 16)), src))
    w = Workload("batch_64", specs, n_steps, dt, T_thr=T_thr)
    w.meta.update(seed=seed)
    return w


def _clip_line(c, d, half):
    """Parameter range of the line c + s d inside the square |x - c0| <= half."""
    lo, hi = -np.inf, np.inf
    for a in range(2):
        if abs(d[a]) < 1e-15:
            if abs(c[a]) > half:
                return None
            continue
        s1, s2 = (-half - c[a]) / d[a], (half - c[a]) / d[a]
        lo, hi = max(lo, min(s1, s2)), min(hi, max(s1, s2))
    return (lo, hi) if hi > lo else None


def part_512(dims=(512, 512, 256), n_layers=5, layer_t=30e-6, tracks_per_layer=50,
             hatch=1e-4, P=200.0, v=1.0, rot_deg=67.0, t_layer=0.5, dt=1e-5,
             T_thr=600.0) -> Workload:
    nx, ny, nz = dims
    L = (nx - 1) * 1e-5
    cx = cy = 0.5 * L
    half = 0.5 * L
    rows, layers = [], []
    for l in range(n_layers):
        th = math.radians(rot_deg * l)
        d = np.array([math.cos(th), math.sin(th)])
        nrm = np.array([-d[1], d[0]])
        t = l * t_layer
        t_begin = t
        k = 0
        for j in range(tracks_per_layer):
            off = (j - 0.5 * (tracks_per_layer - 1)) * hatch
            c = off * nrm
            seg = _clip_line(c, d, half)
            if seg is None:
                continue
            lo, hi = seg
            fwd = k % 2 == 0
            k += 1
            s0 = lo if fwd else hi
            u = d if fwd else -d
            x0, y0 = cx + c[0] + s0 * d[0], cy + c[1] + s0 * d[1]
            rows.append([x0, y0, u[0], u[1], v, P, t, l])
            t += (hi - lo) / v
        z_surf = -(n_layers - 1 - l) * layer_t
        layers.append([z_surf, t_begin, t, (l + 1) * t_layer])
    src = HeatSource(np.array(rows), np.array(layers))
    n_steps = int(round(n_layers * t_layer / dt))
    grid = Grid((0.0, 0.0, 0.0), (1e-5, 1e-5, -1e-5), dims)
    return Workload("part_512", [Specimen(grid, src)], n_steps, dt, T_thr=T_thr)


# ------------------------------------------------------------ random states
# Temperature bands that separate the branches of the model (K): below T_inf,
# martensite range, alpha_s plateau, equilibrium curve, regularisation band,
# beta range, mushy zone, melt.
T_BANDS = ((250.0, 293.0), (293.0, 848.0), (848.0, 935.0), (935.0, 1273.0),
           (1273.0, 1373.0), (1373.0, 1878.0), (1878.0, 1928.0), (1928.0, 2600.0))


def surrogate_lines(seed=None, n_lines=128, n_points=512, n_tracks=3, hatch=1e-4,
                    n_steps=2800, dt=1e-5) -> Workload:
    """Training histories of the window surrogate: n_lines specimens, each a
    line of n_points along x (10 um spacing) at a seeded depth U(0, 100) um
    and lateral offset U(0, (n_tracks - 1) hatch + 100 um), under a short
    serpentine of n_tracks tracks along the line with its own P ~ U(150, 250)
    W and v ~ U(0.8, 1.2) m/s, so the lines see single passes, reheating by
    the neighbouring tracks and the receding-source cooling tail."""
    seed = SEED_BASE + 4 if seed is None else seed
    rng = np.random.default_rng(seed)
    length = (n_points - 1) * 1e-5
    specs = []
    for _ in range(n_lines):
        P = rng.uniform(150.0, 250.0, n_tracks)
        v = rng.uniform(0.8, 1.2, n_tracks)
        depth = rng.uniform(0.0, 1e-4)
        y = rng.uniform(0.0, (n_tracks - 1) * hatch + 1e-4)
        tracks, _ = serpentine_x([j * hatch for j in range(n_tracks)], 0.0, length, v, P)
        grid = Grid((0.0, y, -depth), (1e-5, 1e-5, -1e-5), (n_points, 1, 1))
        specs.append(Specimen(grid, HeatSource(tracks, _one_layer())))
    w = Workload("surrogate_lines", specs, n_steps, dt, T_thr=0.0)
    w.meta.update(seed=seed)
    return w


def random_states(n, seed, block=1, edge_frac=0.15):
    """Random (X_as, X_am, T0, T1) covering every branch region.

    Points come in blocks of ``block`` identical branch choices (the paper's
    synthetic layouts use blocks of 1, 10 and 100).  States satisfy
    X_as + X_am <= 0.9 and avoid 0 < 0.9 - X_alpha < 1e-5 (ill-conditioned in
    FP32: the onset of alpha_s -> beta dissolution scales with that gap to the
    power 1/c_beta).  A fraction ``edge_frac`` sits exactly on the special
    values 0 and 0.9 that select the App. A initiations."""
    rng = np.random.default_rng(seed)
    nb = (n + block - 1) // block
    band0 = rng.integers(0, len(T_BANDS), nb)
    band1 = np.clip(band0 + rng.integers(-1, 2, nb), 0, len(T_BANDS) - 1)
    kind = rng.integers(0, 6, nb)
    rep = lambda a: np.repeat(a, block)[:n]
    b0, b1, kd = rep(band0), rep(band1), rep(kind)
    lo0 = np.array([T_BANDS[b][0] for b in b0]); hi0 = np.array([T_BANDS[b][1] for b in b0])
    lo1 = np.array([T_BANDS[b][0] for b in b1]); hi1 = np.array([T_BANDS[b][1] for b in b1])
    T0 = lo0 + (hi0 - lo0) * rng.random(n)
    T1 = lo1 + (hi1 - lo1) * rng.random(n)
    xa = 0.9 * rng.random(n)
    frac = rng.random(n)
    xas = xa * frac
    xam = xa - xas
    # special states: pure beta, room-temperature equilibrium, alpha_s only, alpha_m only
    edge = rng.random(n) < edge_frac
    xas = np.where(edge & (kd == 0), 0.0, xas); xam = np.where(edge & (kd == 0), 0.0, xam)
    xas = np.where(edge & (kd == 1), 0.9, xas); xam = np.where(edge & (kd == 1), 0.0, xam)
    xam = np.where(kd == 2, 0.0, xam)
    xas = np.where(kd == 3, 0.0, xas)
    s = xas + xam
    bad = (s > 0.9 - 1e-5) & (s < 0.9)
    xas = np.where(bad, xas * (0.9 - 2e-5) / np.maximum(s, 1e-30), xas)
    xam = np.where(bad, xam * (0.9 - 2e-5) / np.maximum(s, 1e-30), xam)
    return xas, xam, T0, T1
