"""Reference of the phase-aware coarsening criterion (test infrastructure
only: tests/, ``__graft_entry__.smoke()`` and bench.py's baseline legs may
import it; the product never does).

The paper (Sec. 3, the adaptive-mesh passage) keeps the microstructure
phases as material history on an adaptive, growing octree mesh: an octant
made of eight sibling cells of one refinement level may be coarsened only
when, for every phase (beta, alpha_s, alpha_m), all its values lie close to
each other.

Written out on the point grid (the phases live at the grid points, as the
phase DoFs sit at the thermal DoFs):

* the finest cells are the grid cells between neighbouring points; an octant
  of level l >= 1 is made of 2 x 2 x 2 sibling octants of level l - 1 (level
  0: the grid cells), so along an axis with n points octant i of level l
  spans the points i 2^l ... (i + 1) 2^l, and there are floor((n - 1) / 2^l)
  of them (an axis with one point is a flat axis: one octant spanning it);
* "all its values close to each other" is read as: for each phase, the
  largest minus the smallest value over the octant's points is at most tol
  (one tolerance for the three phases);
* the mask of level l holds, per octant (x fastest, then y, then z), 1 if the
  octant may be coarsened and 0 otherwise.

Parity: pinned by tests/test_coarsen_oracle.py against closed forms (uniform
fields, a single perturbed point, linear ramps whose range per octant is
known, octants exactly at the tolerance) and by the hierarchy property a
coarsenable octant's children are coarsenable.
"""
from __future__ import annotations

import numpy as np


def octants_per_axis(n: int, level: int) -> int:
    """Octants of `level` along an axis with n points."""
    if n == 1:
        return 1
    return (n - 1) // (1 << level)


def level_shape(dims, level):
    """(nx, ny, nz) octant counts of a level for grid dims (nx, ny, nz)."""
    return tuple(octants_per_axis(int(n), level) for n in dims)


def mask_sizes(dims, n_levels):
    """Octants of levels 1 .. n_levels."""
    return [int(np.prod(level_shape(dims, l))) for l in range(1, n_levels + 1)]


def _span(i, level, n):
    if n == 1:
        return slice(0, 1)
    return slice(i << level, ((i + 1) << level) + 1)


def phase_fields(x_as, x_am, x_beta, dims):
    """The three phases as (nz, ny, nx) arrays (natural grid order, x fastest)."""
    nx, ny, nz = (int(d) for d in dims)
    return [np.asarray(a, dtype=np.float64).reshape(nz, ny, nx) for a in (x_as, x_am, x_beta)]


def octant_ranges(fields, level, i, j, k):
    """max - min of each phase over octant (i, j, k) of `level`; the octant
    may be coarsened when all three are <= tol."""
    nz, ny, nx = fields[0].shape
    sk, sj, si = _span(k, level, nz), _span(j, level, ny), _span(i, level, nx)
    return [float(f[sk, sj, si].max() - f[sk, sj, si].min()) for f in fields]


def coarsen_masks(x_as, x_am, x_beta, dims, tol, n_levels):
    """The masks of levels 1 .. n_levels as a list of uint8 arrays of shape
    (nz_l, ny_l, nx_l): octant (i, j, k) of level l is 1 when every phase's
    max - min over its points is <= tol.  The phase arrays are in natural
    grid order (x fastest)."""
    fields = phase_fields(x_as, x_am, x_beta, dims)
    out = []
    for level in range(1, n_levels + 1):
        cx, cy, cz = level_shape(dims, level)
        m = np.zeros((cz, cy, cx), dtype=np.uint8)
        for k in range(cz):
            for j in range(cy):
                for i in range(cx):
                    ranges = octant_ranges(fields, level, i, j, k)
                    m[k, j, i] = 1 if all(r <= tol for r in ranges) else 0
        out.append(m)
    return out
