"""Partitioning of independent points and specimens across ranks.

The phase model has no spatial coupling (Sec. 3: the ODEs are solved
independently at every point), so a multi-GPU run needs no data exchange:
every rank advances its own specimens or its own z-slab of a block, and the
only collectives are a barrier and a max of the timings.

* ``shard_specimens``: size-balanced greedy assignment of whole specimens
  (largest first, to the least-loaded rank); deterministic.
* ``shard_slabs``: contiguous ranges of z-slabs of one grid (natural order has
  k slowest, so a slab range is a contiguous range of points); ``slab_grid``
  makes a slab a grid of its own with the parent's coordinates (its
  ``k_offset``), so that a sharded run is bit-identical to the whole one
  when the slab boundaries fall on tile boundaries (nx * ny * k0 a multiple
  of 128 points).
"""
from __future__ import annotations


def shard_specimens(sizes, world: int):
    """Lists of specimen indices per rank, balancing the summed sizes."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda j: (-sizes[j], j)):
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += sizes[i]
    return [sorted(p) for p in parts]


def shard_slabs(nz: int, world: int):
    """Half-open z-slab ranges [k0, k1) per rank covering 0 .. nz."""
    if world < 1:
        raise ValueError("world must be >= 1")
    base, extra = divmod(nz, world)
    out, k = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((k, k + n))
        k += n
    return out


def slab_grid(grid, k0: int, k1: int):
    """The z-planes k0 .. k1 - 1 of a grid as a grid of their own (same origin
    and spacing, k_offset = k0 in the parent's frame), so that its points get
    the parent's coordinates to the bit."""
    from dataclasses import replace
    nx, ny, nz = grid.dims
    if not 0 <= k0 < k1 <= nz:
        raise ValueError("slab outside the grid")
    return replace(grid, dims=(nx, ny, k1 - k0), k_offset=int(getattr(grid, "k_offset", 0)) + k0)


def slab_range(grid, k0: int, k1: int):
    """Natural-order point range [start, stop) of the z-planes k0 .. k1 - 1."""
    nx, ny, _ = grid.dims
    return k0 * nx * ny, k1 * nx * ny


def imbalance(sizes, parts) -> float:
    """max rank load / mean rank load."""
    loads = [sum(sizes[i] for i in p) for p in parts]
    mean = sum(loads) / len(loads)
    return max(loads) / mean if mean else 1.0
