"""Shared helpers of the GPU parity tests: run a workload through the C ABI and
through the FP64 oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle as orc
import workloads as wl


def oracle_view(x):
    """Inputs as the FP32 kernels store them: rounded to float32, except that
    the FP32 store's 0.9f stands for the paper's bound 0.9 (App. A's initial
    state and the alpha bound), so it is given to the oracle as 0.9."""
    x = np.asarray(x, dtype=np.float64)
    x32 = x.astype(np.float32).astype(np.float64)
    return np.where(x == 0.9, 0.9, x32)


def oracle_params(ctx_params=None):
    """Oracle parameter vector with the same readings as a ms_params struct."""
    if ctx_params is None:
        return orc.params()
    return orc.params(**{k: float(getattr(ctx_params, k)) for k in orc.DEFAULTS})


def gpu_workload(w: wl.Workload, params=None, n_steps=None, chunks=1, **overrides):
    """Run a workload through ms_run_track; returns the context and the four
    fractions of every point (natural order)."""
    import paper_2402_17580_gb300 as ms
    kw = dict(T_thr=w.T_thr)
    kw.update(overrides)
    ctx = ms.Context(w.n_points, params, **kw)
    ctx.set_points([s.grid for s in w.specimens])
    ctx.set_state(np.full(w.n_points, w.init_xas), np.full(w.n_points, w.init_xam))
    steps = w.n_steps if n_steps is None else n_steps
    done = 0
    for c in range(chunks):
        k = steps // chunks + (1 if c < steps % chunks else 0)
        ctx.run_track([s.source for s in w.specimens], k, w.dt)
        done += k
    return ctx, ctx.fractions()


def spec_offsets(w: wl.Workload):
    return np.cumsum([0] + [s.grid.n for s in w.specimens])


def oracle_workload(w: wl.Workload, idx=None, p=None, n_steps=None):
    """Oracle fractions of the points with global natural indices idx (all if
    None), run from the workload's initial state."""
    offs = spec_offsets(w)
    idx = np.arange(w.n_points) if idx is None else np.asarray(idx, dtype=np.int64)
    steps = w.n_steps if n_steps is None else n_steps
    out = np.empty((4, idx.size))
    spec_of = np.searchsorted(offs, idx, side="right") - 1
    for s in np.unique(spec_of):
        sel = np.nonzero(spec_of == s)[0]
        sp = w.specimens[s]
        x, y, z = sp.grid.coords(idx[sel] - offs[s])
        st = orc.State.uniform(sel.size, w.init_xas, w.init_xam)
        T_last = orc.run_track(st, sp.source, x, y, z, 0, steps, w.dt, p)
        xas, xam, xb, xl = orc.fractions(st, T_last, p)
        out[:, sel] = np.stack([xas, xam, xb, xl])
    return out


def max_abs_diff(gpu, ora, idx=None):
    g = np.stack(gpu) if idx is None else np.stack(gpu)[:, idx]
    return float(np.max(np.abs(g - ora)))
