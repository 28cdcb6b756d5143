"""Autotuner of the ms_run_track launch configuration.

For a set of specimens it times short runs of every candidate configuration
(steps per launch S, CTA size, CUDA-graph replay) from the same start state,
with the library's own CUDA-event timing of the run (``ms_stats.last_run_ms``),
and returns the fastest.  Results depend only on the measured device, so they
are cached per (device name, workload key) for the life of the process.

    from paper_2402_17580_gb300.autotune import autotune
    best = autotune(grids, sources, n_points, dt, T_thr, trial_steps=2048)
    ctx = Context(n_points, **best.params)
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

from ._binding import MS_FLAG_GRAPH, MS_FLAG_TIME_KERNELS, Context

DEFAULT_CANDIDATES = {
    "steps_per_launch": (32, 64, 128, 256),
    "block_threads": (128, 256),
    "graph": (False, True),
}

_cache: dict = {}


@dataclass
class TuneResult:
    params: dict
    ms: float
    table: list = field(default_factory=list)

    def as_dict(self):
        return {"best": self.params, "best_ms": self.ms,
                "table": [{"config": c, "ms": t} for c, t in self.table]}


def autotune(grids, sources, n_points, dt, T_thr=0.0, trial_steps=2048, repeats=2,
             candidates=None, precision=0, key=None, init=(0.9, 0.0)) -> TuneResult:
    """Time every candidate on ``trial_steps`` steps (best of ``repeats``
    after one warm-up) and return the fastest configuration."""
    cand = dict(DEFAULT_CANDIDATES)
    if candidates:
        cand.update(candidates)
    cache_key = None
    if key is not None:
        cache_key = (key, trial_steps, tuple(sorted((k, tuple(v)) for k, v in cand.items())))
        if cache_key in _cache:
            return _cache[cache_key]
    table = []
    for S, bt, graph in itertools.product(cand["steps_per_launch"], cand["block_threads"],
                                          cand["graph"]):
        params = dict(steps_per_launch=int(S), block_threads=int(bt), T_thr=float(T_thr),
                      precision=int(precision),
                      flags=(MS_FLAG_GRAPH if graph else 0))
        ctx = Context(n_points, **params)
        ctx.set_points(grids)
        times = []
        for r in range(repeats + 1):
            ctx.fill_state(*init)
            ctx.run_track(sources, trial_steps, dt)
            ctx.synchronize()
            if r > 0:
                times.append(float(ctx.stats().last_run_ms))
        ctx.close()
        table.append(({"steps_per_launch": int(S), "block_threads": int(bt), "graph": bool(graph)},
                      min(times)))
    best_cfg, best_ms = min(table, key=lambda x: x[1])
    params = {"steps_per_launch": best_cfg["steps_per_launch"],
              "block_threads": best_cfg["block_threads"],
              "flags": MS_FLAG_GRAPH if best_cfg["graph"] else 0}
    res = TuneResult(params, best_ms, table)
    if cache_key is not None:
        _cache[cache_key] = res
    return res


__all__ = ["autotune", "TuneResult", "DEFAULT_CANDIDATES", "MS_FLAG_TIME_KERNELS"]
