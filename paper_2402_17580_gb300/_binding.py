"""ctypes binding of libms_gb300.so (the C ABI in include/ms.h).

Argument marshalling only: every step of the phase model runs in the CUDA
kernels behind the C ABI.  There is no CPU fallback; a missing library or a
failing call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MS_OK = 0
ERRORS = {
    -1: "MS_ERR_INVALID_ARG", -2: "MS_ERR_OOM", -3: "MS_ERR_CUDA", -4: "MS_ERR_DEVICE_TIMEOUT",
    -5: "MS_ERR_NONFINITE", -6: "MS_ERR_STATE", -7: "MS_ERR_UNSUPPORTED",
}
MS_F32, MS_F64ACC, MS_KAHAN, MS_F64 = 0, 1, 2, 3
MS_EXPLICIT, MS_IMPLICIT = 0, 1
MS_PTR_DEVICE = 1
MS_FLAG_TIME_KERNELS = 1
MS_FLAG_GRAPH = 2
MS_FLAG_COUNT_OPS = 4
MS_FLAG_FMA_TRANSCENDENTALS = 8
MS_MLP_IN, MS_MLP_OUT, MS_MLP_PARAMS, MS_MLP_WINDOW = 12, 3, 5187, 8
MS_ACT_GELU, MS_ACT_RELU = 0, 1

d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64


class Params(ctypes.Structure):
    _fields_ = [(n, d) for n in (
        "T_s", "T_l", "T_as_start", "T_as_end", "T_am_start", "T_inf", "k_alpha_eq", "k_am_eq",
        "c_as", "c_b", "k1", "k2", "k3", "f", "T_reg", "init_exit", "init_exit_floor", "T_thr")] + [
        (n, i32) for n in ("martensite_literal", "init_ba_steps", "precision", "steps_per_launch",
                           "rebuild_steps", "block_threads", "flags", "integrator")] + [
        ("dt_sub", d), ("fp_eps_abs", d), ("fp_eps_rel", d), ("fp_max_iter", i32),
        ("tile_order", i32), ("farfield_dist", d)]


class Grid(ctypes.Structure):
    _fields_ = [("origin", d * 3), ("spacing", d * 3), ("dims", i32 * 3), ("k_offset", i32)]


class Track(ctypes.Structure):
    _fields_ = [(n, d) for n in ("x0", "y0", "ux", "uy", "v", "P", "t_start")] + [
        ("layer", i32), ("reserved", i32)]


class Layer(ctypes.Structure):
    _fields_ = [(n, d) for n in ("z_surface", "t_begin", "t_scan_end", "t_end")]


class HeatSource(ctypes.Structure):
    _fields_ = [(n, d) for n in ("A", "k", "alpha", "T0", "T_max", "t_offset", "z_tol")] + [
        ("n_tracks", i32), ("n_layers", i32), ("tracks", ctypes.POINTER(Track)),
        ("layers", ctypes.POINTER(Layer))]


class Stats(ctypes.Structure):
    _fields_ = [(n, i64) for n in ("steps", "point_updates", "tile_steps_total",
                                   "tile_steps_active", "launches")] + [
        ("last_run_ms", d), ("hot_kernel_ms", d), ("hot_kernel_launches", i64),
        ("device_error", i32), ("reserved", i32),
        ("surrogate_windows", i64), ("ode_windows", i64), ("judge_samples", i64),
        ("judge_max_err", d), ("source_evaluations", i64), ("model_point_steps", i64),
        ("fp_iterations", i64), ("fp_unconverged", i64), ("model_sfu_ex2", i64),
        ("model_sfu_slow", i64), ("farfield_node_evaluations", i64),
        ("farfield_point_sources", i64), ("judge_rejected", i64)]


class ThermalParams(ctypes.Structure):
    _fields_ = [(n, d) for n in ("rho", "c", "k_ms", "k_p", "T_s", "T_l", "T0", "T_inf",
                                 "emissivity", "T_max", "beam_radius", "h_powder")] + [
        (n, i32) for n in ("radiation", "dirichlet_bottom", "cap", "reserved")]


STRUCTS = (Params, Grid, Track, Layer, HeatSource, Stats, ThermalParams)

_lib = None


class MSError(RuntimeError):
    def __init__(self, code, where, detail):
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({detail})")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libms_gb300.so (building it first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path}")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.ms_version.restype = ctypes.c_char_p
    lib.ms_strerror.restype = ctypes.c_char_p
    lib.ms_strerror.argtypes = [ctypes.c_int]
    lib.ms_last_error.restype = ctypes.c_char_p
    lib.ms_struct_size.restype = ctypes.c_size_t
    lib.ms_struct_size.argtypes = [ctypes.c_int]
    lib.ms_farfield_table.argtypes = [ctypes.POINTER(ctypes.c_float), i32]
    lib.ms_params_default.argtypes = [ctypes.POINTER(Params)]
    lib.ms_params_check.argtypes = [ctypes.POINTER(Params)]
    lib.ms_create.argtypes = [ctypes.POINTER(Params), i64, ctypes.POINTER(P)]
    lib.ms_destroy.argtypes = [P]
    lib.ms_destroy.restype = None
    lib.ms_set_stream.argtypes = [P, P]
    lib.ms_set_points.argtypes = [P, ctypes.POINTER(Grid), i32]
    lib.ms_set_state.argtypes = [P, P, P, P]
    lib.ms_set_points_subset.argtypes = [P, ctypes.POINTER(Grid), ctypes.POINTER(i64), i64]
    lib.ms_get_temperature.argtypes = [P, P]
    lib.ms_step.argtypes = [P, P, P, d, i32]
    lib.ms_run_track.argtypes = [P, ctypes.POINTER(HeatSource), i64, d]
    lib.ms_get_fractions.argtypes = [P, P, P, P, P]
    lib.ms_get_aux.argtypes = [P, P]
    lib.ms_get_state.argtypes = [P, P, ctypes.POINTER(ctypes.c_size_t)]
    lib.ms_set_state_blob.argtypes = [P, P, ctypes.c_size_t]
    lib.ms_stats.argtypes = [P, ctypes.POINTER(Stats)]
    lib.ms_fill_state.argtypes = [P, d, d]
    lib.ms_reset_stats.argtypes = [P]
    lib.ms_synchronize.argtypes = [P]
    lib.ms_probe_sfu.argtypes = [ctypes.c_int, ctypes.POINTER(d), ctypes.POINTER(d)]
    lib.ms_run_track_noalloc.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Grid),
                                         ctypes.POINTER(HeatSource), P, P, P, i64, i64, i64, d, P]
    lib.ms_surrogate_create.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.POINTER(P)]
    lib.ms_surrogate_create_ex.argtypes = [ctypes.POINTER(ctypes.c_float), i32, i32,
                                           ctypes.POINTER(P)]
    lib.ms_surrogate_get_config.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.ms_surrogate_destroy.argtypes = [P]
    lib.ms_surrogate_destroy.restype = None
    lib.ms_surrogate_set_stream.argtypes = [P, P]
    lib.ms_surrogate_get_params.argtypes = [P, P]
    lib.ms_surrogate_forward.argtypes = [P, P, P, i64]
    lib.ms_surrogate_gradient.argtypes = [P, P, P, i64, P, ctypes.POINTER(d)]
    lib.ms_surrogate_train_step.argtypes = [P, P, P, i64, d, ctypes.POINTER(d)]
    lib.ms_set_surrogate.argtypes = [P, P, d]
    lib.ms_set_judge_tol.argtypes = [P, d]
    lib.ms_apply_correction.argtypes = [P, P, i32, P, P, i64]
    lib.ms_verify.argtypes = [P, P, P, i64, P]
    lib.ms_thermal_params_default.argtypes = [ctypes.POINTER(ThermalParams)]
    lib.ms_thermal_create.argtypes = [ctypes.POINTER(ThermalParams), ctypes.POINTER(Grid),
                                      ctypes.POINTER(P)]
    lib.ms_thermal_destroy.argtypes = [P]
    lib.ms_thermal_destroy.restype = None
    lib.ms_thermal_set_stream.argtypes = [P, P]
    lib.ms_thermal_reset.argtypes = [P]
    lib.ms_thermal_set_source.argtypes = [P, ctypes.POINTER(HeatSource)]
    lib.ms_thermal_step.argtypes = [P, d]
    lib.ms_thermal_fields.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P)]
    lib.ms_thermal_get.argtypes = [P, P, P]
    lib.ms_thermal_stats.argtypes = [P, ctypes.POINTER(d), ctypes.POINTER(i64), ctypes.POINTER(d)]
    lib.ms_thermal_run_coupled.argtypes = [P, P, i64, d]
    lib.ms_coarsen_sizes.argtypes = [ctypes.POINTER(i32), i32, ctypes.POINTER(i64),
                                     ctypes.POINTER(ctypes.c_size_t)]
    lib.ms_coarsen_mask.argtypes = [P, P, P, ctypes.POINTER(i32), d, i32, P,
                                    ctypes.POINTER(i64), P, ctypes.c_size_t, i32, P]
    lib.ms_coarsen_ctx.argtypes = [P, d, i32, P, ctypes.POINTER(i64)]
    lib.ms_eval_transcendental.argtypes = [ctypes.c_int, P, P, i64]
    for i, s in enumerate(STRUCTS):
        if lib.ms_struct_size(i) != ctypes.sizeof(s):
            raise RuntimeError(f"ABI mismatch for {s.__name__}: C {lib.ms_struct_size(i)} "
                               f"vs ctypes {ctypes.sizeof(s)}")
    _lib = lib
    return lib


def _grid(g) -> Grid:
    """ms_grid of a workloads.Grid-like object (origin, spacing, dims, and
    optionally k_offset)."""
    return Grid((d * 3)(*g.origin), (d * 3)(*g.spacing), (i32 * 3)(*g.dims),
                int(getattr(g, "k_offset", 0)))


def _check(rc, where):
    if rc != MS_OK:
        raise MSError(rc, where, load().ms_last_error().decode())


def run_track_noalloc(params, grid, source, xas_ptr, xam_ptr, aux_ptr, n_points, step0, n_steps,
                      dt, stream_handle=0):
    """ms_run_track_noalloc: advance one specimen whose state lives in the
    caller's device arrays (raw pointers), without any allocation."""
    g = _grid(grid)
    h, keep = make_heat_source(source)
    _check(load().ms_run_track_noalloc(ctypes.byref(params), ctypes.byref(g), ctypes.byref(h),
                                       ctypes.c_void_p(xas_ptr), ctypes.c_void_p(xam_ptr),
                                       ctypes.c_void_p(aux_ptr), int(n_points), int(step0),
                                       int(n_steps), float(dt), ctypes.c_void_p(stream_handle or 0)),
           "ms_run_track_noalloc")
    del keep


COARSEN_MAX_LEVELS = 30   # MS_COARSEN_MAX_LEVELS


def coarsen_sizes(dims, n_levels, with_scratch=False):
    """ms_coarsen_sizes: octants of levels 1 .. n_levels of a grid (host
    only); with_scratch also returns the device scratch bytes."""
    out = (i64 * int(n_levels))()
    sb = ctypes.c_size_t(0)
    _check(load().ms_coarsen_sizes((i32 * 3)(*dims), int(n_levels), out, ctypes.byref(sb)),
           "ms_coarsen_sizes")
    counts = [int(v) for v in out]
    return (counts, int(sb.value)) if with_scratch else counts


def _split_masks(flat, dims, n_levels):
    out, off = [], 0
    for l in range(1, n_levels + 1):
        shp = tuple(1 if n == 1 else (n - 1) >> l for n in dims)
        c = int(np.prod(shp))
        out.append(flat[off:off + c].reshape(shp[::-1]))
        off += c
    return out


def coarsen_mask(x_as, x_am, x_beta, dims, tol, n_levels):
    """ms_coarsen_mask on host arrays: the masks of levels 1 .. n_levels as
    uint8 arrays of shape (nz_l, ny_l, nx_l), and the coarsenable octants
    per level."""
    a, m, b = (np.ascontiguousarray(v, dtype=np.float64) for v in (x_as, x_am, x_beta))
    n = int(np.prod(dims))
    assert a.size == n and m.size == n and b.size == n
    flat = np.empty(sum(coarsen_sizes(dims, n_levels)), dtype=np.uint8)
    cnt = (i64 * int(n_levels))()
    _check(load().ms_coarsen_mask(_ptr(a), _ptr(m), _ptr(b), (i32 * 3)(*dims), float(tol),
                                  int(n_levels), _ptr(flat), cnt, None, 0, 0, None),
           "ms_coarsen_mask")
    return _split_masks(flat, dims, n_levels), [int(v) for v in cnt]


def coarsen_mask_device(xas_ptr, xam_ptr, xbeta_ptr, dims, tol, n_levels, mask_ptr,
                        stream_handle=0, scratch_ptr=0, scratch_bytes=0):
    """ms_coarsen_mask on device arrays (raw pointers, and optionally the
    caller's scratch); returns the coarsenable octants per level."""
    cnt = (i64 * int(n_levels))()
    _check(load().ms_coarsen_mask(ctypes.c_void_p(xas_ptr), ctypes.c_void_p(xam_ptr),
                                  ctypes.c_void_p(xbeta_ptr), (i32 * 3)(*dims), float(tol),
                                  int(n_levels), ctypes.c_void_p(mask_ptr), cnt,
                                  ctypes.c_void_p(scratch_ptr or 0), int(scratch_bytes),
                                  MS_PTR_DEVICE, ctypes.c_void_p(stream_handle or 0)),
           "ms_coarsen_mask")
    return [int(v) for v in cnt]


TRANSCENDENTALS = ("fma_ex2", "fma_lg2", "sfu_ex2", "sfu_lg2")


def eval_transcendental(which: str, x):
    """ms_eval_transcendental: the device's exp2 / log2 (FMA-pipe polynomial
    or SFU) of a float32 array."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    _check(load().ms_eval_transcendental(TRANSCENDENTALS.index(which), _ptr(x), _ptr(y), x.size),
           "ms_eval_transcendental")
    return y


PROBE_OPS = ("ex2", "lg2", "rsqrt", "rcp", "ffma")


def probe_pipe(op: str):
    """(thread-level ops/s, SM MHz seen) of one pipe probe on the current device."""
    v, mhz = d(), d()
    _check(load().ms_probe_sfu(PROBE_OPS.index(op), ctypes.byref(v), ctypes.byref(mhz)),
           "ms_probe_sfu")
    return v.value, mhz.value


FF_TABLE_FLOATS = 1032   # MS_FF_TABLE_FLOATS


def farfield_table():
    """The far field's interpolation table (ms_farfield_table): Lagrange
    weights [8, 128] of the 8 Chebyshev nodes at a row tile's 128 points, and
    the node positions [8] on the tile's x-range [0, 1]."""
    out = (ctypes.c_float * FF_TABLE_FLOATS)()
    _check(load().ms_farfield_table(out, FF_TABLE_FLOATS), "ms_farfield_table")
    a = np.frombuffer(out, dtype=np.float32).copy()
    return a[:1024].reshape(8, 128), a[1024:]


def check_params(p: Params) -> None:
    """ms_params_check: raises MSError if ms_create would reject p."""
    _check(load().ms_params_check(ctypes.byref(p)), "ms_params_check")


def default_params(**overrides) -> Params:
    p = Params()
    _check(load().ms_params_default(ctypes.byref(p)), "ms_params_default")
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _f64(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def make_heat_source(src) -> tuple:
    """ms_heat_source for an object with the fields of workloads.HeatSource;
    returns (struct, keep-alive arrays)."""
    tr = np.asarray(src.tracks, dtype=np.float64).reshape(-1, 8)
    ly = np.asarray(src.layers, dtype=np.float64).reshape(-1, 4)
    tracks = (Track * max(1, len(tr)))()
    for i, r in enumerate(tr):
        tracks[i] = Track(r[0], r[1], r[2], r[3], r[4], r[5], r[6], int(r[7]), 0)
    layers = (Layer * len(ly))()
    for i, r in enumerate(ly):
        layers[i] = Layer(*r)
    h = HeatSource(src.A, src.k, src.alpha, src.T0, src.T_max, src.t_offset, src.z_tol,
                   len(tr), len(ly), ctypes.cast(tracks, ctypes.POINTER(Track)),
                   ctypes.cast(layers, ctypes.POINTER(Layer)))
    return h, (tracks, layers)


class Context:
    """One ms_ctx: n_points points on the current CUDA device."""

    def __init__(self, n_points: int, params: Params | None = None, **overrides):
        self._lib = load()
        p = params if params is not None else default_params(**overrides)
        if params is not None:
            for k, v in overrides.items():
                setattr(p, k, v)
        self.params = p
        self.n = int(n_points)
        self._h = ctypes.c_void_p()
        _check(self._lib.ms_create(ctypes.byref(p), self.n, ctypes.byref(self._h)), "ms_create")
        self._keep = None

    def close(self):
        if self._h:
            self._lib.ms_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def set_surrogate(self, surrogate: "Surrogate | None", judge_frac: float = 0.0):
        """Attach (or with None detach) a surrogate: ms_run_track then runs
        the hybrid window kernel."""
        _check(self._lib.ms_set_surrogate(self._h, surrogate.handle if surrogate else None,
                                          float(judge_frac)), "ms_set_surrogate")
        self._surrogate = surrogate

    def set_judge_tol(self, tol: float):
        """ms_set_judge_tol: judged tile-windows whose network result differs
        from the explicit steps' by more than tol take the explicit result."""
        _check(self._lib.ms_set_judge_tol(self._h, float(tol)), "ms_set_judge_tol")

    def verify(self, ref: "Context", idx=None, n=None):
        """Device-side verification against another context (ms_verify):
        (max |dX| over the four fractions, max |sum - 1| of self, of ref)."""
        out = np.zeros(3)
        if idx is not None:
            idx = np.ascontiguousarray(idx, dtype=np.int64)
            n = idx.size
        elif n is None:
            n = ref.n
        _check(self._lib.ms_verify(self._h, ref.handle, None if idx is None else _ptr(idx), int(n),
                                   _ptr(out)), "ms_verify")
        return float(out[0]), float(out[1]), float(out[2])

    def apply_correction(self, T, xas, xam):
        """The correction g applied to independent points at the temperatures
        T ([n] or [n, m]: m levels in turn); returns the corrected (xas, xam)."""
        a = np.array(xas, dtype=np.float64, copy=True).ravel()
        b = np.array(xam, dtype=np.float64, copy=True).ravel()
        T = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(a.size, -1))
        assert b.size == a.size
        _check(self._lib.ms_apply_correction(self._h, _ptr(T), T.shape[1], _ptr(a), _ptr(b), a.size),
               "ms_apply_correction")
        return a, b

    def set_stream(self, stream_handle: int | None):
        _check(self._lib.ms_set_stream(self._h, ctypes.c_void_p(stream_handle or 0)), "ms_set_stream")

    def set_points(self, grids):
        arr = (Grid * len(grids))()
        for i, g in enumerate(grids):
            arr[i] = _grid(g)
        _check(self._lib.ms_set_points(self._h, arr, len(grids)), "ms_set_points")

    def set_points_subset(self, grid, idx):
        """The context's points are grid points idx (natural grid indices)."""
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        g = _grid(grid)
        _check(self._lib.ms_set_points_subset(self._h, ctypes.byref(g),
                                              idx.ctypes.data_as(ctypes.POINTER(i64)), idx.size),
               "ms_set_points_subset")

    def temperature(self):
        out = np.empty(self.n)
        _check(self._lib.ms_get_temperature(self._h, _ptr(out)), "ms_get_temperature")
        return out

    def set_state(self, xas, xam, aux=None):
        xas, xam = _f64(xas, self.n), _f64(xam, self.n)
        a = None if aux is None else _f64(aux, self.n)
        _check(self._lib.ms_set_state(self._h, _ptr(xas), _ptr(xam), None if a is None else _ptr(a)),
               "ms_set_state")

    def fill_state(self, xas=0.9, xam=0.0):
        """Uniform state on the device (no host copy); resets the step counter."""
        _check(self._lib.ms_fill_state(self._h, float(xas), float(xam)), "ms_fill_state")

    def reset_stats(self):
        _check(self._lib.ms_reset_stats(self._h), "ms_reset_stats")

    def step(self, T_prev, T_new, dt):
        """One explicit step with host temperature arrays (float32)."""
        t0 = np.ascontiguousarray(T_prev, dtype=np.float32)
        t1 = np.ascontiguousarray(T_new, dtype=np.float32)
        assert t0.size == self.n and t1.size == self.n
        _check(self._lib.ms_step(self._h, _ptr(t0), _ptr(t1), float(dt), 0), "ms_step")

    def step_device(self, T_prev_ptr: int, T_new_ptr: int, dt):
        """One explicit step with device temperature arrays (raw pointers)."""
        _check(self._lib.ms_step(self._h, ctypes.c_void_p(T_prev_ptr), ctypes.c_void_p(T_new_ptr),
                                 float(dt), MS_PTR_DEVICE), "ms_step")

    def run_track(self, sources, n_steps, dt):
        hs = [make_heat_source(s) for s in sources]
        arr = (HeatSource * len(hs))(*[h for h, _ in hs])
        self._keep = (arr, hs)
        _check(self._lib.ms_run_track(self._h, arr, int(n_steps), float(dt)), "ms_run_track")

    def fractions(self, with_beta=True):
        out = [np.empty(self.n) for _ in range(4)]
        _check(self._lib.ms_get_fractions(self._h, _ptr(out[0]), _ptr(out[1]),
                                          _ptr(out[2]) if with_beta else None,
                                          _ptr(out[3]) if with_beta else None), "ms_get_fractions")
        return tuple(out) if with_beta else (out[0], out[1])

    def fractions_into(self, outs):
        """Write X_as, X_am, X_beta, X_liq into four caller arrays (float64,
        n_points each, e.g. pinned host memory)."""
        assert len(outs) == 4 and all(o.dtype == np.float64 and o.size == self.n and
                                      o.flags["C_CONTIGUOUS"] for o in outs)
        _check(self._lib.ms_get_fractions(self._h, *[_ptr(o) for o in outs]), "ms_get_fractions")

    def coarsen(self, tol, n_levels, dims):
        """ms_coarsen_ctx: the coarsening masks of the context's grid (dims
        as given to set_points) on its current state; (masks, counts)."""
        flat = np.empty(sum(coarsen_sizes(dims, n_levels)), dtype=np.uint8)
        cnt = (i64 * int(n_levels))()
        _check(self._lib.ms_coarsen_ctx(self._h, float(tol), int(n_levels), _ptr(flat), cnt),
               "ms_coarsen_ctx")
        return _split_masks(flat, dims, n_levels), [int(v) for v in cnt]

    def aux(self):
        out = np.empty(self.n)
        _check(self._lib.ms_get_aux(self._h, _ptr(out)), "ms_get_aux")
        return out

    def checkpoint(self) -> bytes:
        n = ctypes.c_size_t(0)
        _check(self._lib.ms_get_state(self._h, None, ctypes.byref(n)), "ms_get_state")
        buf = ctypes.create_string_buffer(n.value)
        _check(self._lib.ms_get_state(self._h, buf, ctypes.byref(n)), "ms_get_state")
        return buf.raw

    def restore(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(self._lib.ms_set_state_blob(self._h, buf, len(blob)), "ms_set_state_blob")

    def stats(self) -> Stats:
        s = Stats()
        _check(self._lib.ms_stats(self._h, ctypes.byref(s)), "ms_stats")
        return s

    def synchronize(self):
        _check(self._lib.ms_synchronize(self._h), "ms_synchronize")


class Surrogate:
    """One ms_surrogate: the window MLP's FP32 master parameters, Adam state
    and BF16 inference copy on the current device, with its hidden activation
    (MS_ACT_GELU, MS_ACT_RELU) and temperature stride (windows of 8 x stride
    steps).  Data arguments are device pointers (e.g.
    torch.Tensor.data_ptr() of contiguous float32 tensors)."""

    def __init__(self, params, activation: int = MS_ACT_GELU, stride: int = 1):
        self._lib = load()
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != MS_MLP_PARAMS:
            raise ValueError(f"expected {MS_MLP_PARAMS} parameters, got {p.size}")
        self._h = ctypes.c_void_p()
        _check(self._lib.ms_surrogate_create_ex(p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                int(activation), int(stride),
                                                ctypes.byref(self._h)), "ms_surrogate_create_ex")

    def config(self) -> tuple[int, int]:
        """(activation, stride) as the library holds them."""
        a, r = ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.ms_surrogate_get_config(self._h, ctypes.byref(a), ctypes.byref(r)),
               "ms_surrogate_get_config")
        return a.value, r.value

    @property
    def activation(self) -> int:
        return self.config()[0]

    @property
    def stride(self) -> int:
        return self.config()[1]

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            self._lib.ms_surrogate_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_handle: int | None):
        _check(self._lib.ms_surrogate_set_stream(self._h, ctypes.c_void_p(stream_handle or 0)),
               "ms_surrogate_set_stream")

    def params(self) -> np.ndarray:
        out = np.empty(MS_MLP_PARAMS, dtype=np.float32)
        _check(self._lib.ms_surrogate_get_params(self._h, _ptr(out)), "ms_surrogate_get_params")
        return out

    def forward(self, x_ptr: int, y_ptr: int, n: int):
        _check(self._lib.ms_surrogate_forward(self._h, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr),
                                              int(n)), "ms_surrogate_forward")

    def gradient(self, x_ptr: int, t_ptr: int, n: int, grad_ptr: int | None = None) -> float:
        loss = d()
        _check(self._lib.ms_surrogate_gradient(self._h, ctypes.c_void_p(x_ptr), ctypes.c_void_p(t_ptr),
                                               int(n), ctypes.c_void_p(grad_ptr or 0),
                                               ctypes.byref(loss)), "ms_surrogate_gradient")
        return loss.value

    def train_step(self, x_ptr: int, t_ptr: int, n: int, lr: float, want_loss: bool = False):
        loss = d()
        _check(self._lib.ms_surrogate_train_step(self._h, ctypes.c_void_p(x_ptr),
                                                 ctypes.c_void_p(t_ptr), int(n), float(lr),
                                                 ctypes.byref(loss) if want_loss else None),
               "ms_surrogate_train_step")
        return loss.value if want_loss else None


def thermal_params(**overrides) -> ThermalParams:
    p = ThermalParams()
    _check(load().ms_thermal_params_default(ctypes.byref(p)), "ms_thermal_params_default")
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Thermal:
    """One ms_thermal: the grid thermal solver on the current device."""

    def __init__(self, grid, params: ThermalParams | None = None, **overrides):
        self._lib = load()
        p = params if params is not None else thermal_params(**overrides)
        self.params = p
        g = _grid(grid)
        self.n = int(grid.dims[0]) * int(grid.dims[1]) * int(grid.dims[2])
        self._h = ctypes.c_void_p()
        _check(self._lib.ms_thermal_create(ctypes.byref(p), ctypes.byref(g), ctypes.byref(self._h)),
               "ms_thermal_create")
        self._keep = None

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            self._lib.ms_thermal_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_handle: int | None):
        _check(self._lib.ms_thermal_set_stream(self._h, ctypes.c_void_p(stream_handle or 0)),
               "ms_thermal_set_stream")

    def reset(self):
        _check(self._lib.ms_thermal_reset(self._h), "ms_thermal_reset")

    def set_source(self, source):
        h, keep = make_heat_source(source)
        self._keep = keep
        _check(self._lib.ms_thermal_set_source(self._h, ctypes.byref(h)), "ms_thermal_set_source")

    def step(self, dt: float):
        _check(self._lib.ms_thermal_step(self._h, float(dt)), "ms_thermal_step")

    def fields(self):
        """Device pointers (T_prev, T_cur, r_c) as integers."""
        a, b, c = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(self._lib.ms_thermal_fields(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "ms_thermal_fields")
        return a.value, b.value, c.value

    def get(self):
        T, rc = np.empty(self.n), np.empty(self.n)
        _check(self._lib.ms_thermal_get(self._h, _ptr(T), _ptr(rc)), "ms_thermal_get")
        return T, rc

    def stats(self):
        t, n, ms_ = d(), i64(), d()
        _check(self._lib.ms_thermal_stats(self._h, ctypes.byref(t), ctypes.byref(n), ctypes.byref(ms_)),
               "ms_thermal_stats")
        return {"time_s": t.value, "substeps": n.value, "kernel_ms": ms_.value}

    def run_coupled(self, ctx: Context, n_steps: int, dt: float):
        _check(self._lib.ms_thermal_run_coupled(self._h, ctx.handle, int(n_steps), float(dt)),
               "ms_thermal_run_coupled")
