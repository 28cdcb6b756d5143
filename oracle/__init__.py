"""FP64 CPU oracle of the Ti-6Al-4V phase model (arXiv 2402.17580).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2402_17580_gb300``) never does, and the two
share no code.

The arithmetic lives in ``ms_oracle.c`` (plain C, double precision, libm,
OpenMP over independent points).  This module compiles it with gcc on first
use (or via :func:`build`) and marshals numpy arrays through ctypes.

Default parameters are the paper's Table 1 (T_s, T_l), Table 2 (transformation
temperatures, equilibrium constants) and Table 3 (fitted diffusion
parameters), plus T_reg = 100 K (Sec. 2.2) and the App. A initiation exit
threshold 1e-15.  ``init_exit_floor`` is reading A5 (the FP32 kernels cannot
resolve X~_beta below ~1e-7 against 0.9, so initiation is left only once
X~_beta >= 1e-3); set it to 0 for the literal App. A rule.

Parity status: every function here is pinned by tests/test_oracle_pins.py
(closed forms, an independent ODE integration, invariants, the PDE the
moving source satisfies, the values the paper prints); the readings A3, A5
and A6 themselves are not fixed by the paper ("parity unpinned" for the choice
of reading, not for its arithmetic).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ms_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libms_oracle.so")

# parameter vector layout: must match the enum at the top of ms_oracle.c
PARAM_NAMES = (
    "T_s", "T_l", "T_as_start", "T_as_end", "T_am_start", "T_inf",
    "k_alpha_eq", "k_am_eq", "c_as", "c_b", "k1", "k2", "k3", "f",
    "T_reg", "init_exit", "init_exit_floor", "martensite_literal", "init_ba_steps",
    "integrator", "dt_sub", "fp_eps_abs", "fp_eps_rel", "fp_max_iter",
)

DEFAULTS = {
    # Table 1 / Table 2
    "T_s": 1878.0, "T_l": 1928.0,
    "T_as_start": 1273.0, "T_as_end": 935.0, "T_am_start": 848.0, "T_inf": 293.0,
    "k_alpha_eq": 0.0068, "k_am_eq": 0.00415,
    # Table 3
    "c_as": 2.51, "c_b": 11.0, "k1": 0.294, "k2": 850.0, "k3": 0.0337, "f": 3.8,
    # Sec. 2.2 regularisation width, App. A exit threshold, readings
    "T_reg": 100.0, "init_exit": 1e-15, "init_exit_floor": 1e-3,
    "martensite_literal": 0.0, "init_ba_steps": 0.0,
    # Sec. 3 implicit scheme: Crank-Nicolson, substeps <= 0.01 s, WRMS
    # tolerances 1e-10 / 1e-3; the iteration cap is this build's choice
    "integrator": 0.0, "dt_sub": 0.01, "fp_eps_abs": 1e-10, "fp_eps_rel": 1e-3,
    "fp_max_iter": 100.0,
}

MODE_NONE, MODE_AS_TO_B, MODE_B_TO_AS = 0, 1, 2

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ms_oracle.c into a shared library (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # MS_ORACLE_LIB loads a deliberately broken copy of the oracle
            # (tests/test_oracle_mutations.py checks that the pins catch it)
            lib = ctypes.CDLL(os.environ.get("MS_ORACLE_LIB") or build())
            d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
            P = ctypes.c_void_p
            for name in ("orc_liquid_fraction", "orc_xalpha_eq", "orc_xam0_eq", "orc_k_alpha_s"):
                f = getattr(lib, name)
                f.argtypes, f.restype = [P, d], d
            lib.orc_xam_eq.argtypes, lib.orc_xam_eq.restype = [P, d, d], d
            lib.orc_logistic_step.argtypes, lib.orc_logistic_step.restype = [d, d, d, d, d], d
            lib.orc_rates.argtypes, lib.orc_rates.restype = [P, d, d, d, P, P], None
            lib.orc_correct.argtypes, lib.orc_correct.restype = [P, d, P, P], None
            lib.orc_fractions.argtypes, lib.orc_fractions.restype = [P, i64, P, P, P, P, P], None
            lib.orc_run_temps.argtypes = [P, i64, i64, d, P, P, P, P, P]
            lib.orc_run_temps.restype = None
            lib.orc_temperature.argtypes = [P, P, i32, P, i32, i64, P, P, P, d, P, P]
            lib.orc_temperature.restype = None
            lib.orc_run_track.argtypes = [P, P, P, i32, P, i32, i64, P, P, P, i64, i64, d,
                                          P, P, P, P, P]
            lib.orc_run_track.restype = None
            lib.orc_run_track_windows.argtypes = [P, P, P, i32, P, i32, i64, P, P, P, i64, i64,
                                                  d, i32, i32, d, i64, P, P, P, P, P, P]
            lib.orc_run_track_windows.restype = None
            lib.orc_cn_step.argtypes, lib.orc_cn_step.restype = [P, d, d, d, P, P, P], ctypes.c_int
            lib.orc_n_substeps.argtypes, lib.orc_n_substeps.restype = [P, d], i64
            lib.orc_num_threads.restype = ctypes.c_int
            lib.orc_set_num_threads.argtypes, lib.orc_set_num_threads.restype = [ctypes.c_int], None
            lib.orc_param_count.restype = ctypes.c_int
            assert lib.orc_param_count() == len(PARAM_NAMES)
            _lib = lib
    return _lib


def params(**overrides) -> np.ndarray:
    """Parameter vector (float64) with the paper's defaults and overrides."""
    unknown = set(overrides) - set(DEFAULTS)
    if unknown:
        raise KeyError(f"unknown oracle parameters: {sorted(unknown)}")
    vals = dict(DEFAULTS)
    vals.update({k: float(v) for k, v in overrides.items()})
    return np.array([vals[n] for n in PARAM_NAMES], dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _prm(p):
    return params() if p is None else np.ascontiguousarray(p, dtype=np.float64)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's point loops from now on (n > 0)."""
    _load().orc_set_num_threads(int(n))


# ---------------------------------------------------------------- model pieces
def _scalar_fn(name, T, p=None):
    lib, p = _load(), _prm(p)
    f = getattr(lib, name)
    T = np.asarray(T, dtype=np.float64)
    out = np.array([f(_ptr(p), float(t)) for t in T.ravel()]).reshape(T.shape)
    return out if out.shape else float(out)


def liquid_fraction(T, p=None):
    return _scalar_fn("orc_liquid_fraction", T, p)


def xalpha_eq(T, p=None):
    return _scalar_fn("orc_xalpha_eq", T, p)


def xam0_eq(T, p=None):
    return _scalar_fn("orc_xam0_eq", T, p)


def k_alpha_s(T, p=None):
    return _scalar_fn("orc_k_alpha_s", T, p)


def xam_eq(T, xas, p=None):
    lib, p = _load(), _prm(p)
    return float(lib.orc_xam_eq(_ptr(p), float(T), float(xas)))


def logistic_step(X, D, k, c, dt):
    return float(_load().orc_logistic_step(float(X), float(D), float(k), float(c), float(dt)))


def rates(T, xas, xam, p=None):
    lib, p = _load(), _prm(p)
    a, m = ctypes.c_double(), ctypes.c_double()
    lib.orc_rates(_ptr(p), float(T), float(xas), float(xam), ctypes.byref(a), ctypes.byref(m))
    return a.value, m.value


def correct(T, xas, xam, p=None):
    lib, p = _load(), _prm(p)
    a, m = ctypes.c_double(float(xas)), ctypes.c_double(float(xam))
    lib.orc_correct(_ptr(p), float(T), ctypes.byref(a), ctypes.byref(m))
    return a.value, m.value


def cn_step(T0, T1, dt, xas, xam, p=None):
    """One Crank-Nicolson step with the fixed-point iteration (no substeps, no
    initiation): returns (X_as, X_am, iterations, converged)."""
    lib, p = _load(), _prm(p)
    a, m = ctypes.c_double(float(xas)), ctypes.c_double(float(xam))
    conv = ctypes.c_int(0)
    it = lib.orc_cn_step(_ptr(p), float(T0), float(T1), float(dt), ctypes.byref(a),
                         ctypes.byref(m), ctypes.byref(conv))
    return a.value, m.value, int(it), bool(conv.value)


def n_substeps(dt, p=None):
    lib, p = _load(), _prm(p)
    return int(lib.orc_n_substeps(_ptr(p), float(dt)))


# ---------------------------------------------------------------- point state
@dataclass
class State:
    """Per-point oracle state: X_as, X_am, the App. A variable X~ and the mode."""
    xas: np.ndarray
    xam: np.ndarray
    xt: np.ndarray
    mode: np.ndarray

    @classmethod
    def make(cls, xas, xam, xt=None, mode=None) -> "State":
        xas = np.array(xas, dtype=np.float64, copy=True).ravel()
        xam = np.array(xam, dtype=np.float64, copy=True).ravel()
        n = xas.size
        xt = np.zeros(n) if xt is None else np.array(xt, dtype=np.float64, copy=True).ravel()
        mode = (np.zeros(n, dtype=np.int32) if mode is None
                else np.array(mode, dtype=np.int32, copy=True).ravel())
        return cls(xas, xam, xt, mode)

    @classmethod
    def uniform(cls, n, xas=0.9, xam=0.0) -> "State":
        return cls.make(np.full(n, xas), np.full(n, xam))

    def copy(self) -> "State":
        return State(self.xas.copy(), self.xam.copy(), self.xt.copy(), self.mode.copy())

    @property
    def n(self) -> int:
        return self.xas.size


def fractions(state: State, T, p=None):
    """(X_as, X_am, X_beta, X_liq) with X_beta = 1 - g(T) - X_as - X_am."""
    lib, p = _load(), _prm(p)
    T = np.ascontiguousarray(np.broadcast_to(np.asarray(T, dtype=np.float64), (state.n,)))
    xb, xl = np.empty(state.n), np.empty(state.n)
    lib.orc_fractions(_ptr(p), state.n, _ptr(state.xas), _ptr(state.xam), _ptr(T), _ptr(xb), _ptr(xl))
    return state.xas.copy(), state.xam.copy(), xb, xl


def run_temps(state: State, T_hist, dt, p=None) -> State:
    """Advance every point through a given temperature history in place.

    ``T_hist`` has shape (n_steps + 1, n): row s is T^s of every point."""
    lib, p = _load(), _prm(p)
    T = np.ascontiguousarray(T_hist, dtype=np.float64)
    if T.ndim == 1:
        T = T[:, None].repeat(state.n, axis=1) if state.n > 1 else T[:, None]
        T = np.ascontiguousarray(T)
    assert T.shape[1] == state.n and T.shape[0] >= 1
    lib.orc_run_temps(_ptr(p), state.n, T.shape[0] - 1, float(dt), _ptr(T),
                      _ptr(state.xas), _ptr(state.xam), _ptr(state.xt), _ptr(state.mode))
    return state


def step(state: State, T0, T1, dt, p=None) -> State:
    """One step (the parameters' integrator) with per-point temperatures
    T0 = T^n, T1 = T^{n+1}."""
    T0 = np.broadcast_to(np.asarray(T0, dtype=np.float64), (state.n,))
    T1 = np.broadcast_to(np.asarray(T1, dtype=np.float64), (state.n,))
    return run_temps(state, np.stack([T0, T1]), dt, p)


# ------------------------------------------------------------ moving source
def _src_arrays(src):
    spec = np.array([src.A, src.k, src.alpha, src.T0, src.T_max, src.t_offset, src.z_tol],
                    dtype=np.float64)
    tracks = np.ascontiguousarray(src.tracks, dtype=np.float64).reshape(-1, 8)
    layers = np.ascontiguousarray(src.layers, dtype=np.float64).reshape(-1, 4)
    return spec, tracks, layers


def temperature(src, x, y, z, t):
    """Temperature of points (x, y, z) at global time t; returns (T, active)."""
    lib = _load()
    spec, tracks, layers = _src_arrays(src)
    x, y, z = (np.ascontiguousarray(np.atleast_1d(a), dtype=np.float64) for a in (x, y, z))
    n = x.size
    T, act = np.empty(n), np.empty(n, dtype=np.int32)
    lib.orc_temperature(_ptr(spec), _ptr(tracks), tracks.shape[0], _ptr(layers), layers.shape[0],
                        n, _ptr(x), _ptr(y), _ptr(z), float(t), _ptr(T), _ptr(act))
    return T, act


def run_track(state: State, src, x, y, z, n0, n_steps, dt, p=None):
    """Advance points at (x, y, z) from time level n0 by n_steps under the
    moving source; returns the temperature at the final level."""
    lib, p = _load(), _prm(p)
    spec, tracks, layers = _src_arrays(src)
    x, y, z = (np.ascontiguousarray(np.atleast_1d(a), dtype=np.float64) for a in (x, y, z))
    assert x.size == state.n
    T_last = np.empty(state.n)
    lib.orc_run_track(_ptr(p), _ptr(spec), _ptr(tracks), tracks.shape[0], _ptr(layers),
                      layers.shape[0], state.n, _ptr(x), _ptr(y), _ptr(z), int(n0), int(n_steps),
                      float(dt), _ptr(state.xas), _ptr(state.xam), _ptr(state.xt),
                      _ptr(state.mode), _ptr(T_last))
    return T_last


def run_track_windows(state: State, src, x, y, z, n0, n_steps, dt, window=8, band_half=40.0,
                      p=None, return_fixed=False, stride=1, group=1):
    """The hybrid path's window form with a zero network (see
    orc_run_track_windows): windows of window x stride levels whose start
    and samples (every stride-th level) pass the band test apply only the
    correction g at the samples in turn; the others take the explicit steps;
    points on the alpha_s plateau's fixed point keep their state over
    windows sampled below T_as,end; within a group of `group` consecutive
    points one explicit window sends the group's g-only windows to the
    explicit steps.  Returns per point the number of g-only windows (and,
    with return_fixed, of fixed-point windows)."""
    assert window >= 1 and stride >= 1 and group >= 1
    lib, p = _load(), _prm(p)
    spec, tracks, layers = _src_arrays(src)
    x, y, z = (np.ascontiguousarray(np.atleast_1d(a), dtype=np.float64) for a in (x, y, z))
    assert x.size == state.n
    n_mlp = np.zeros(state.n, dtype=np.int64)
    n_fixed = np.zeros(state.n, dtype=np.int64)
    lib.orc_run_track_windows(_ptr(p), _ptr(spec), _ptr(tracks), tracks.shape[0], _ptr(layers),
                              layers.shape[0], state.n, _ptr(x), _ptr(y), _ptr(z), int(n0),
                              int(n_steps), float(dt), int(window), int(stride),
                              float(band_half), int(group),
                              _ptr(state.xas), _ptr(state.xam), _ptr(state.xt), _ptr(state.mode),
                              _ptr(n_mlp), _ptr(n_fixed))
    return (n_mlp, n_fixed) if return_fixed else n_mlp
