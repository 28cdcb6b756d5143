"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/ms.h declares, its struct layouts match the
binding, its defaults are the paper's tables, and argument validation that
happens before any device work returns the documented codes."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2402_17580_gb300 as ms
from paper_2402_17580_gb300 import _binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ms_\w+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    lib = ms.load()
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", ms.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\b(ms_\w+)\b", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_struct_layouts_match():
    lib = ms.load()
    for i, s in enumerate(B.STRUCTS):
        assert lib.ms_struct_size(i) == ctypes.sizeof(s), s.__name__
    assert lib.ms_struct_size(99) == 0


def test_defaults_are_the_paper_tables(golden):
    p = ms.default_params()
    t2, t3 = golden["table2_micro"], golden["table3_diffusion"]
    for k, v in t2.items():
        if not k.startswith("_"):
            assert getattr(p, k) == v, k
    for k, v in t3.items():
        if not k.startswith("_"):
            assert getattr(p, k) == v, k
    assert p.T_reg == golden["T_reg"]["value"]
    assert p.init_exit == golden["init_exit"]["value"]
    assert p.precision == ms.MS_F32


def test_defaults_agree_with_the_oracle():
    import oracle
    p = ms.default_params()
    for k, v in oracle.DEFAULTS.items():
        assert float(getattr(p, k)) == v, k


def test_strerror_and_version():
    lib = ms.load()
    assert b"sm_103a" in lib.ms_version()
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert lib.ms_strerror(code)
    assert lib.ms_strerror(-99) == b"unknown status"


def test_validation_before_device_work():
    lib = ms.load()
    h = ctypes.c_void_p()
    p = ms.default_params()
    assert lib.ms_create(ctypes.byref(p), 0, ctypes.byref(h)) == -1
    assert lib.ms_create(None, 10, ctypes.byref(h)) == -1
    bad = ms.default_params(c_b=1.0)
    assert lib.ms_create(ctypes.byref(bad), 10, ctypes.byref(h)) == -1
    bad = ms.default_params(steps_per_launch=0)
    assert lib.ms_create(ctypes.byref(bad), 10, ctypes.byref(h)) == -1
    bad = ms.default_params(block_threads=48)
    assert lib.ms_create(ctypes.byref(bad), 10, ctypes.byref(h)) == -1
    bad = ms.default_params(integrator=7)
    assert lib.ms_create(ctypes.byref(bad), 10, ctypes.byref(h)) == -1
    bad = ms.default_params(integrator=1, precision=2)          # implicit + compensated
    assert lib.ms_create(ctypes.byref(bad), 10, ctypes.byref(h)) == -7
    bad = ms.default_params(integrator=1, fp_max_iter=0)
    assert lib.ms_create(ctypes.byref(bad), 10, ctypes.byref(h)) == -1
    tp = ms.thermal_params(k_ms=-1.0)
    g = ms._binding.Grid((ctypes.c_double * 3)(0, 0, 0), (ctypes.c_double * 3)(1e-5, 1e-5, -1e-5),
                         (ctypes.c_int32 * 3)(4, 4, 4), 0)
    assert lib.ms_thermal_create(ctypes.byref(tp), ctypes.byref(g), ctypes.byref(h)) == -1
    assert lib.ms_thermal_create(None, ctypes.byref(g), ctypes.byref(h)) == -1
    assert lib.ms_thermal_params_default(None) == -1
    assert lib.ms_params_default(None) == -1
    for fn, args in (("ms_set_points", (None, None, 1)), ("ms_set_state", (None, None, None, None)),
                     ("ms_step", (None, None, None, 1e-5, 0)), ("ms_run_track", (None, None, 1, 1e-5)),
                     ("ms_get_fractions", (None, None, None, None, None)), ("ms_get_aux", (None, None)),
                     ("ms_stats", (None, None)), ("ms_synchronize", (None,))):
        assert getattr(lib, fn)(*args) == -1, fn
    w = (ctypes.c_float * 5187)()
    for act, stride in ((2, 1), (-1, 1), (0, 0), (1, 3), (1, 32), (1, 12)):
        assert lib.ms_surrogate_create_ex(w, act, stride, ctypes.byref(h)) == -1, (act, stride)
        assert not h.value
    a, r = ctypes.c_int32(), ctypes.c_int32()
    assert lib.ms_surrogate_get_config(None, ctypes.byref(a), ctypes.byref(r)) == -1
    lib.ms_destroy(None)


def test_product_and_oracle_share_no_code():
    """The CUDA path never imports the oracle and the oracle never imports the
    CUDA path; only workloads/ (inputs, no model arithmetic) serves both."""
    pkg = os.path.join(ROOT, "paper_2402_17580_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.findall(r"(?:import|from)\s+(\w+)", src), f
                assert "ms_oracle" not in src, f
    osrc = open(os.path.join(ROOT, "oracle", "ms_oracle.c")).read()
    assert "#include \"" not in osrc
    opy = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    imports = re.findall(r"^\s*(?:import|from)\s+([\w.]+)", opy, flags=re.M)
    assert not [m for m in imports if m.split(".")[0] in ("paper_2402_17580_gb300", "workloads")]


def test_farfield_table_is_lagrange_interpolation_at_chebyshev_nodes():
    """The far field's table (host-only): the nodes are the 8 Chebyshev points
    of the first kind on [0, 1], and the weights at the tile's 128 points
    t_i = i / 127 reproduce every polynomial of degree <= 7 (so they sum to
    1), up to FP32 rounding of the stored table."""
    import numpy as np
    from paper_2402_17580_gb300._binding import farfield_table
    w, s = farfield_table()
    k = np.arange(8)
    np.testing.assert_allclose(s, 0.5 * (1.0 - np.cos((2 * k + 1) * np.pi / 16)), atol=1e-7)
    t = np.arange(128) / 127.0
    for m in range(8):
        np.testing.assert_allclose((w * (s.astype(np.float64)[:, None] ** m)).sum(axis=0), t ** m,
                                   atol=2e-6)
    # the Lebesgue function sum_k |w_k(t)| bounds how much FP32 error in the
    # node sums the interpolation can amplify; for 8 Chebyshev nodes it is
    # about (2 / pi) ln 8 + 1, its largest at the tile's ends t = 0, 1
    leb = np.abs(w.astype(np.float64)).sum(axis=0)
    assert leb.max() < 2.6, leb.max()
    with pytest.raises(ms.MSError):
        out = (ctypes.c_float * 10)()
        B._check(ms.load().ms_farfield_table(out, 10), "ms_farfield_table")


def test_params_check_rules_on_the_host():
    """ms_params_check applies ms_create's parameter checks without a GPU: the
    paper's defaults pass, and each rule rejects one field changed away from
    them, with the code the header names."""
    from paper_2402_17580_gb300 import _binding as b
    nan, inf = float("nan"), float("inf")
    b.check_params(b.default_params())
    b.check_params(b.default_params(integrator=b.MS_IMPLICIT, precision=b.MS_F64))
    b.check_params(b.default_params(farfield_dist=5e-3))
    invalid = [dict(T_s=0.0), dict(T_l=1800.0), dict(T_s=nan), dict(T_as_end=1300.0),
               dict(T_am_start=-1.0), dict(T_inf=0.0), dict(k_alpha_eq=0.0), dict(k_am_eq=-1.0),
               dict(k1=inf), dict(k2=nan), dict(k3=0.0), dict(f=0.0), dict(c_as=1.0),
               dict(c_b=0.5), dict(T_reg=0.0), dict(init_exit=-1.0), dict(init_exit_floor=nan),
               dict(T_thr=inf), dict(precision=7), dict(steps_per_launch=0),
               dict(steps_per_launch=100000), dict(block_threads=48), dict(block_threads=512),
               dict(integrator=2), dict(farfield_dist=-1.0), dict(farfield_dist=nan),
               dict(tile_order=2), dict(tile_order=-1),
               dict(integrator=b.MS_IMPLICIT, fp_eps_rel=0.0),
               dict(integrator=b.MS_IMPLICIT, fp_eps_abs=-1.0),
               dict(integrator=b.MS_IMPLICIT, fp_max_iter=0),
               dict(integrator=b.MS_IMPLICIT, dt_sub=nan)]
    for bad in invalid:
        with pytest.raises(b.MSError, match="INVALID_ARG"):
            b.check_params(b.default_params(**bad))
    b.check_params(b.default_params(farfield_dist=5e-3, precision=b.MS_F64))
    b.check_params(b.default_params(farfield_dist=5e-3, integrator=b.MS_IMPLICIT))
    unsupported = [dict(integrator=b.MS_IMPLICIT, precision=b.MS_KAHAN),
                   dict(integrator=b.MS_IMPLICIT, precision=b.MS_F64ACC)]
    for bad in unsupported:
        with pytest.raises(b.MSError, match="UNSUPPORTED"):
            b.check_params(b.default_params(**bad))
    assert b.load().ms_params_check(None) == -1


def test_every_entry_point_states_its_errors():
    """Each declaration in include/ms.h has its own comment, and every call
    that returns a status names its errors there."""
    import re
    hdr = open(os.path.join(ROOT, "include", "ms.h")).read()
    missing = []
    for m in re.finditer(r"^(int|void|const char\*|size_t)\s+(ms_\w+)\(", hdr, re.M):
        before = hdr[:m.start()].rstrip()
        if not before.endswith("*/"):
            missing.append(m.group(2) + ": no comment")
            continue
        comment = before[before.rfind("/*"):]
        if m.group(1) == "int" and not re.search(r"Errors?:|MS_ERR_", comment):
            missing.append(m.group(2) + ": no errors")
    assert not missing, missing
