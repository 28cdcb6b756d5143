"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of oracle/ms_oracle.c (a dropped term,
a wrong sign, index or exponent, a transposed operand), compiles it on the
CPU and runs tests/test_oracle_pins.py against it; the pins must fail.  The
same is done for the Python parts: the thermal reference oracle/thermal.py
(pins: tests/test_thermal_oracle.py), the surrogate's network oracle/mlp.py
(pins: the network tests of tests/test_mlp_oracle.py) and the coarsening
criterion oracle/coarsen.py (pins: tests/test_coarsen_oracle.py).
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ms_oracle.c")
THERMAL_SRC = os.path.join(ROOT, "oracle", "thermal.py")

MUTANTS = {
    "xalpha_eq_sign": ("exp(-p[P_K_ALPHA_EQ] * (p[P_T_AS_START] - T))",
                       "exp(p[P_K_ALPHA_EQ] * (p[P_T_AS_START] - T))"),
    "xam0_eq_constant": ("exp(-p[P_K_AM_EQ] * (p[P_T_AM_START] - T))",
                         "exp(-p[P_K_ALPHA_EQ] * (p[P_T_AM_START] - T))"),
    "xam_eq_factor": ("(XMAX - xas) / XMAX", "(XMAX + xas) / XMAX"),
    "k_beta_drops_f": ("double k = k_alpha_s(p, T), kb = p[P_F] * k;",
                       "double k = k_alpha_s(p, T), kb = k;"),
    "r3_exponents_swapped": ("powpos(XMAX - xa, (cb - 1.0) / cb) * powpos(xa - xeq, (cb + 1.0) / cb)",
                             "powpos(XMAX - xa, (cb + 1.0) / cb) * powpos(xa - xeq, (cb - 1.0) / cb)"),
    "r1_exponents_swapped": ("k * powpos(xas, (ca - 1.0) / ca) * powpos(xeq - xa, (ca + 1.0) / ca)",
                             "k * powpos(xas, (ca + 1.0) / ca) * powpos(xeq - xa, (ca - 1.0) / ca)"),
    "r2_dropped": ("*das = r1 + r2 - r3;", "*das = r1 - r3;"),
    "rescale_inverted": ("double s = XMAX / xa;", "double s = xa / XMAX;"),
    "regularisation_sign": ("(p[P_T_AS_START] + p[P_T_REG] - T) / p[P_T_REG]",
                            "(T - p[P_T_AS_START]) / p[P_T_REG]"),
    "dissolution_dropped": ("    xam = v > 0.0 ? v : 0.0;\n", "    (void)v;\n"),
    "rates_at_T1": ("rates(p, T0, xas, xam, &das, &dam);", "rates(p, T1, xas, xam, &das, &dam);"),
    "logistic_power": ("pow(xi / (1.0 - xi), 1.0 / c)", "pow(xi / (1.0 - xi), c)"),
    "appendix_shift_dropped": ("double D = (1.0 - xeq0) - 0.1;", "double D = 1.0 - xeq0;"),
    "beta_rate_in_init": ("xt = logistic_step(xt, D, kb, p[P_C_B], dt);",
                          "xt = logistic_step(xt, D, k, p[P_C_B], dt);"),
    "liquid_fraction_flipped": ("return (T - p[P_T_S]) / (p[P_T_L] - p[P_T_S]);",
                                "return (p[P_T_L] - T) / (p[P_T_L] - p[P_T_S]);"),
    "source_full_space": ("(2.0 * M_PI * spec[S_K] * R)", "(4.0 * M_PI * spec[S_K] * R)"),
    "source_xi_sign": ("exp(-tr[TR_V] * (R + xi)", "exp(-tr[TR_V] * (R - xi)"),
    "source_depth_dropped": ("dx * dx + dy * dy + dz * dz", "dx * dx + dy * dy"),
    "interlayer_dropped": ("double T = spec[S_T0] + scale * sum;", "double T = spec[S_T0] + sum;"),
    "clamp_dropped": ("  if (xas < 0.0) xas = 0.0;\n", ""),
    "cn_half_dropped": ("double nas = xas + 0.5 * dt * (das + das0);",
                        "double nas = xas + dt * (das + das0);"),
    "cn_old_rates_at_T1": ("rates(p, T0, xas, xam, &das0, &dam0);",
                           "rates(p, T1, xas, xam, &das0, &dam0);"),
    "substep_temperature_frozen": ("const double Tb = T0 + (T1 - T0) * ((double)(s + 1) / (double)ns);",
                                   "const double Tb = T0 + (T1 - T0) * ((double)s / (double)ns);"),
    "xam_clamp_dropped": ("  if (xam < 0.0) xam = 0.0;\n", ""),
    "cap_floor_dropped": ("    if (cap < 0.0) cap = 0.0;\n", ""),
    "cap_from_T_reg_up": ("  if (T > p[P_T_AS_START]) {\n    double cap",
                          "  if (T > p[P_T_AS_START] + p[P_T_REG]) {\n    double cap"),
    "dissolution_ignores_X_as": ("    double v = xeq - xas;\n", "    double v = xeq;\n"),
    "formation_literal_by_default": ("else if (e > xam) xam = e;", "else xam = e;"),
    "xam0_eq_cap_dropped": ("return v < XMAX ? v : XMAX;", "return v;"),
    "init_exit_without_dt": ("xt * dt > p[P_INIT_EXIT]", "xt > p[P_INIT_EXIT]"),
    "appendix_unshifted_alpha_s": ("    nas = XMAX - xt;\n", "    nas = 1.0 - xt;\n"),
    "appendix_entry_with_martensite": ("&& XMAX - xa <= 0.0 && xam == 0.0) {\n    mode = MODE_AS_TO_B;",
                                       "&& XMAX - xa <= 0.0) {\n    mode = MODE_AS_TO_B;"),
    "cap_keeps_initiation": ("if (nas < before) mode = MODE_NONE;", "if (0) mode = MODE_NONE;"),
    "ba_initiation_drops_r2": ("nas = logistic_step(xas, D, k, ca, dt) + dt * r2;",
                               "nas = logistic_step(xas, D, k, ca, dt);"),
    "unstarted_tracks_heat": ("|| tl < tr[TR_TS]) continue;", ") continue;"),
    "other_layers_tracks_heat": ("if ((int32_t)tr[TR_LAYER] != l || tl < tr[TR_TS]) continue;",
                                 "if (tl < tr[TR_TS]) continue;"),
    "undeposited_points_advance": ("if (a1) advance(", "(void)a1; advance("),
    "interlayer_factor_goes_negative": ("    if (scale < 0.0) scale = 0.0;\n", ""),
    "cn_iterate_rates_at_T0": ("rates(p, T1, nas, nam, &das1, &dam1);",
                               "rates(p, T0, nas, nam, &das1, &dam1);"),
    "cn_iterate_without_g": ("    correct(p, T1, &nas, &nam);\n    double das1", "    double das1"),
    "cn_stops_after_one_iteration": ("    if (e < 1.0) {", "    if (1) {"),
    "substeps_round_up_decimal_multiples": ("ceil(dt / p[P_DT_SUB] - 1e-9)", "ceil(dt / p[P_DT_SUB])"),
    "substep_length_is_dt_sub": ("const double h = dt / (double)ns;",
                                 "const double h = p[P_DT_SUB] > 0.0 ? p[P_DT_SUB] : dt;"),
    "implicit_without_beta_to_alpha_initiation": ("    if (xa < xeq0 && *xas == 0.0) init = 1;\n", ""),
    "implicit_without_alpha_to_beta_initiation": (
        "    if (xa > xeq0 && XMAX - xa <= 0.0 && *xam == 0.0) init = 1;\n", ""),
    "implicit_initiation_over_the_whole_step": ("      point_step(p, Ta, Tb, h, xas, xam, xt, mode);",
                                                "      point_step(p, T0, T1, h, xas, xam, xt, mode);"),
}


# mistakes in the window form of the hybrid path (orc_run_track_windows),
# caught by tests/test_mlp_oracle.py
WINDOW_MUTANTS = {
    "fixed_point_bound_T_as_start": ("cool &= Ti[l] < p[P_T_AS_END];",
                                     "cool &= Ti[l] < p[P_T_AS_START];"),
    "fixed_point_any_alpha": ("xas[i] == 0.9 && xam[i] == 0.0", "xas[i] >= 0.5"),
    "windows_skip_correction": (
        "for (int64_t l = stride; l <= K; l += stride) correct(p, Ti[l], &xas[i], &xam[i]);",
        "(void)0;"),
    "windows_correct_at_last_level_only": (
        "for (int64_t l = stride; l <= K; l += stride) correct(p, Ti[l], &xas[i], &xam[i]);",
        "correct(p, Ti[K], &xas[i], &xam[i]);"),
    "band_misses_regularisation_end": (" || fabs(T - (p[P_T_AS_START] + p[P_T_REG])) < h) return 1;",
                                       ") return 1;"),
    "band_misses_melt": ("  if (!(T <= p[P_T_S] - h)) return 1;\n", ""),
    "band_ignores_start_level": ("int band = in_band(p, Ti[0], band_half), cool",
                                 "int band = 0, cool"),
    "tail_window_to_network": ("else if (K == len && all_act && !band", "else if (all_act && !band"),
    "jump_rule_dropped": (" || !(fabs(Ti[l] - Ti[l - stride]) <= band_half)", ""),
    "group_rule_ignored": ("} else if (kind[k] == 2 && !any_explicit) {", "} else if (kind[k] == 2) {"),
    "vertex_rule_dropped": ("band |= extreme_near(p, Ti[l - 2 * stride], Ti[l - stride], Ti[l]);",
                            "(void)0;"),
    "vertex_between_outer_samples_only": ("!(fabs(s) <= 4.0 * fabs(k))", "!(fabs(s) <= 2.0 * fabs(k))"),
    "initiation_window_to_network": ("&& !band && mode[i] == MODE_NONE)\n", "&& !band)\n"),
    "fixed_point_ignores_initiation": ("cool && mode[i] == MODE_NONE && xas[i] == 0.9",
                                       "cool && xas[i] == 0.9"),
}


def _run_pins_on_mutant(name, old, new, tmp_path, pins):
    """The C oracle: compile the mutant and run the pins against it; returns
    (caught, message)."""
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fopenmp",
                    "-shared", "-fPIC", str(mut), "-o", str(lib), "-lm"], check=True)
    env = dict(os.environ, MS_ORACLE_LIB=str(lib), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode != 0, f"pins did not catch mutant {name}:\n{r.stdout[-2000:]}"


THERMAL_MUTANTS = {
    "face_mean_arithmetic": ("2.0 * a * b / np.where(s > 0.0, s, 1.0)", "0.5 * s"),
    "radiation_ambient_dropped": ("(Tt ** 4 - p.T_inf ** 4)", "Tt ** 4"),
    "radiation_on_bottom": ("flux[g.top] -= p.emissivity", "flux[g.bottom] -= p.emissivity"),
    "dirichlet_dropped": ("        Tn[g.bottom] = p.T0\n", "        pass\n"),
    "cap_dropped": ("        Tn = np.minimum(Tn, p.T_max)\n", "        pass\n"),
    "substeps_past_stability": ("dt / (0.9 * dt_stab)", "dt / (2.5 * dt_stab)"),
    "z_face_area": ("(dx * dy / dz)", "(dx * dz / dy)"),
    "x_face_area": ("(dy * dz / dx)", "(dx * dz / dy)"),
    "source_normalisation_halved": ("2.0 * W / (math.pi", "W / (math.pi"),
    "powder_layer_inclusive": ("inside = (depth >= 0.0) & (depth < p.h_powder)",
                               "inside = (depth >= 0.0) & (depth <= p.h_powder)"),
    "consolidation_not_running_max": ("rcn = np.maximum(rc, liquid_fraction(p, Tn))",
                                      "rcn = liquid_fraction(p, Tn)"),
    "conductivity_swapped": ("(1.0 - rc) * p.k_p + rc * p.k_ms", "rc * p.k_p + (1.0 - rc) * p.k_ms"),
    "source_at_substep_end": ("ts = t + s * h", "ts = t + (s + 1) * h"),
    "track_runs_to_layer_end": ("            t_end = tracks[j + 1, 6]", "            t_end = t_end"),
    "laser_direction_reversed": ("tr[0] + tr[2] * d", "tr[0] - tr[2] * d"),
}

_IMPORT_GUARD = """import os
from oracle import {module}


def pytest_configure(config):
    here = os.path.dirname(os.path.abspath(__file__))
    assert os.path.abspath({module}.__file__).startswith(here), {module}.__file__
"""


def _run_py_pins_on_mutant(module, name, old, new, tmp_path, pins, select=None):
    """A Python part of the oracle: the mutant goes into a package ``oracle``
    of its own beside a copy of the pins, so that the pins import it and not
    the real one (a conftest checks that); the repository stays on the path
    for the workload generators.  Returns (caught, message)."""
    src = open(os.path.join(ROOT, "oracle", module + ".py")).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    pkg = tmp_path / "oracle"
    pkg.mkdir()
    (pkg / "__init__.py").write_text("")
    (pkg / (module + ".py")).write_text(src.replace(old, new))
    (tmp_path / "conftest.py").write_text(_IMPORT_GUARD.format(module=module))
    (tmp_path / pins).write_text(open(os.path.join(ROOT, "tests", pins)).read())
    env = dict(os.environ, PYTHONPATH=ROOT)
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
           "--rootdir", str(tmp_path), str(tmp_path / pins)]
    if select:
        cmd += ["-k", select]
    r = subprocess.run(cmd, cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=600)
    # 1: a pin failed (a conftest that rejects the import ends with another code)
    return r.returncode == 1, f"pins did not catch mutant {name}:\n{r.stdout[-2000:]}"


# mistakes in the surrogate's reference network, caught by the network pins
# of tests/test_mlp_oracle.py (its window-form pins need the compiled oracle)
MLP_MUTANTS = {
    "layout_transposed": ("p[OFF_W1:OFF_B1].reshape(N_H, N_IN)",
                          "p[OFF_W1:OFF_B1].reshape(N_IN, N_H).T"),
    "gelu_constant": ("GELU_A = 0.044715", "GELU_A = 0.047715"),
    "gelu_grad_term_dropped": ("(1.0 + 3.0 * GELU_A * x ** 2)", "1.0"),
    "round_half_up": ("(u + 0x7FFF + lsb)", "(u + 0x7FFF)"),
    "input_not_rounded": ("x = rnd(np.asarray(X, dtype=np.float64))",
                          "x = np.asarray(X, dtype=np.float64)"),
    "W1_not_rounded": ("W1, W2, W3 = rnd(W1), rnd(W2), rnd(W3)", "W2, W3 = rnd(W2), rnd(W3)"),
    "hidden1_not_rounded": ("a1 = rnd(f(h1))", "a1 = f(h1)"),
    "hidden2_not_rounded": ("a2 = rnd(f(h2))", "a2 = f(h2)"),
    "relu_grad_one_at_kink": ("(np.asarray(x) > 0.0)", "(np.asarray(x) >= 0.0)"),
    "relu_leaky": ("np.maximum(x, 0.0)", "np.maximum(x, 0.01 * x)"),
    "relu_grad_gelu": ('"relu": (relu, relu_grad)', '"relu": (relu, gelu_grad)'),
    "bias_b2_dropped": ("h2 = a1 @ W2.T + b2", "h2 = a1 @ W2.T"),
    "loss_mean_over_samples_only": ("loss = float(np.sum(r * r) / (N_OUT * n))",
                                    "loss = float(np.sum(r * r) / n)"),
    "gradient_unrounded_input": ("g[OFF_W1:OFF_B1] = (dh1.T @ x).ravel()",
                                 "g[OFF_W1:OFF_B1] = (dh1.T @ np.asarray(X, dtype=np.float64)).ravel()"),
    "backprop_unrounded_W3": ("dh2 = (dy @ W3) * fg(h2)",
                              "dh2 = (dy @ unpack(params)[4]) * fg(h2)"),
    "gradient_sign": ("dy = 2.0 * r / (N_OUT * n)", "dy = -2.0 * r / (N_OUT * n)"),
}


# mistakes in the coarsening criterion, caught by tests/test_coarsen_oracle.py
COARSEN_MUTANTS = {
    "span_half_open": ("slice(i << level, ((i + 1) << level) + 1)", "slice(i << level, (i + 1) << level)"),
    "strict_tolerance": ("1 if all(r <= tol for r in ranges)", "1 if all(r < tol for r in ranges)"),
    "beta_ignored": ("for a in (x_as, x_am, x_beta)]", "for a in (x_as, x_am, x_am)]"),
    "count_rounds_up": ("return (n - 1) // (1 << level)", "return -(-(n - 1) // (1 << level))"),
    "flat_axis_empty": ("    if n == 1:\n        return 1\n", ""),
    "x_y_transposed": (".reshape(nz, ny, nx) for a", ".reshape(nz, nx, ny) for a"),
    "min_over_one_phase": ("f[sk, sj, si].max() - f[sk, sj, si].min()) for f in fields]",
                           "f[sk, sj, si].max() - fields[0][sk, sj, si].min()) for f in fields]"),
    "level_width_off_by_one": ("def _span(i, level, n):\n    if n == 1:\n        return slice(0, 1)\n    return slice(i << level,",
                               "def _span(i, level, n):\n    if n == 1:\n        return slice(0, 1)\n    level -= 1\n    return slice(i << level,"),
}


# Every mutant is a compile and a pytest run of its own; they run in parallel
# threads (each waits on its subprocesses) once per module, and each test
# reads its mutant's outcome.
def _jobs():
    jobs = {}
    for name, (old, new) in MUTANTS.items():
        jobs[("c", name)] = (_run_pins_on_mutant, (name, old, new), "test_oracle_pins.py", None)
    for name, (old, new) in WINDOW_MUTANTS.items():
        jobs[("window", name)] = (_run_pins_on_mutant, (name, old, new), "test_mlp_oracle.py", None)
    for module, table, pins, select in (("thermal", THERMAL_MUTANTS, "test_thermal_oracle.py", None),
                                        ("mlp", MLP_MUTANTS, "test_mlp_oracle.py", "not windows"),
                                        ("coarsen", COARSEN_MUTANTS, "test_coarsen_oracle.py", None)):
        for name, (old, new) in table.items():
            jobs[(module, name)] = (_run_py_pins_on_mutant, (module, name, old, new), pins, select)
    return jobs


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    from concurrent.futures import ThreadPoolExecutor
    jobs = _jobs()
    dirs = {key: tmp_path_factory.mktemp("mutant_" + "_".join(key)) for key in jobs}

    def run(key):
        fn, args, pins, select = jobs[key]
        d = dirs[key]
        if fn is _run_pins_on_mutant:
            return fn(*args, d, pins)
        return fn(*args, d, pins, select=select)

    with ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        futures = {key: ex.submit(run, key) for key in jobs}
        return {key: f.result() for key, f in futures.items()}


def _check(outcomes, key):
    caught, message = outcomes[key]
    assert caught, message


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, outcomes):
    _check(outcomes, ("c", name))


@pytest.mark.parametrize("name", sorted(WINDOW_MUTANTS))
def test_window_pins_catch_mutant(name, outcomes):
    _check(outcomes, ("window", name))


@pytest.mark.parametrize("name", sorted(THERMAL_MUTANTS))
def test_thermal_pins_catch_mutant(name, outcomes):
    _check(outcomes, ("thermal", name))


@pytest.mark.parametrize("name", sorted(MLP_MUTANTS))
def test_network_pins_catch_mutant(name, outcomes):
    _check(outcomes, ("mlp", name))


@pytest.mark.parametrize("name", sorted(COARSEN_MUTANTS))
def test_coarsen_pins_catch_mutant(name, outcomes):
    _check(outcomes, ("coarsen", name))
