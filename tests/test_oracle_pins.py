"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it pins and the mistake it would catch.  None of
them re-runs the oracle's own formula as the expected value: expectations come
from the paper's printed numbers (tests/golden/paper_values.json), from closed
forms checked against an independent ODE integration (scipy), from invariants,
limits and continuity, from the heat equation the moving source must satisfy,
or from convergence under dt-halving.
"""
import math

import numpy as np
import pytest

import oracle as orc
import workloads as wl
from workloads import Grid, HeatSource, NEVER

P = orc.params()


# ----------------------------------------------------------------- constants
def test_defaults_are_the_paper_tables(golden):
    """Tables 1-3, T_reg (Sec. 2.2), the App. A exit threshold."""
    t2, t3 = golden["table2_micro"], golden["table3_diffusion"]
    for k in ("T_as_start", "T_as_end", "T_am_start", "T_inf", "k_alpha_eq", "k_am_eq", "T_s", "T_l"):
        assert orc.DEFAULTS[k] == t2[k], k
    for k in ("c_as", "c_b", "k1", "k2", "k3", "f"):
        assert orc.DEFAULTS[k] == t3[k], k
    assert orc.DEFAULTS["T_reg"] == golden["T_reg"]["value"]
    assert orc.DEFAULTS["init_exit"] == golden["init_exit"]["value"]


# ------------------------------------------------------------- equilibria
def test_equilibria_sum_at_T_inf(golden):
    """Sec. 2.2 prints that X_alpha^eq + X_am,0^eq = 1.8 at T = T_inf (catches a
    wrong branch, sign or constant in either equilibrium)."""
    s = orc.xalpha_eq(293.0) + orc.xam0_eq(293.0)
    assert abs(s - golden["equilibria_sum_at_T_inf"]["value"]) < 1e-3


def test_xalpha_eq_shape():
    """eq:equilibrium_phase_as: 0.9 below T_as,end, 0 above T_as,start,
    continuous at T_as,start, monotone, and within 5e-4 of 0.9 at T_as,end
    (the Table 2 constants make the branches meet; a swapped constant or
    sign breaks this)."""
    T = np.linspace(200, 2000, 3601)
    x = orc.xalpha_eq(T)
    assert np.all((x >= 0) & (x <= 0.9))
    assert np.all(np.diff(x) <= 1e-15)
    assert orc.xalpha_eq(1273.0 - 1e-9) < 1e-10 and orc.xalpha_eq(1273.5) == 0.0
    assert orc.xalpha_eq(934.999) == 0.9
    assert abs(orc.xalpha_eq(935.0) - 0.9) < 5e-4
    # Koistinen-Marburger law: ln(1 - X) linear in T with slope k_alpha_eq (Table 2)
    Tm = np.linspace(950, 1250, 7)
    slope = np.diff(np.log(1 - orc.xalpha_eq(Tm))) / np.diff(Tm)
    assert np.allclose(slope, P[orc.PARAM_NAMES.index("k_alpha_eq")], rtol=1e-9)


def test_xam0_eq_shape():
    """eq:equilibrium_phase_am0 (reading A1): 0 above T_am,start, continuous
    there, monotone, ~0.9 at T_inf, capped at 0.9 (A2)."""
    T = np.linspace(200, 1500, 2601)
    x = orc.xam0_eq(T)
    assert np.all((x >= 0) & (x <= 0.9))
    assert np.all(np.diff(x) <= 1e-15)
    assert orc.xam0_eq(848.0) == 0.0 and orc.xam0_eq(847.9999) < 1e-5
    assert orc.xam0_eq(900.0) == 0.0 and orc.xam0_eq(1200.0) == 0.0  # A1: not only above T_as,start
    assert abs(orc.xam0_eq(293.5) - 0.9) < 2e-3
    Tm = np.linspace(400, 800, 5)
    slope = np.diff(np.log(1 - orc.xam0_eq(Tm))) / np.diff(Tm)
    assert np.allclose(slope, P[orc.PARAM_NAMES.index("k_am_eq")], rtol=1e-9)


def test_xam_eq_respects_alpha_bound(golden):
    """eq:equilibrium_phase_am: X_as + X_am^eq <= 0.9 for every T and X_as."""
    for T in np.linspace(250, 900, 27):
        for xas in np.linspace(0, 0.9, 19):
            assert xas + orc.xam_eq(T, xas) <= golden["alpha_max"]["value"] + 1e-12


def test_rate_constant_sigmoid():
    """k_as(T) = k1 / (1 + exp(-k3 (T - k2))): midpoint k1/2 at k2, limits 0 and k1,
    slope k1 k3 / 4 at k2."""
    assert abs(orc.k_alpha_s(850.0) - 0.294 / 2) < 1e-15
    assert orc.k_alpha_s(5000.0) == pytest.approx(0.294, rel=1e-12)
    assert orc.k_alpha_s(100.0) < 1e-10
    h = 1e-3
    slope = (orc.k_alpha_s(850 + h) - orc.k_alpha_s(850 - h)) / (2 * h)
    assert slope == pytest.approx(0.294 * 0.0337 / 4, rel=1e-6)


# -------------------------------------------------- generalised logistic ODE
def closed_form(t, D, k, c, X0=0.0):
    """X(t) of dX/dt = k X^((c-1)/c) (D - X)^((c+1)/c), i.e. of
    dxi/dt = D k xi^((c-1)/c) (1-xi)^((c+1)/c) with xi = X / D:
    (xi/(1-xi))^(1/c) grows linearly at rate D k / c."""
    u0 = 0.0 if X0 == 0 else (X0 / D / (1 - X0 / D)) ** (1 / c)
    y = (u0 + D * k * t / c) ** c
    return D * y / (1 + y)


@pytest.mark.parametrize("c,X0", [(2.51, 0.05), (11.0, 1e-3), (11.0, 0.2)])
def test_closed_form_solves_the_ode(c, X0):
    """The closed form used by the pins below solves the ODE (independent
    integration with scipy's adaptive Runge-Kutta)."""
    from scipy.integrate import solve_ivp
    D, k = 0.6, 0.8
    # the paper's rate form: dX/dt = k X^((c-1)/c) (D - X)^((c+1)/c)
    f = lambda t, y: [k * max(y[0], 0) ** ((c - 1) / c) * max(D - y[0], 0) ** ((c + 1) / c)]
    ts = np.array([1.0, 5.0, 20.0])
    sol = solve_ivp(f, (0, ts[-1]), [X0], t_eval=ts, rtol=1e-11, atol=1e-14, method="DOP853")
    assert np.allclose(sol.y[0], [closed_form(t, D, k, c, X0) for t in ts], rtol=1e-7, atol=1e-12)


def test_logistic_step_is_exact():
    """eq:analytical_solution_beta is exact for constant k: stepping it with any
    dt lands on the closed form (App. A)."""
    D, k, c = 0.5087, 1.117, 11.0
    for dt in (1e-5, 0.37, 2.0):
        X, t = 0.0, 0.0
        for _ in range(20):
            X = orc.logistic_step(X, D, k, c, dt)
            t += dt
        assert X == pytest.approx(closed_form(t, D, k, c), rel=1e-9, abs=1e-300)


# ------------------------------------------------------ P1: beta -> alpha_s
def test_p1_isothermal_beta_to_alpha_s_converges_first_order():
    """eq:beta_to_alpha_s at 900 K from pure beta (X_am stays 0, X_alpha^eq = 0.9):
    the explicit scheme with the A6 first step converges to the closed form
    with error ratio ~2 per dt halving (Sec. 3.1, explicit Euler)."""
    T = 900.0
    D, k, c = 0.9, orc.k_alpha_s(T), 2.51
    errs = []
    for dt in (0.02, 0.01, 0.005):
        s = orc.State.uniform(1, 0.0, 0.0)
        n = int(round(20.0 / dt))
        orc.run_temps(s, np.full(n + 1, T), dt)
        errs.append(abs(s.xas[0] - closed_form(20.0, D, k, c)))
    assert s.xam[0] == 0.0
    assert errs[2] < 2e-3
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.6 < r1 < 2.5 and 1.6 < r2 < 2.5, errs


def test_p1_analytic_steps_exact_with_init_ba_steps():
    """Reading A6 with INIT_BA_STEPS and an exit threshold never met: every
    step is the closed form, exact for any dt at constant T."""
    p = orc.params(init_ba_steps=1, init_exit=1e300)
    s = orc.State.uniform(1, 0.0, 0.0)
    orc.run_temps(s, np.full(11, 900.0), 1.0, p)
    assert s.xas[0] == pytest.approx(closed_form(10.0, 0.9, orc.k_alpha_s(900.0), 2.51), rel=1e-9)


# ----------------------------------------------- P2: App. A alpha_s -> beta
@pytest.mark.parametrize("floor", [0.0, 1e-3])
def test_p2_appendix_a_case(golden, floor):
    """App. A: T = 1200 K from (0.9, 0, 0.1).  The first step equals the closed
    form at t = dt (values below 1e-16 survive, ~3.6e-70); the run converges
    to the closed form with the beta rate k_beta = f k_as and equilibrium
    D = X_beta^eq - 0.1.  Checked for the literal exit rule (floor 0) and
    reading A5's floor."""
    case = golden["appendix_a_case"]
    T = case["T"]
    p = orc.params(init_exit_floor=floor)
    D = (1 - orc.xalpha_eq(T)) - case["X_beta0"]
    kb = 3.8 * orc.k_alpha_s(T)
    s = orc.State.uniform(1, case["X_as0"], 0.0)
    orc.run_temps(s, np.array([T, T]), 1e-5, p)
    assert s.mode[0] == orc.MODE_AS_TO_B and s.xas[0] == 0.9
    assert s.xt[0] == pytest.approx(closed_form(1e-5, D, kb, 11.0), rel=1e-9)
    assert 1e-71 < s.xt[0] < 1e-69
    errs = []
    for dt in (4e-3, 2e-3, 1e-3):
        s = orc.State.uniform(1, 0.9, 0.0)
        n = int(round(30.0 / dt))
        orc.run_temps(s, np.full(n + 1, T), dt, p)
        xb = 1 - s.xas[0] - s.xam[0]
        errs.append(abs((xb - 0.1) - closed_form(30.0, D, kb, 11.0)))
    assert s.mode[0] == orc.MODE_NONE
    assert errs[2] < 1e-3
    assert 1.6 < errs[0] / errs[1] < 2.6 and 1.6 < errs[1] / errs[2] < 2.6, errs


def test_p2_exit_rule_literal_vs_floor_agree():
    """Reading A5's floor only moves the switch from the closed form to Euler:
    the two runs differ by Euler's truncation error, which falls with dt and is
    far inside the 1e-4 budget at the workloads' dt."""
    diffs = []
    for dt in (1e-3, 2.5e-4):
        out = []
        for floor in (0.0, 1e-3):
            s = orc.State.uniform(1, 0.9, 0.0)
            orc.run_temps(s, np.full(int(round(20.0 / dt)) + 1, 1150.0), dt,
                          orc.params(init_exit_floor=floor))
            out.append(s.xas[0])
        diffs.append(abs(out[0] - out[1]))
    assert diffs[1] < 0.35 * diffs[0] and diffs[1] < 1e-5, diffs


def test_p2_exit_floor_leaves_the_workloads_unchanged():
    """At the workloads' dt = 1e-5 s a point heats through the alpha_s -> beta
    band in milliseconds, and X~_beta stays far below 1e-10 there (App. A's
    closed form: X~_beta ~ D (D k_beta t / c_beta)^c_beta with c_beta = 11),
    so the literal exit rule (floor 0) and reading A5's floor give the same
    bits on the line, a small block and two layers with interlayer cooling."""
    from tests._util import oracle_workload
    for w in (wl.line_4096(),
              wl.block_256(dims=(40, 24, 10), n_tracks=4, n_steps=1500, T_thr=0.0),
              wl.part_512(dims=(24, 20, 8), n_layers=2, tracks_per_layer=4, t_layer=2e-3,
                          hatch=5e-5)):
        a = oracle_workload(w)
        b = oracle_workload(w, p=orc.params(init_exit_floor=0.0))
        assert np.array_equal(a, b), w.name


# --------------------------------------------------- alpha_m -> alpha_s (r2)
def test_alpha_m_to_alpha_s_closed_form():
    """eq:alpha_m_to_alpha_s alone (900 K: X_alpha = X_alpha^eq = 0.9 so r1 = r3 = 0,
    no martensite formation or dissolution): X_as/0.9 follows the same
    generalised logistic with D = 0.9, k = k_as."""
    T, dt = 900.0, 2e-3
    k = orc.k_alpha_s(T)
    s = orc.State.make([0.3], [0.6])
    n = int(round(15.0 / dt))
    orc.run_temps(s, np.full(n + 1, T), dt)
    assert s.xas[0] + s.xam[0] == pytest.approx(0.9, abs=1e-12)
    assert s.xas[0] == pytest.approx(closed_form(15.0, 0.9, k, 2.51, X0=0.3), abs=2e-4)


def test_explicit_rates_use_T_n():
    """eq:explicit_integration evaluates the diffusive rates at T^n: when the
    correction g is the identity at both candidate T^{n+1}, the step result
    must not depend on T^{n+1}."""
    for T0, xas, xam in ((1000.0, 0.3, 0.0), (1100.0, 0.2, 0.1), (900.0, 0.4, 0.3)):
        out = []
        for T1 in (880.0, 905.0, 930.0):
            s = orc.State.make([xas], [xam])
            orc.run_temps(s, np.array([T0, T1]), 0.5)
            out.append((s.xas[0], s.xam[0]))
        assert out[0] == out[1] == out[2], (T0, out)
        assert out[0][0] != xas


# --------------------------------------------------------- P3 equilibria
@pytest.mark.parametrize("T", [1000.0, 1100.0])
def test_p3_long_holds_reach_equilibrium_from_both_sides(T):
    """Long isothermal holds in (T_as,end, T_as,start) converge to the
    Koistinen-Marburger equilibrium from pure beta (r1) and from 0.9 (r3 via
    App. A); X_am stays 0 above T_am,start."""
    xeq = 1 - math.exp(-0.0068 * (1273 - T))
    for x0 in (0.0, 0.9):
        s = orc.State.uniform(1, x0, 0.0)
        orc.run_temps(s, np.full(40001, T), 0.01)
        assert s.xam[0] == 0.0
        assert abs(s.xas[0] - xeq) < 3e-3, (x0, s.xas[0], xeq)


def test_p3_high_temperature_and_melt(golden):
    """Above T_as,start + T_reg only beta remains (Sec. 2.2 regularisation);
    in the mushy zone X_beta = 1 - (T - T_s)/(T_l - T_s); above T_l all liquid."""
    for T, xb_expect, xl_expect in ((1400.0, 1.0, 0.0), (1888.0, 0.8, 0.2), (2000.0, 0.0, 1.0)):
        s = orc.State.make([0.5], [0.3])
        orc.run_temps(s, np.array([T, T]), 1e-5)
        _, _, xb, xl = orc.fractions(s, T)
        assert s.xas[0] == 0.0 and s.xam[0] == 0.0
        assert xb[0] == pytest.approx(xb_expect, abs=1e-12)
        assert xl[0] == pytest.approx(xl_expect, abs=1e-12)


def test_room_temperature_state_is_stationary(golden):
    """(0.9, 0, 0.1) below T_as,end is an equilibrium (Sec. 4.2: beta reaches
    its 10 % equilibrium; Sec. 4.3: 90 % alpha_s)."""
    s = orc.State.uniform(1, 0.9, 0.0)
    orc.run_temps(s, np.full(1001, 353.0), 0.1)
    _, _, xb, _ = orc.fractions(s, 353.0)
    assert s.xas[0] == 0.9 and s.xam[0] == 0.0
    assert xb[0] == pytest.approx(golden["beta_room_temperature"]["value"], abs=1e-14)


# ---------------------------------------------------------- P4 / P5 martensite
@pytest.mark.parametrize("T1", [353.0, 600.0, 800.0])
def test_p4_quench_forms_pseudo_equilibrium_martensite(T1):
    """eq:inst_martensite_formation: an instant drop from the beta range below
    T_am,start gives X_am = X_am,0^eq(T1) (X_as = 0)."""
    s = orc.State.make([0.0], [0.0])
    orc.run_temps(s, np.array([1400.0, T1]), 1e-5)
    assert s.xas[0] == 0.0
    assert s.xam[0] == pytest.approx(1 - math.exp(-0.00415 * (848 - T1)), rel=1e-12)


def test_p5_martensite_only_on_fast_cooling():
    """Sec. 2.2: high cooling rates give martensite, low rates stable alpha_s."""
    def cool(rate, dt):
        n = int(round((1400 - 353) / rate / dt))
        T = np.linspace(1400.0, 353.0, n + 1)
        s = orc.State.make([0.0], [0.0])
        orc.run_temps(s, T, dt)
        return s.xas[0], s.xam[0]
    xas, xam = cool(1e5, 1e-5)
    assert xas < 1e-3 and xam == pytest.approx(1 - math.exp(-0.00415 * 495), abs=2e-3)
    xas, xam = cool(0.1, 0.5)
    assert xas > 0.89 and xam < 1e-2


def test_martensite_readings_agree_on_monotone_cooling():
    """Reading A3: formation-only and the literal equality agree when T only falls."""
    T = np.linspace(1500.0, 300.0, 5001)
    a, b = orc.State.make([0.0], [0.0]), orc.State.make([0.0], [0.0])
    orc.run_temps(a, T, 1e-4)
    orc.run_temps(b, T, 1e-4, orc.params(martensite_literal=1))
    assert a.xam[0] == pytest.approx(b.xam[0], abs=1e-12)
    assert a.xas[0] == pytest.approx(b.xas[0], abs=1e-12)


def test_martensite_does_not_revert_on_mild_reheating():
    """Reading A3 default: reheating below T_as,end keeps martensite (dissolution
    needs X_alpha > X_alpha^eq = 0.9, eq:inst_martensite_dissolution)."""
    s = orc.State.make([0.0], [0.0])
    orc.run_temps(s, np.array([1400.0, 400.0, 700.0, 700.0]), 1e-5)
    assert s.xam[0] == pytest.approx(1 - math.exp(-0.00415 * 448), abs=1e-6)


# ------------------------------------------------------------ g function
def test_correction_clamp_and_rescale():
    """eq:explicit_correction text: negative fractions become 0; X_alpha > 0.9 is
    scaled back to 0.9 keeping X_as / X_am."""
    xas, xam = orc.correct(900.0, -0.1, 0.3)
    assert xas == 0.0 and xam == 0.3
    xas, xam = orc.correct(900.0, 0.3, -0.1)
    assert xas == 0.3 and xam == 0.0
    xas, xam = orc.correct(900.0, 0.6, 0.4)
    assert xas + xam == pytest.approx(0.9, abs=1e-15) and xas / xam == pytest.approx(1.5, rel=1e-13)


def test_correction_regularisation_linear():
    """Sec. 2.2 regularisation (reading A4): the cap falls linearly from 0.9 at
    T_as,start to 0 at T_as,start + T_reg and stays 0 above."""
    caps = [orc.correct(T, 0.9, 0.0)[0] for T in (1273.0, 1298.0, 1323.0, 1348.0, 1373.0, 1500.0)]
    assert caps == pytest.approx([0.9, 0.675, 0.45, 0.225, 0.0, 0.0], abs=1e-12)


def test_correction_dissolution():
    """eq:inst_martensite_dissolution: if X_alpha > X_alpha^eq then
    X_am = max(X_alpha^eq - X_as, 0)."""
    T = 1100.0
    xeq = orc.xalpha_eq(T)
    xas, xam = orc.correct(T, 0.2, 0.6)
    assert xas == 0.2 and xam == pytest.approx(xeq - 0.2, abs=1e-14)
    xas, xam = orc.correct(T, 0.8, 0.05)
    assert xas == 0.8 and xam == 0.0


# ---------------------------------------------------------- P6 invariants
def test_p6_invariants_random_histories():
    """Phase continuity (eq:phase_continuity_*): every fraction in [0, 1],
    X_alpha <= 0.9, the four fractions sum to 1, along random temperature
    walks through every branch."""
    rng = np.random.default_rng(7)
    n, steps = 400, 300
    T = np.empty((steps + 1, n))
    T[0] = rng.uniform(250, 2600, n)
    for s in range(steps):
        T[s + 1] = np.clip(T[s] + rng.normal(0, 60, n), 250, 2600)
    st = orc.State.make(rng.uniform(0, 0.45, n), rng.uniform(0, 0.45, n))
    for s in range(steps):
        orc.run_temps(st, T[s:s + 2], 1e-3)
        xas, xam, xb, xl = orc.fractions(st, T[s + 1])
        for a in (xas, xam, xb, xl):
            assert np.all(a >= -1e-14) and np.all(a <= 1 + 1e-14)
        assert np.all(xas + xam <= 0.9 + 1e-14)
        assert np.allclose(xas + xam + xb + xl, 1.0, atol=1e-12)


# ---------------------------------------------------------- moving source
def _one_track(P=200.0, v=1.0):
    tracks = np.array([[0.0, 0.0, 1.0, 0.0, v, P, 0.0, 0]])
    return HeatSource(tracks, np.array([[0.0, 0.0, NEVER, NEVER]]), T_max=1e9)


def test_source_satisfies_heat_equation():
    """The synthetic driver must be a solution of dT/dt = alpha lap(T) away from
    the source (checked by finite differences in space and time)."""
    src = _one_track()
    t = 2e-3
    rng = np.random.default_rng(3)
    for _ in range(12):
        x = 2e-3 + rng.uniform(-4e-4, 1e-4)
        y = rng.uniform(-2e-4, 2e-4)
        z = -rng.uniform(5e-5, 3e-4)
        h, dt = 3e-7, 2e-8  # well below the 2 alpha / v = 6 um decay length
        T = lambda a, b, c, tt: orc.temperature(src, a, b, c, tt)[0][0]
        lap = sum(T(x + e[0], y + e[1], z + e[2], t) for e in
                  ((h, 0, 0), (-h, 0, 0), (0, h, 0), (0, -h, 0), (0, 0, h), (0, 0, -h)))
        lap = (lap - 6 * T(x, y, z, t)) / h ** 2
        dTdt = (T(x, y, z, t + dt) - T(x, y, z, t - dt)) / (2 * dt)
        assert dTdt == pytest.approx(3e-6 * lap, rel=5e-4, abs=1e-3)


def test_source_energy_balance_and_adiabatic_surface():
    """Conducted heat through a tiny hemisphere around the source equals the
    absorbed power A P (fixes the 2 pi k R normalisation of a half-space), and
    the surface z = 0 carries no flux away from the source."""
    src = _one_track(P=200.0)
    t = 1e-3
    sx = 1e-3
    r = 1e-8
    k = 7.0
    nth, nph = 120, 240
    th = (np.arange(nth) + 0.5) * (0.5 * math.pi / nth)   # polar angle from -z
    ph = (np.arange(nph) + 0.5) * (2 * math.pi / nph)
    flux = 0.0
    dr = 1e-11
    for a in th:
        ca, sa = math.cos(a), math.sin(a)
        dirs = np.stack([sa * np.cos(ph), sa * np.sin(ph), -ca * np.ones(nph)])
        p1 = np.array([[sx], [0], [0]]) + r * dirs
        p2 = np.array([[sx], [0], [0]]) + (r + dr) * dirs
        T1 = orc.temperature(src, *p1, t)[0]
        T2 = orc.temperature(src, *p2, t)[0]
        dTdr = (T2 - T1) / dr
        flux += np.sum(-k * dTdr) * r * r * sa * (0.5 * math.pi / nth) * (2 * math.pi / nph)
    assert flux == pytest.approx(0.35 * 200.0, rel=2e-3)
    h = 1e-7
    for x in (5e-4, 8e-4, 1.2e-3):
        Tm = orc.temperature(src, x, 1e-4, -h, t)[0][0]
        Tp = orc.temperature(src, x, 1e-4, h, t)[0][0]
        assert abs(Tp - Tm) < 1e-9 * Tm


def test_source_superposition_cap_and_layers():
    """Sources add linearly (below the cap); distance 0 gives T_max (reading A7);
    points above the current layer surface are inactive; the interlayer
    factor brings the field back to T0."""
    tr = np.array([[0.0, 0.0, 1.0, 0.0, 1.0, 200.0, 0.0, 0],
                   [0.0, 1e-4, 1.0, 0.0, 0.9, 150.0, 1e-3, 0]])
    L = np.array([[0.0, 0.0, NEVER, NEVER]])
    both = HeatSource(tr, L)
    a, b = HeatSource(tr[:1], L), HeatSource(tr[1:], L)
    x, y, z = np.array([3e-3, 2e-3]), np.array([5e-4, 2e-4]), np.array([-1e-4, -3e-4])
    t = 4e-3
    Tab = orc.temperature(both, x, y, z, t)[0]
    Ta, Tb = orc.temperature(a, x, y, z, t)[0], orc.temperature(b, x, y, z, t)[0]
    assert np.allclose(Tab - 353.0, (Ta - 353.0) + (Tb - 353.0), rtol=1e-12)
    T0, _ = orc.temperature(a, 1e-3, 0.0, 0.0, 1e-3)
    assert T0[0] == 4130.0
    # layers: surface at -3e-5 during layer 0, at 0 during layer 1
    tr2 = np.array([[0.0, 0.0, 1.0, 0.0, 1.0, 200.0, 0.0, 0],
                    [0.0, 0.0, 1.0, 0.0, 1.0, 200.0, 0.02, 1]])
    L2 = np.array([[-3e-5, 0.0, 0.005, 0.01], [0.0, 0.01, 0.03, 0.04]])
    src = HeatSource(tr2, L2)
    _, act = orc.temperature(src, [1e-3, 1e-3], [0, 0], [-1e-5, -3e-5], 1e-3)
    assert list(act) == [0, 1]
    T_end, _ = orc.temperature(src, 1e-3, 0.0, -3e-5, 0.00999999)
    assert T_end[0] == pytest.approx(353.0, abs=0.05)
    # after the last layer's end the field stays at T0 (the factor does not
    # turn negative)
    T_after, _ = orc.temperature(src, [1e-3, 5e-3], [0.0, 1e-4], [-3e-5, 0.0], 0.08)
    assert np.all(T_after == 353.0)
    T_mid, _ = orc.temperature(src, 1e-3, 0.0, -3e-5, 0.0075)
    T_scan, _ = orc.temperature(src, 1e-3, 0.0, -3e-5, 0.0050)
    assert (T_mid[0] - 353) == pytest.approx(0.5 * (orc.temperature(
        HeatSource(tr2[:1], np.array([[-3e-5, 0, NEVER, NEVER]])), 1e-3, 0, -3e-5, 0.0075)[0][0] - 353), rel=1e-9)
    assert T_scan[0] > T_mid[0]
    _, act = orc.temperature(src, [1e-3], [0], [-1e-5], 0.015)
    assert list(act) == [1]
    # layer 1 has begun but its track has not: the receding layer-0 source
    # (15 mm down the line, ~70 K of tail here) belongs to the old layer
    T_l1, _ = orc.temperature(src, [1e-3, 5e-3], [0, 0], [0.0, -3e-5], 0.015)
    assert np.all(T_l1 == 353.0)
    # tracks that have not started add nothing, also near their start
    xs, ys, zs = np.array([-4e-4, 0.0, 2e-4]), np.array([1e-4] * 3), np.array([-1e-5] * 3)
    assert np.array_equal(orc.temperature(both, xs, ys, zs, 0.5e-3)[0],
                          orc.temperature(a, xs, ys, zs, 0.5e-3)[0])
    # before the specimen's start offset nothing is hot
    off = HeatSource(tr[:1], L, t_offset=0.5)
    assert orc.temperature(off, 1e-4, 0, 0, 0.3)[0][0] == 353.0


def test_points_above_the_surface_are_not_advanced():
    """A point above the current layer's surface is not yet deposited: it
    keeps its state while the layer below is scanned right under it (the
    same point one layer down melts and re-forms), and takes part once its
    own layer begins."""
    tr = np.array([[0.0, 0.0, 1.0, 0.0, 1.0, 200.0, 0.0, 0],
                   [0.0, 0.0, 1.0, 0.0, 1.0, 200.0, 0.0105, 1]])
    L = np.array([[-3e-5, 0.0, 0.004, 0.01], [0.0, 0.01, 0.014, 0.02]])
    src = HeatSource(tr, L)
    x, y, z = np.array([1e-3, 1e-3]), np.array([0.0, 0.0]), np.array([-1e-5, -3e-5])
    s = orc.State.uniform(2, 0.9, 0.0)
    dt = 1e-5
    orc.run_track(s, src, x, y, z, 0, 999, dt)          # layer 0 only
    assert s.xas[0] == 0.9 and s.xam[0] == 0.0
    assert s.xam[1] > 0.5                                # melted and quenched
    orc.run_track(s, src, x, y, z, 999, 1000, dt)        # into layer 1
    assert s.xam[0] > 0.5


# ------------------------------------------- App. A entry, exits and r2
def test_full_alpha_with_martensite_dissolves_instantly():
    """A full alpha state with martensite (X_alpha = 0.9, X_am > 0) heated
    above T_as,end: r3 is zero (its factor 0.9 - X_alpha is), so alpha_s
    gains only the small alpha_m -> alpha_s transfer r2 dt in the step, and
    eq:inst_martensite_dissolution cuts X_am to X_alpha^eq - X_as at once
    (1000 K: X_alpha^eq = 0.843766, P3); the App. A alpha_s -> beta
    initiation is not entered (it starts from martensite-free full alpha)."""
    assert 0.5 + 0.4 == 0.9                              # X_alpha exactly 0.9
    s = orc.State.make([0.5], [0.4])
    orc.run_temps(s, np.array([1000.0, 1000.0]), 1e-5)
    assert 0.5 <= s.xas[0] < 0.5 + 1e-6
    assert s.xas[0] + s.xam[0] == pytest.approx(0.843766, abs=1e-6)
    assert s.mode[0] == orc.MODE_NONE


def test_regularisation_cap_ends_the_initiation():
    """Reading A5: once the alpha_s cap of the regularisation (Sec. 2.2) sets
    X_as, the App. A initiation ends; alpha_s -> beta then goes on by r3
    (X_alpha < 0.9 now), so at the same temperature the next step takes X_as
    strictly below the cap."""
    s = orc.State.uniform(1, 0.9, 0.0)
    orc.run_temps(s, np.array([1200.0, 1200.0, 1330.0]), 1e-5)
    cap = 0.9 * (1373.0 - 1330.0) / 100.0
    assert s.mode[0] == orc.MODE_NONE and s.xt[0] == 0.0
    assert s.xas[0] == pytest.approx(cap, abs=1e-14)
    orc.run_temps(s, np.array([1330.0, 1330.0]), 1e-3)
    assert s.xas[0] < cap - 1e-6


def test_persisted_beta_to_alpha_s_initiation_keeps_alpha_m_transfer():
    """Reading A6 with INIT_BA_STEPS: while the closed-form initiation
    advances alpha_s (D = X_alpha^eq - X_am), the alpha_m -> alpha_s rate r2
    (eq:alpha_m_to_alpha_s) still moves alpha_m into alpha_s, so X_alpha
    changes by the closed form's increment alone and X_am falls."""
    p = orc.params(init_ba_steps=1, init_exit=1e300)
    T, dt, xas0, xam0 = 900.0, 1e-2, 0.05, 0.3
    s = orc.State.make([xas0], [xam0])
    s.mode[:] = orc.MODE_B_TO_AS
    orc.run_temps(s, np.array([T, T]), dt, p)
    D, k, c = 0.9 - xam0, orc.k_alpha_s(T), 2.51
    # time at which the closed form (P1) passes X_as0, then dt later
    t0 = (c / (D * k)) * (xas0 / (D - xas0)) ** (1.0 / c)
    assert s.xas[0] + s.xam[0] - (xas0 + xam0) == pytest.approx(
        closed_form(t0 + dt, D, k, c) - xas0, rel=1e-9)
    assert s.xam[0] < xam0 - 1e-6


# ------------------------------------------------------------- dt halving
def test_dt_halving_on_a_moving_source_run():
    """Sec. 3.1: the explicit scheme converges at first order on a real heating
    / melting / quench history (a line of points under one moving source)."""
    src = HeatSource(np.array([[0.0, 0.0, 1.0, 0.0, 1.0, 200.0, 0.0, 0]]),
                     np.array([[0.0, 0.0, NEVER, NEVER]]))
    g = Grid((2e-4, 0.0, 0.0), (2.7e-5, 1.3e-5, -1e-5), (6, 2, 3))
    x, y, z = g.coords()
    t_end = 6e-3
    res = {}
    for dt in (8e-6, 4e-6, 2e-6, 1e-6, 2.5e-7):
        s = orc.State.uniform(g.n, 0.9, 0.0)
        orc.run_track(s, src, x, y, z, 0, int(round(t_end / dt)), dt)
        res[dt] = np.concatenate([s.xas, s.xam])
    ref = res[2.5e-7]
    e = [np.max(np.abs(res[d] - ref)) for d in (8e-6, 4e-6, 2e-6, 1e-6)]
    assert e[-1] < 1e-4
    assert all(e[i + 1] < 0.75 * e[i] for i in range(3)), e


# --------------------------------------- implicit scheme (Sec. 3, eq:implicit_*)
def _implicit(**kw):
    base = dict(integrator=1, dt_sub=0.0, fp_eps_abs=1e-16, fp_eps_rel=1e-13, fp_max_iter=500)
    base.update(kw)
    return orc.params(**base)


def test_implicit_crank_nicolson_is_second_order():
    """eq:beta_to_alpha_s at 900 K from X_as = 0.1 (no initiation, X_am = 0):
    Crank-Nicolson with the iteration converged tightly approaches the closed
    form with error ratio ~4 per dt halving; forward Euler with ~2."""
    T, X0, t_end = 900.0, 0.1, 4.0
    D, k, c = 0.9, orc.k_alpha_s(T), 2.51
    exact = orc.logistic_step(X0, D, k, c, t_end)
    errs = {}
    for name, p in (("cn", _implicit()), ("euler", orc.params())):
        errs[name] = []
        for dt in (0.4, 0.2, 0.1):
            s = orc.State.uniform(1, X0, 0.0)
            n = int(round(t_end / dt))
            orc.run_temps(s, np.full(n + 1, T), dt, p)
            errs[name].append(abs(s.xas[0] - exact))
    e = errs["cn"]
    assert 3.5 < e[0] / e[1] < 4.6 and 3.5 < e[1] / e[2] < 4.6, e
    f = errs["euler"]
    assert 1.6 < f[0] / f[1] < 2.5, f
    assert e[2] < f[2] / 20


def test_implicit_step_solves_its_equation():
    """A converged Crank-Nicolson step satisfies
    m = g(T1, m^n + dt/2 (mdot(T1, m) + mdot(T0, m^n))) (eq:implicit_integration
    with eq:implicit_correction), checked with the rate and correction
    functions pinned above, on states and temperature pairs of every branch."""
    import workloads as wl
    p = _implicit()
    xas, xam, T0, T1 = wl.random_states(400, seed=77)
    checked = 0
    for i in range(400):
        if xas[i] == 0.0 or xas[i] + xam[i] >= 0.9:   # initiation states
            continue
        for dt in (1e-4, 1e-2):
            a, m, it, conv = orc.cn_step(T0[i], T1[i], dt, xas[i], xam[i], p)
            assert conv and it >= 1
            r0 = orc.rates(T0[i], xas[i], xam[i], p)
            r1 = orc.rates(T1[i], a, m, p)
            ea, em = orc.correct(T1[i], xas[i] + 0.5 * dt * (r1[0] + r0[0]),
                                 xam[i] + 0.5 * dt * (r1[1] + r0[1]), p)
            assert abs(ea - a) < 1e-12 and abs(em - m) < 1e-12, (i, dt, a, ea, m, em)
            checked += 1
    assert checked > 400


def test_implicit_wrms_stop_and_iteration_count():
    """The WRMS stop (Sec. 3: eps_abs 1e-10, eps_rel 1e-3, no root): small
    steps converge in one or two iterations, larger steps need more; the
    stopped iterate lies within the tolerance of the tightly converged one."""
    p = orc.params(integrator=1)
    a1, m1, it_small, ok1 = orc.cn_step(1100.0, 1099.0, 1e-5, 0.3, 0.2, p)
    a2, m2, it_big, ok2 = orc.cn_step(1100.0, 1099.0, 0.01, 0.3, 0.2, p)
    assert ok1 and ok2 and it_small <= 2 and it_big >= it_small
    at, mt, _, _ = orc.cn_step(1100.0, 1099.0, 0.01, 0.3, 0.2, _implicit())
    assert abs(a2 - at) <= 1e-3 * 0.3 and abs(m2 - mt) <= 1e-3 * 0.2


def test_implicit_subcycling_is_substeps_with_linear_temperature():
    """One step of 0.1 s with dt_sub = 0.01 s is 10 substeps with the
    temperature linear in time (reading I3); exact multiples are not rounded
    up (0.1 / 0.01 -> 10 substeps)."""
    p = orc.params(integrator=1, dt_sub=0.01)
    assert orc.n_substeps(0.1, p) == 10 and orc.n_substeps(0.01, p) == 1
    assert orc.n_substeps(0.0101, p) == 2 and orc.n_substeps(1e-5, p) == 1
    # every step written as k hundredths takes k substeps, also where the
    # quotient rounds just above k (0.07 / 0.01 = 7.000000000000001)
    ks = range(1, 101)
    assert [orc.n_substeps(float(f"{k / 100:.2f}"), p) for k in ks] == list(ks)
    # (T0, T1, dt, substeps): cooling and heating, a multiple and not one;
    # the states include both App. A initiations (pure beta, full alpha)
    for T0, T1, dt, n in ((1150.0, 700.0, 0.1, 10), (1150.0, 700.0, 0.015, 2),
                          (900.0, 1210.0, 0.035, 4)):
        a = orc.State.uniform(5, 0.0, 0.0)
        a.xas[:] = [0.3, 0.6, 0.05, 0.0, 0.9]
        a.xam[:] = [0.2, 0.0, 0.4, 0.0, 0.0]
        b = a.copy()
        orc.step(a, T0, T1, dt, p)
        hist = np.array([[T0 + (T1 - T0) * (s / n)] * 5 for s in range(n + 1)])
        orc.run_temps(b, hist, dt / n, orc.params(integrator=1, dt_sub=0.0))
        np.testing.assert_array_equal(a.xas, b.xas)
        np.testing.assert_array_equal(a.xam, b.xam)
        np.testing.assert_array_equal(a.mode, b.mode)


def test_implicit_reaches_equilibria_and_quench_values():
    """With large steps (0.1 s, substeps of 0.01 s) the implicit scheme reaches
    the P3 equilibrium at 1000 K from pure beta (initiated by the App. A
    closed form, reading I2) as the explicit scheme does, and an instant drop
    gives the P4 quench value."""
    p = orc.params(integrator=1, dt_sub=0.01)
    s = orc.State.uniform(1, 0.0, 0.0)
    orc.run_temps(s, np.full(4001, 1000.0), 0.1, p)
    # the approach is a power law (gap^((c+1)/c)), as in the explicit P3 pin
    assert abs(s.xas[0] - (1 - math.exp(-0.0068 * 273.0))) < 3e-3
    e = orc.State.uniform(1, 0.0, 0.0)
    orc.run_temps(e, np.full(40001, 1000.0), 0.01)
    assert abs(s.xas[0] - e.xas[0]) < 1e-4
    # from full alpha (the App. A alpha_s -> beta initiation, reading I2;
    # its half time at 1000 K is c_beta / (D k_beta) = 176 s) it falls to the
    # equilibrium X_alpha^eq(1000 K) = 0.843766 (P3)
    f = orc.State.uniform(1, 0.9, 0.0)
    orc.run_temps(f, np.full(8001, 1000.0), 0.1, p)
    assert f.xas[0] == pytest.approx(0.843766, abs=1e-5)
    # an instant drop is one step without substeps (with substeps the 0.5 s
    # step cools linearly and a little alpha_s forms on the way)
    q = orc.State.uniform(1, 0.0, 0.0)
    orc.step(q, 1400.0, 353.0, 0.5, orc.params(integrator=1, dt_sub=0.0))
    assert q.xam[0] == pytest.approx(1 - math.exp(-0.00415 * (848 - 353)), rel=1e-12)
    assert q.xas[0] == 0.0


# ------------------------------------------------- tolerance derivation
def test_run_tolerance_covers_fp32_level_temperature_errors():
    """The whole-run bar max|dX| <= 1e-4 for the FP32 path, derived: on the
    4096-point line, rounding the stored fractions to FP32 after every step
    moves the FP64 result by ~3e-8 (no accumulation), and perturbing every
    temperature by a relative 2^-22 (the level of the approximate ex2, lg2
    and rsqrt) by < 1e-5, most of it in the mushy zone under the source,
    where X_liq = (T - T_s) / 50 passes a temperature error straight on.
    The bar leaves a factor of ten over that."""
    import workloads as wl
    w = wl.line_4096()
    sp = w.specimens[0]
    x, y, z = sp.grid.coords()
    T = np.stack([orc.temperature(sp.source, x, y, z, l * w.dt)[0] for l in range(w.n_steps + 1)])
    ref = orc.State.uniform(w.n_points, 0.9, 0.0)
    orc.run_temps(ref, T, w.dt)
    f_ref = np.stack(orc.fractions(ref, T[-1]))
    rng = np.random.default_rng(1)
    Tp = T * (1.0 + 2.0 ** -22 * rng.uniform(-1.0, 1.0, T.shape))
    per = orc.State.uniform(w.n_points, 0.9, 0.0)
    orc.run_temps(per, Tp, w.dt)
    d = np.abs(np.stack(orc.fractions(per, Tp[-1])) - f_ref).max(axis=0)
    assert d.max() < 1e-5
    mushy = (T[-1] > 1878.0) & (T[-1] < 1928.0)
    assert d.argmax() in np.nonzero(mushy)[0]
    st = orc.State.uniform(w.n_points, 0.9, 0.0)
    for s in range(w.n_steps):
        orc.run_temps(st, T[s:s + 2], w.dt)
        st.xas[:] = st.xas.astype(np.float32)
        st.xam[:] = st.xam.astype(np.float32)
    assert max(np.abs(st.xas - ref.xas).max(), np.abs(st.xam - ref.xam).max()) < 1e-7
