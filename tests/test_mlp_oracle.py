"""Pins of the surrogate's reference network (oracle/mlp.py) and of the
hybrid window form of the oracle (orc_run_track_windows), on the CPU."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
import workloads


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e4, 1000), rng.normal(0, 1e-6, 1000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, -3.0078125, 65504.0]])
    # exact ties of float32 values at bf16 precision, both parities
    ties = (np.arange(1, 200, dtype=np.uint32) << 16 | 0x8000).view(np.float32) * np.float32(1.0)
    x = np.concatenate([x, ties.astype(np.float64), -ties.astype(np.float64)])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)


def test_gelu_closed_forms():
    x = np.linspace(-8, 8, 2001)
    g = mlp.gelu(x)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    np.testing.assert_allclose(g - mlp.gelu(-x), x, rtol=0, atol=1e-13)  # tanh is odd
    assert abs(mlp.gelu(np.array([10.0]))[0] - 10.0) < 1e-12
    assert abs(mlp.gelu(np.array([-10.0]))[0]) < 1e-12
    # the tanh form approximates x * Phi(x) (Hendrycks and Gimpel 2016)
    from scipy.special import erf
    exact = 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))
    assert np.max(np.abs(g - exact)) < 1e-3
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(x), fd, rtol=0, atol=1e-8)


def test_single_path_network_by_hand():
    """Only W1[5][3], W2[7][5], W3[2][7] and b3 are non-zero, so
    y2 = c gelu(b gelu(a x3)) + d2 and y0, y1 are their biases; this fixes
    the parameter layout (row-major out x in) and the layer order."""
    a, b, c = 0.75, -1.25, 2.0
    d = np.array([0.1, -0.2, 0.3])
    p = np.zeros(mlp.N_PARAMS)
    p[mlp.OFF_W1 + 5 * mlp.N_IN + 3] = a
    p[mlp.OFF_W2 + 7 * mlp.N_H + 5] = b
    p[mlp.OFF_W3 + 2 * mlp.N_H + 7] = c
    p[mlp.OFF_B3:] = d
    X = np.random.default_rng(2).normal(0, 1, (50, mlp.N_IN))

    def g(v):
        return 0.5 * v * (1.0 + math.tanh(math.sqrt(2.0 / math.pi) * (v + 0.044715 * v ** 3)))

    y, _ = mlp.forward(p, X, bf16=False)
    expect2 = np.array([c * g(b * g(a * x3)) + d[2] for x3 in X[:, 3]])
    np.testing.assert_allclose(y[:, 2], expect2, rtol=1e-13, atol=1e-15)
    np.testing.assert_array_equal(y[:, 0], d[0])
    np.testing.assert_array_equal(y[:, 1], d[1])


def _single_path_bf16():
    """The one-path network of the test above with weights that bf16 cannot
    hold exactly, and torch's bfloat16 conversion as the rounding."""
    torch = pytest.importorskip("torch")

    def r(v):
        return torch.tensor(float(v), dtype=torch.float32).to(torch.bfloat16).double().item()

    a, b, c = 0.7513, -1.2571, 2.0113
    d = np.array([0.1, -0.2, 0.3])
    p = np.zeros(mlp.N_PARAMS)
    p[mlp.OFF_W1 + 5 * mlp.N_IN + 3] = a
    p[mlp.OFF_W2 + 7 * mlp.N_H + 5] = b
    p[mlp.OFF_W3 + 2 * mlp.N_H + 7] = c
    p[mlp.OFF_B3:] = d
    return r, (a, b, c, d), p


def test_single_path_network_in_bf16():
    """With bf16 on, the weights, the inputs and both hidden activations are
    rounded before they are used: on the one-path network
    y2 = r(c) r(gelu(r(b) r(gelu(r(a) r(x3))))) + d2, with r the rounding."""
    r, (a, b, c, d), p = _single_path_bf16()
    X = np.random.default_rng(12).normal(0, 1, (40, mlp.N_IN))
    y, _ = mlp.forward(p, X, bf16=True)
    for i, x3 in enumerate(X[:, 3]):
        a1 = r(mlp.gelu(np.array([r(a) * r(x3)]))[0])
        a2 = r(mlp.gelu(np.array([r(b) * a1]))[0])
        assert y[i, 2] == pytest.approx(r(c) * a2 + d[2], rel=1e-14, abs=1e-15), i
    np.testing.assert_array_equal(y[:, :2], np.tile(d[:2], (40, 1)))


def test_single_path_gradient_in_bf16_holds_the_rounded_values():
    """The bf16 gradient is backpropagation through the network with the
    rounded weights, inputs and activations held fixed (rounding passes the
    gradient unchanged): on the one-path network, by the chain rule,
    dL/dc = sum dy r(a2), dL/db = sum dy r(c) gelu'(h2) r(a1),
    dL/da = sum dy r(c) gelu'(h2) r(b) gelu'(h1) r(x3), and
    dL/dW1[5][4] the same with r(x4), dy = 2 (y2 - t2) / (3 n)."""
    r, (a, b, c, d), p = _single_path_bf16()
    rng = np.random.default_rng(13)
    n = 30
    X = rng.normal(0, 1, (n, mlp.N_IN))
    T = rng.normal(0, 1, (n, mlp.N_OUT))
    y, _ = mlp.forward(p, X, bf16=True)
    _, g = mlp.loss_and_gradient(p, X, T, bf16=True)
    dc = db = da = da4 = db3 = 0.0
    for i in range(n):
        dy = 2.0 * (y[i, 2] - T[i, 2]) / (3 * n)
        h1 = r(a) * r(X[i, 3])
        a1 = r(mlp.gelu(np.array([h1]))[0])
        h2 = r(b) * a1
        a2 = r(mlp.gelu(np.array([h2]))[0])
        back = dy * r(c) * mlp.gelu_grad(np.array([h2]))[0]
        dc += dy * a2
        db += back * a1
        da += back * r(b) * mlp.gelu_grad(np.array([h1]))[0] * r(X[i, 3])
        da4 += back * r(b) * mlp.gelu_grad(np.array([h1]))[0] * r(X[i, 4])
        db3 += dy
    assert g[mlp.OFF_W3 + 2 * mlp.N_H + 7] == pytest.approx(dc, rel=1e-12)
    assert g[mlp.OFF_W2 + 7 * mlp.N_H + 5] == pytest.approx(db, rel=1e-12)
    assert g[mlp.OFF_W1 + 5 * mlp.N_IN + 3] == pytest.approx(da, rel=1e-12)
    assert g[mlp.OFF_W1 + 5 * mlp.N_IN + 4] == pytest.approx(da4, rel=1e-12)
    assert g[mlp.OFF_B3 + 2] == pytest.approx(db3, rel=1e-12)


def test_gradient_against_finite_differences():
    rng = np.random.default_rng(3)
    p = rng.normal(0, 0.3, mlp.N_PARAMS)
    X = rng.normal(0, 1, (40, mlp.N_IN))
    T = rng.normal(0, 1, (40, mlp.N_OUT))
    loss, g = mlp.loss_and_gradient(p, X, T, bf16=False)
    blocks = [(mlp.OFF_W1, mlp.OFF_B1), (mlp.OFF_B1, mlp.OFF_W2), (mlp.OFF_W2, mlp.OFF_B2),
              (mlp.OFF_B2, mlp.OFF_W3), (mlp.OFF_W3, mlp.OFF_B3), (mlp.OFF_B3, mlp.N_PARAMS)]
    idx = np.concatenate([rng.choice(np.arange(lo, hi), min(12, hi - lo), replace=False)
                          for lo, hi in blocks])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_and_gradient(pp, X, T, bf16=False)[0] -
              mlp.loss_and_gradient(pm, X, T, bf16=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])
    # the loss is the mean over samples and outputs
    y, _ = mlp.forward(p, X, bf16=False)
    assert abs(loss - np.mean((y - T) ** 2)) < 1e-14


def test_relu_closed_forms():
    x = np.array([-3.0, -1e-300, -0.0, 0.0, 1e-300, 2.5])
    np.testing.assert_array_equal(mlp.relu(x), [0.0, 0.0, 0.0, 0.0, 1e-300, 2.5])
    # the derivative the kernels use: 1 above the kink, 0 at and below it
    np.testing.assert_array_equal(mlp.relu_grad(x), [0.0, 0.0, 0.0, 0.0, 1.0, 1.0])


def test_single_path_relu_network_by_hand():
    """ReLU on the one-path network with a, b, c > 0 and a first-layer bias
    e: y2 = c max(b max(a x3 + e, 0), 0) + d2 = b c max(a x3 + e, 0) + d2;
    the gradient follows by hand: dL/da = sum dy b c x3 [a x3 + e > 0],
    dL/de = sum dy b c [a x3 + e > 0], dL/dc = sum dy b max(a x3 + e, 0)."""
    a, b, c, e = 0.75, 1.25, 2.0, -0.3
    d = np.array([0.1, -0.2, 0.3])
    p = np.zeros(mlp.N_PARAMS)
    p[mlp.OFF_W1 + 5 * mlp.N_IN + 3] = a
    p[mlp.OFF_B1 + 5] = e
    p[mlp.OFF_W2 + 7 * mlp.N_H + 5] = b
    p[mlp.OFF_W3 + 2 * mlp.N_H + 7] = c
    p[mlp.OFF_B3:] = d
    rng = np.random.default_rng(22)
    n = 60
    X = rng.normal(0, 1, (n, mlp.N_IN))
    T = rng.normal(0, 1, (n, mlp.N_OUT))
    y, _ = mlp.forward(p, X, bf16=False, act="relu")
    on = a * X[:, 3] + e > 0
    np.testing.assert_allclose(y[:, 2], b * c * np.where(on, a * X[:, 3] + e, 0.0) + d[2],
                               rtol=1e-14, atol=1e-15)
    assert 0 < on.sum() < n
    _, g = mlp.loss_and_gradient(p, X, T, bf16=False, act="relu")
    dy = 2.0 * (y[:, 2] - T[:, 2]) / (3 * n)
    assert g[mlp.OFF_W1 + 5 * mlp.N_IN + 3] == pytest.approx(np.sum(dy * b * c * X[:, 3] * on),
                                                             rel=1e-12)
    assert g[mlp.OFF_B1 + 5] == pytest.approx(np.sum(dy * b * c * on), rel=1e-12)
    assert g[mlp.OFF_W3 + 2 * mlp.N_H + 7] == pytest.approx(
        np.sum(dy * b * np.where(on, a * X[:, 3] + e, 0.0)), rel=1e-12)
    # the other first-layer rows carry no gradient (their units stay at 0)
    assert np.all(g[mlp.OFF_W1:mlp.OFF_W1 + 5 * mlp.N_IN] == 0.0)


def test_single_path_relu_network_in_bf16():
    """ReLU with bf16 on: y2 = r(c) r(relu(r(b) r(relu(r(a) r(x3))))) + d2."""
    r, (a, b, c, d), p = _single_path_bf16()
    p[mlp.OFF_W2 + 7 * mlp.N_H + 5] = -b       # a positive path
    X = np.random.default_rng(14).normal(0, 1, (40, mlp.N_IN))
    y, _ = mlp.forward(p, X, bf16=True, act="relu")
    for i, x3 in enumerate(X[:, 3]):
        a1 = r(max(r(a) * r(x3), 0.0))
        a2 = r(max(r(-b) * a1, 0.0))
        assert y[i, 2] == pytest.approx(r(c) * a2 + d[2], rel=1e-14, abs=1e-15), i


def test_relu_gradient_against_finite_differences():
    """Central differences of the ReLU network's loss on samples whose
    pre-activations all stay 1e-3 away from the kink (the step is 1e-6)."""
    rng = np.random.default_rng(4)
    p = rng.normal(0, 0.3, mlp.N_PARAMS)
    X = rng.normal(0, 1, (200, mlp.N_IN))
    _, (x, h1, a1, h2, a2, *_w) = mlp.forward(p, X, bf16=False, act="relu")
    keep = (np.abs(h1).min(1) > 1e-3) & (np.abs(h2).min(1) > 1e-3)
    X = X[keep][:40]
    assert len(X) >= 10
    T = rng.normal(0, 1, (len(X), mlp.N_OUT))
    _, g = mlp.loss_and_gradient(p, X, T, bf16=False, act="relu")
    blocks = [(mlp.OFF_W1, mlp.OFF_B1), (mlp.OFF_B1, mlp.OFF_W2), (mlp.OFF_W2, mlp.OFF_B2),
              (mlp.OFF_B2, mlp.OFF_W3), (mlp.OFF_W3, mlp.OFF_B3), (mlp.OFF_B3, mlp.N_PARAMS)]
    idx = np.concatenate([rng.choice(np.arange(lo, hi), min(12, hi - lo), replace=False)
                          for lo, hi in blocks])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_and_gradient(pp, X, T, bf16=False, act="relu")[0] -
              mlp.loss_and_gradient(pm, X, T, bf16=False, act="relu")[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_zero_network_outputs_biases():
    p = np.zeros(mlp.N_PARAMS)
    p[mlp.OFF_B3:] = [1.0, 2.0, 3.0]
    y, _ = mlp.forward(p, np.ones((4, mlp.N_IN)))
    np.testing.assert_array_equal(y, np.tile([1.0, 2.0, 3.0], (4, 1)))


# ------------------------------------------------------------ window form
def _line(P, n=256, T0=353.0):
    w = workloads.line_4096(n_points=n, n_steps=400)
    src = w.specimens[0].source
    src.tracks[:, 5] = P
    src.T0 = T0
    if P == 0.0:  # keep the points off the path (R = 0 gives T_max, reading A7)
        w.specimens[0].grid.origin = (0.0, 1e-3, 0.0)
    return w, src


def test_windows_all_band_equal_explicit_run():
    """A band wider than every temperature sends every window to the
    explicit steps: the window form is then orc_run_track itself."""
    w, src = _line(200.0)
    x, y, z = w.specimens[0].grid.coords()
    p = oracle.params()
    a = oracle.State.uniform(x.size)
    b = oracle.State.uniform(x.size)
    oracle.run_track(a, src, x, y, z, 0, 203, w.dt, p)
    n_mlp = oracle.run_track_windows(b, src, x, y, z, 0, 203, w.dt, band_half=1e9, p=p)
    assert n_mlp.sum() == 0
    np.testing.assert_array_equal(a.xas, b.xas)
    np.testing.assert_array_equal(a.xam, b.xam)
    # the App. A state too (an initiation's X~ can sit far below what
    # changes X_as)
    np.testing.assert_array_equal(a.mode, b.mode)
    np.testing.assert_array_equal(a.xt, b.xt)


def test_windows_cold_quench_reduces_to_correction():
    """No source (P = 0) at T0 = 353 K: every full window is outside the band
    and applies g at 353 K, which from pure beta forms martensite
    X_am = 1 - exp(-k_am (848 - 353)) (P4 quench); the short tail window
    takes the explicit steps."""
    w, src = _line(0.0)
    x, y, z = w.specimens[0].grid.coords()
    p = oracle.params()
    st = oracle.State.uniform(x.size)
    st.xas[:] = 0.0
    st.xam[:] = 0.0
    n_mlp = oracle.run_track_windows(st, src, x, y, z, 0, 8 * 5, w.dt, p=p)
    assert np.all(n_mlp == 5)
    np.testing.assert_allclose(st.xam, 1.0 - math.exp(-0.00415 * (848.0 - 353.0)), rtol=0,
                               atol=1e-15)
    assert np.all(st.xas == 0.0)
    st2 = oracle.State.uniform(x.size)
    st2.xas[:] = 0.5
    st2.xam[:] = 0.1
    n_mlp = oracle.run_track_windows(st2, src, x, y, z, 0, 8 * 5 + 3, w.dt, p=p)
    assert np.all(n_mlp == 5)


def test_windows_band_edges():
    """A window whose temperatures sit inside the band takes the explicit
    steps; just outside it keeps its fractions (zero network)."""
    p = oracle.params()
    for T_hold, in_band in ((848.0 + 39.0, True), (848.0 + 41.0, False), (1838.5, True),
                            (1837.5, False), (1373.0 - 39.0, True), (1000.0, False)):
        w, src = _line(0.0, n=4, T0=T_hold)
        x, y, z = w.specimens[0].grid.coords()
        st = oracle.State.uniform(4)
        st.xas[:] = 0.6      # off the alpha_s plateau's fixed point
        st.xam[:] = 0.1
        n_mlp = oracle.run_track_windows(st, src, x, y, z, 0, 16, w.dt, p=p)
        assert np.all(n_mlp == (0 if in_band else 2)), T_hold


def test_windows_heating_through_T_as_end_leave_the_fixed_point():
    """A line 0.1 mm beside the track heats through T_as,end to ~1050 K: its
    points enter the alpha_s -> beta initiation, so windows that reach
    T_as,end are not fixed-point windows.  With every window sent to the
    explicit steps (band wider than every temperature) the window form must
    equal the explicit run in every variable, initiation state included."""
    w, src = _line(200.0)
    w.specimens[0].grid.origin = (0.0, 1e-4, 0.0)
    x, y, z = w.specimens[0].grid.coords()
    p = oracle.params()
    a = oracle.State.uniform(x.size)
    b = oracle.State.uniform(x.size)
    oracle.run_track(a, src, x, y, z, 0, 200, w.dt, p)
    oracle.run_track_windows(b, src, x, y, z, 0, 200, w.dt, band_half=1e9, p=p)
    assert np.any(a.mode == oracle.MODE_AS_TO_B)
    for f in ("xas", "xam", "xt", "mode"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))


def test_windows_fixed_point_is_the_explicit_identity():
    """The room-temperature state (0.9, 0, 0.1) is a fixed point of the
    explicit step below T_as,end (X_alpha^eq = 0.9, no rate acts, formation's
    target X_am^eq (0.9 - X_as) / 0.9 is 0): the explicit run leaves it
    exactly unchanged at every constant temperature below 935 K, also inside
    the bands at 848 K, and the window form counts those windows as fixed;
    at 1000 K the alpha_s -> beta initiation starts and nothing is fixed."""
    p = oracle.params()
    for T_hold in (353.0, 600.0, 847.0, 848.0, 849.0, 900.0, 934.0):
        w, src = _line(0.0, n=4, T0=T_hold)
        x, y, z = w.specimens[0].grid.coords()
        a = oracle.State.uniform(4)
        oracle.run_track(a, src, x, y, z, 0, 40, w.dt, p)
        assert np.all(a.xas == 0.9) and np.all(a.xam == 0.0) and np.all(a.mode == 0), T_hold
        b = oracle.State.uniform(4)
        n_mlp, n_fixed = oracle.run_track_windows(b, src, x, y, z, 0, 40, w.dt, p=p,
                                                   return_fixed=True)
        assert np.all(n_fixed == 5) and np.all(n_mlp == 0), T_hold
    w, src = _line(0.0, n=4, T0=1000.0)
    x, y, z = w.specimens[0].grid.coords()
    a = oracle.State.uniform(4)
    oracle.run_track(a, src, x, y, z, 0, 40, w.dt, p)
    assert np.all(a.mode == oracle.MODE_AS_TO_B)   # App. A: X~_beta far below 1e-16 yet
    n_mlp, n_fixed = oracle.run_track_windows(oracle.State.uniform(4), src, x, y, z, 0, 40, w.dt,
                                               p=p, return_fixed=True)
    assert np.all(n_fixed == 0)


def _hold(T_hold, n=2):
    w, src = _line(0.0, n=n, T0=T_hold)
    return (src,) + w.specimens[0].grid.coords() + (w.dt,)


def test_window_starting_inside_an_initiation_takes_the_explicit_steps():
    """Reading S1: a window with an App. A initiation running at its start
    (here alpha_s -> beta at a constant 1000 K, outside every band) takes the
    explicit steps, so the window form equals the explicit run."""
    src, x, y, z, dt = _hold(1000.0)
    p = oracle.params()
    mk = lambda: oracle.State.make([0.9 - 1e-3] * 2, [0.0] * 2, xt=[1e-3] * 2,
                                   mode=[oracle.MODE_AS_TO_B] * 2)
    a, b = mk(), mk()
    oracle.run_track(a, src, x, y, z, 0, 8, dt, p)
    n_mlp = oracle.run_track_windows(b, src, x, y, z, 0, 8, dt, p=p)
    assert np.all(n_mlp == 0)
    for f in ("xas", "xam", "xt", "mode"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))


def test_window_start_level_counts_in_the_band():
    """Reading S1: the band test covers the window's start temperature too.
    A point held at 886.5 K (38.5 K above T_am,start) is warmed by ~4 K, to
    just outside every band, from the first new level on by a weak track
    that starts half a step after the window's start and stays 5.3 mm away
    (the samples then differ from the start by less than 40 K): the window
    takes the explicit steps, while the same window started one window
    later, at the warm temperature, passes the test."""
    dt = 1e-5
    tracks = np.array([[0.0, 0.0, 1.0, 0.0, 1.0, 2.8, 40.5 * dt, 0]])
    src = workloads.HeatSource(tracks, np.array([[0.0, 0.0, workloads.NEVER, workloads.NEVER]]),
                               T0=886.5)
    x, y, z = np.array([-5.3e-3]), np.array([0.0]), np.array([0.0])
    T = np.array([oracle.temperature(src, x, y, z, (40 + l) * dt)[0][0] for l in range(17)])
    assert T[0] == 886.5 and np.all((T[1:] > 888.5) & (T[1:] < 894.5)), T
    p = oracle.params()
    a, b = oracle.State.make([0.6], [0.1]), oracle.State.make([0.6], [0.1])
    oracle.run_track(a, src, x, y, z, 40, 8, dt, p)
    n_mlp = oracle.run_track_windows(b, src, x, y, z, 40, 8, dt, p=p)
    assert n_mlp[0] == 0
    np.testing.assert_array_equal(a.xas, b.xas)
    np.testing.assert_array_equal(a.xam, b.xam)
    c = oracle.State.make([0.6], [0.1])
    assert oracle.run_track_windows(c, src, x, y, z, 48, 8, dt, p=p)[0] == 1


def test_g_only_window_corrects_at_every_level():
    """A window outside the bands applies g at each of its new temperatures in
    turn.  A point 100 um beside the track heats from ~420 K to ~530 K within
    one window: from pure beta the martensite that forms is that of the
    window's coldest (first) level, X_am = 1 - exp(-k_am (848 - T_1)) (P4),
    and the warmer levels after it form no more (reading A3)."""
    dt = 1e-5
    tracks = np.array([[0.0, 0.0, 1.0, 0.0, 1.0, 200.0, 0.0, 0]])
    src = workloads.HeatSource(tracks, np.array([[0.0, 0.0, workloads.NEVER, workloads.NEVER]]))
    x, y, z = np.array([0.5e-3]), np.array([100e-6]), np.array([0.0])
    n0 = 66
    T = np.array([oracle.temperature(src, x, y, z, (n0 + l) * dt)[0][0] for l in range(9)])
    assert np.all(np.diff(T) > 0) and T[8] < 808.0 and T[8] - T[1] > 80.0
    st = oracle.State.make([0.0], [0.0])
    n_mlp = oracle.run_track_windows(st, src, x, y, z, n0, 8, dt, p=oracle.params())
    assert n_mlp[0] == 1
    assert st.xam[0] == pytest.approx(1.0 - math.exp(-0.00415 * (848.0 - T[1])), rel=1e-12)
    assert st.xas[0] == 0.0


def test_windows_leave_undeposited_points_alone():
    """Points above the current layer's surface keep their state in the
    window form too: with every window sent to the explicit steps it equals
    the explicit run on two layers, the undeposited point untouched through
    the first."""
    dt = 1e-5
    tr = np.array([[0.0, 0.0, 1.0, 0.0, 1.0, 200.0, 0.0, 0],
                   [0.0, 0.0, 1.0, 0.0, 1.0, 200.0, 0.0105, 1]])
    L = np.array([[-3e-5, 0.0, 0.004, 0.01], [0.0, 0.01, 0.014, 0.02]])
    src = workloads.HeatSource(tr, L)
    x, y, z = np.array([1e-3, 1e-3]), np.array([0.0, 0.0]), np.array([-1e-5, -3e-5])
    a, b = oracle.State.uniform(2), oracle.State.uniform(2)
    oracle.run_track(a, src, x, y, z, 0, 999, dt)
    oracle.run_track_windows(b, src, x, y, z, 0, 999, dt, band_half=1e9)
    assert b.xas[0] == 0.9 and b.xam[0] == 0.0
    for f in ("xas", "xam", "xt", "mode"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))


def test_host_band_mask_matches_the_oracle_band():
    """surrogate.band_mask (which windows the training data may give to the
    network) uses the oracle window form's band: within 40 K of T_am,start,
    T_as,end, T_as,start or T_as,start + T_reg, or above T_s - 40 K, at the
    window's start or any sample, or two consecutive temperatures more than
    40 K apart.  Checked on windows ramping by 30 K per sample away from an
    edge value planted at the start or the end (each temperature's band
    membership taken from the oracle's window form on a hold at it), and on
    jumps of 39 K and 41 K between out-of-band temperatures."""
    from paper_2402_17580_gb300 import _binding as B
    from paper_2402_17580_gb300.surrogate import band_mask
    p = B.default_params()
    po = oracle.params()
    for T_edge in (848.0 + 39.0, 848.0 + 41.0, 935.0 - 39.5, 935.0 + 40.5, 1273.0 + 39.0,
                   1373.0 - 41.0, 1838.5, 1837.5, 600.0, 1100.0):
        for sign in (1.0, -1.0):
            ramp = T_edge + sign * 30.0 * np.arange(9)
            want = bool(np.any([oracle_in_band(t, po) for t in ramp]))
            for T in (ramp, ramp[::-1]):
                assert bool(band_mask(T[None, :], p)[0]) == want, (T_edge, sign)
    for jump, want in ((39.0, False), (41.0, True)):
        for at in range(1, 9):
            T = np.full(9, 1100.0)
            T[at:] += jump
            assert bool(band_mask(T[None, :], p)[0]) == want, (jump, at)


def test_window_form_sends_sample_jumps_to_the_explicit_steps():
    """A point 0.12 mm beside and 0.05 mm below a 200 W track, stepped at
    20 us, heats by up to ~14 K per step while it stays below every band:
    windows of 32 levels sampled at every level pass the band test on the
    rise, the same windows sampled at every 4th level (jumps > 40 K) take
    the explicit steps; elsewhere both forms give the same g-only windows."""
    w, src = _line(200.0, n=1)
    w.specimens[0].grid.origin = (3.0e-4, 1.2e-4, -5.0e-5)
    x, y, z = w.specimens[0].grid.coords()
    dt = 2.0e-5
    p = oracle.params()
    T = np.array([oracle.temperature(src, x, y, z, l * dt)[0][0] for l in range(161)])
    assert T.max() < 848.0 - 40.0, T.max()
    jumps = [np.abs(np.diff(T[32 * k:32 * k + 33:4])).max() > 40.0 for k in range(5)]
    steps = [np.abs(np.diff(T[32 * k:32 * k + 33])).max() > 40.0 for k in range(5)]
    assert any(jumps) and not any(steps)
    a, b = oracle.State.make([0.6], [0.1]), oracle.State.make([0.6], [0.1])
    n1 = oracle.run_track_windows(a, src, x, y, z, 0, 160, dt, window=32, stride=1, p=p)
    n4 = oracle.run_track_windows(b, src, x, y, z, 0, 160, dt, window=8, stride=4, p=p)
    assert n1[0] == 5 and n4[0] == 5 - sum(jumps)


def test_window_form_sends_a_turn_between_samples_to_the_explicit_steps():
    """On a seeded training line (its first specimen, point 192, levels
    1184..1216) a point cools from 795 K to a minimum of 771.08 K at level
    1215 before the next pass reheats it; sampled at every 4th level the
    temperatures fall monotonically (771.27 K last), so g at the samples
    would miss the martensite the dip forms (3.3e-3 per K of undercooling).
    The parabola through the last three samples has its vertex 1.1
    spacings past the middle one: the window form sends the window to the
    explicit steps, and the host mask agrees; sampled at every level the
    same 32-level window applies g at the minimum itself and passes."""
    from paper_2402_17580_gb300 import _binding as B
    from paper_2402_17580_gb300.surrogate import band_mask
    w = workloads.surrogate_lines(n_lines=1)
    sp = w.specimens[0]
    x, y, z = (a[192:193] for a in sp.grid.coords())
    n0, dt = 1184, w.dt
    T = np.array([oracle.temperature(sp.source, x, y, z, (n0 + l) * dt)[0][0] for l in range(33)])
    s4 = T[::4]
    assert np.all(np.diff(s4) < 0) and 790.0 < s4[0] < 808.0
    assert np.argmin(T) == 31 and T.min() < s4[-1] - 0.15
    k = s4[6] - 2 * s4[7] + s4[8]
    assert 2.0 * k < abs(s4[8] - s4[6]) <= 4.0 * k      # vertex 1 to 2 spacings out
    p = oracle.params()
    st = oracle.State.uniform(sp.grid.n, 0.9, 0.0)
    oracle.run_track(st, sp.source, *sp.grid.coords(), 0, n0, dt, p)
    a, b = (oracle.State.make([st.xas[192]], [st.xam[192]]) for _ in range(2))
    assert a.mode[0] == 0 and 0.1 < a.xam[0] < 0.3
    assert oracle.run_track_windows(a, sp.source, x, y, z, n0, 32, dt, window=8, stride=4,
                                    p=p)[0] == 0
    assert oracle.run_track_windows(b, sp.source, x, y, z, n0, 32, dt, window=32, stride=1,
                                    p=p)[0] == 1
    # g at the minimum forms the undercooling's martensite, g at the samples not
    gs, gm = st.xas[192], st.xam[192]
    for t in s4[1:]:
        gs, gm = oracle.correct(t, gs, gm, p)
    assert b.xam[0] > gm + 4e-4
    assert bool(band_mask(s4[None, :], B.default_params(), 4)[0])
    assert not bool(band_mask(s4[None, :], B.default_params(), 1)[0])


def test_window_form_group_takes_explicit_steps_together():
    """Points grouped like the hybrid kernel's tiles: a line off the fixed
    point under a track has, in every window, hot points near the source in
    the band and cold points outside it.  Alone (group 1) the cold points
    apply g only; as one group every window sends them to the explicit steps
    with the hot ones, and the window form equals the explicit run."""
    w, src = _line(200.0)
    x, y, z = w.specimens[0].grid.coords()
    p = oracle.params()
    mk = lambda: oracle.State.make([0.6] * x.size, [0.1] * x.size)
    a, b, c = mk(), mk(), mk()
    oracle.run_track(a, src, x, y, z, 0, 96, w.dt, p)
    n1 = oracle.run_track_windows(b, src, x, y, z, 0, 96, w.dt, p=p, group=1)
    nn = oracle.run_track_windows(c, src, x, y, z, 0, 96, w.dt, p=p, group=x.size)
    assert n1.sum() > 0 and nn.sum() == 0
    for f in ("xas", "xam", "xt", "mode"):
        np.testing.assert_array_equal(getattr(a, f), getattr(c, f))


def oracle_in_band(T, po):
    """Whether a window held at T is sent to the explicit steps by the
    oracle's window form (a 16-step hold from a state off the fixed point)."""
    w, src = _line(0.0, n=1, T0=T)
    x, y, z = w.specimens[0].grid.coords()
    st = oracle.State.make([0.6], [0.1])
    n_mlp = oracle.run_track_windows(st, src, x, y, z, 0, 16, w.dt, p=po)
    return n_mlp[0] == 0
