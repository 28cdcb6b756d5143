"""GPU tests of the window surrogate: the network kernels against the FP64
reference network (oracle/mlp.py), the hybrid window machinery against the
oracle's window form, and a trained surrogate against the explicit oracle.

Tolerances.
* Network: inference and training round weights, inputs and hidden
  activations to BF16 like the reference, but evaluate GELU's tanh with
  tanh.approx.f32 (relative error about 2^-11) and sum in FP32 (ReLU is
  exact; its outputs differ from the reference by the FP32 sums, which can
  still move an activation across a BF16 rounding boundary).  A hidden
  activation can then land on the neighbouring BF16 value (2^-8 relative),
  which moves an output by about |w| 2^-8 |a| ~ 1e-3 for the weight scales
  used; outputs are held to 2e-2 x max(1, |y|) element-wise and 2e-3 on
  average, gradients to 2e-2 of their norm.
* Zero network: MLP windows reduce to the correction g at the window's
  samples, so the hybrid is held to the explicit path's run tolerance
  (1e-4) against the oracle's window form, for windows sampled at every
  level and at every 4th, 8th and 16th.
* Trained network: no closed form; the bar is the hybrid path's target,
  max|dX| <= 5e-3 against the FP64 explicit oracle (50x the explicit FP32
  path's bar), with the judge's own per-window error reported beside it.
  What the network buys is measured against the same windows with a zero
  network (correction g only, no diffusion in MLP windows): the trained
  hybrid must be at least 5x closer to the oracle than that.  Three network
  designs are trained and held to these bars: GELU with windows of 8 steps
  sampled at every level, and ReLU with windows of 32 and 64 steps sampled
  at every 4th and 8th level.  On held-out windows whose residuals stay
  within 1e-4 (at least 99.9 % of them) the mean absolute error must be
  below half the residuals' own mean absolute value with every level
  sampled (measured 0.32), below 0.7 of it with r > 1 (measured 0.16 at
  r = 4, 0.60 at r = 8), and with every level sampled the RMS error over
  all windows below half their RMS (the network explains at least 75 % of
  their variance).  With r > 1 the samples do not determine the path
  between them, on which the diffusion depends: part of each residual is
  beyond any function of the network's inputs, and the few larger
  residuals come from temperature extremes between the samples that the
  band test does not catch.  The block test is the bar that counts: at
  r = 8 the trained hybrid sits 30x closer to the oracle than the zero
  network.
"""
import math

import numpy as np
import pytest

import oracle as orc
import workloads as wl
from oracle import mlp as omlp
from tests._util import max_abs_diff, oracle_params

pytestmark = pytest.mark.gpu

RUN_TOL = 1e-4
HYBRID_TOL = 5e-3     # the hybrid path's max|dX| target
GAIN_MIN = 5.0        # zero-network error / trained error (measured: 11)


@pytest.fixture(scope="module")
def ms():
    import paper_2402_17580_gb300 as m
    m.load()
    return m


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    xas = rng.uniform(0, 0.9, n)
    xam = rng.uniform(0, 1, n) * (0.9 - xas)
    T = rng.uniform(353, 1800, (n, 8))
    x = np.empty((n, 12), dtype=np.float32)
    x[:, 0], x[:, 1], x[:, 2] = xas, xam, 1 - xas - xam
    x[:, 3:11] = (T - 1000) * 1e-3
    x[:, 11] = rng.choice([0.0, -1.0, 1.0], n)
    return x


def _params(seed):
    rng = np.random.default_rng(seed)
    p = np.empty(omlp.N_PARAMS, dtype=np.float32)
    p[omlp.OFF_W1:omlp.OFF_B1] = rng.normal(0, 1 / math.sqrt(12), 64 * 12)
    p[omlp.OFF_B1:omlp.OFF_W2] = rng.normal(0, 0.2, 64)
    p[omlp.OFF_W2:omlp.OFF_B2] = rng.normal(0, 1 / 8, 64 * 64)
    p[omlp.OFF_B2:omlp.OFF_W3] = rng.normal(0, 0.2, 64)
    p[omlp.OFF_W3:omlp.OFF_B3] = rng.normal(0, 1 / 8, 3 * 64)
    p[omlp.OFF_B3:] = rng.normal(0, 0.2, 3)
    return p


ACTS = [(0, "gelu"), (1, "relu")]   # MS_ACT_GELU, MS_ACT_RELU


@pytest.mark.parametrize("act,name", ACTS)
def test_forward_matches_reference_network(ms, torch, act, name):
    n = 128 * 37 + 45  # several warps and CTAs and a ragged tail
    x = np.concatenate([_inputs(n - 200, 1), np.random.default_rng(2).normal(0, 1, (200, 12))
                        .astype(np.float32)])
    p = _params(3)
    s = ms.Surrogate(p, act)
    assert s.config() == (act, 1)
    # the surrogate's own stream; the results are read after a device-wide sync
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    s.forward(xd.data_ptr(), yd.data_ptr(), n)
    torch.cuda.synchronize()
    y = yd.cpu().numpy().astype(np.float64)
    ref, _ = omlp.forward(p.astype(np.float64), x.astype(np.float64), bf16=True, act=name)
    err = np.abs(y - ref)
    assert np.all(err <= 2e-2 * np.maximum(1.0, np.abs(ref))), err.max()
    assert err.mean() <= 2e-3
    np.testing.assert_array_equal(s.params(), p)
    s.close()


@pytest.mark.parametrize("act,name", ACTS)
def test_gradient_matches_reference_network(ms, torch, act, name):
    n = 3000
    x = _inputs(n, 4)
    t = np.random.default_rng(5).normal(0, 0.5, (n, 3)).astype(np.float32)
    p = _params(6)
    s = ms.Surrogate(p, act)
    # the surrogate's own stream; the results are read after a device-wide sync
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    gd = torch.empty(omlp.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = s.gradient(xd.data_ptr(), td.data_ptr(), n, gd.data_ptr())
    g = gd.cpu().numpy().astype(np.float64)
    ref_loss, ref_g = omlp.loss_and_gradient(p.astype(np.float64), x.astype(np.float64),
                                             t.astype(np.float64), bf16=True, act=name)
    assert abs(loss - ref_loss) <= 1e-3 * ref_loss
    assert np.linalg.norm(g - ref_g) <= 2e-2 * np.linalg.norm(ref_g)
    s.close()


@pytest.mark.parametrize("act", [0, 1])
def test_training_reduces_loss(ms, torch, act):
    """Adam on a smooth synthetic target (numpy, seeded) lowers the loss by
    more than 5x in 400 steps."""
    n = 20000
    x = _inputs(n, 7)
    A = np.random.default_rng(8).normal(0, 1, (12, 3))
    t = np.tanh(x.astype(np.float64) @ A).astype(np.float32)
    from paper_2402_17580_gb300 import surrogate
    s = ms.Surrogate(surrogate.init_params(9), act)
    # the surrogate's own stream; the results are read after a device-wide sync
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    first = s.gradient(xd.data_ptr(), td.data_ptr(), n)
    for _ in range(400):
        s.train_step(xd.data_ptr(), td.data_ptr(), n, 3e-3)
    last = s.gradient(xd.data_ptr(), td.data_ptr(), n)
    assert last < first / 5, (first, last)
    assert np.all(np.isfinite(s.params()))
    s.close()


# ------------------------------------------------------------- hybrid path
def _run(ms, w, surrogate, judge=0.0, **kw):
    ctx = ms.Context(w.n_points, T_thr=w.T_thr, **kw)
    ctx.set_points([sp.grid for sp in w.specimens])
    ctx.fill_state(w.init_xas, w.init_xam)
    if surrogate is not None:
        ctx.set_surrogate(surrogate, judge)
    ctx.run_track([sp.source for sp in w.specimens], w.n_steps, w.dt)
    return ctx, ctx.fractions()


@pytest.mark.parametrize("precision,stride,act", [(0, 1, 0), (2, 1, 0), (0, 4, 1), (2, 8, 1),
                                                  (0, 16, 1)])
def test_zero_network_hybrid_matches_window_oracle(ms, precision, stride, act):
    """A network with all parameters 0 outputs 0, so every MLP window only
    applies g at its samples in turn: the hybrid kernel must then follow
    orc_run_track_windows (band test, window classification, fallback
    steps, the 128-point tiles taking the explicit steps together) on every
    point of the 4096-point line."""
    w = wl.line_4096()
    s = ms.Surrogate(np.zeros(omlp.N_PARAMS, dtype=np.float32), act, stride)
    ctx, g = _run(ms, w, s, judge=1.0, precision=precision, steps_per_launch=128)
    st = ctx.stats()
    sp = w.specimens[0]
    x, y, z = sp.grid.coords()
    o = orc.State.uniform(w.n_points, w.init_xas, w.init_xam)
    p = oracle_params()
    n_mlp, n_fixed = orc.run_track_windows(o, sp.source, x, y, z, 0, w.n_steps, w.dt, p=p,
                                           return_fixed=True, stride=stride, group=128)
    T_last = orc.temperature(sp.source, x, y, z, w.n_steps * w.dt)[0]
    of = np.stack(orc.fractions(o, T_last, p))
    assert max_abs_diff(g, of) <= RUN_TOL
    # windows are g-only (MLP), explicit (ODE) or, on the alpha_s plateau's
    # fixed point below T_as,end, left alone (most of the line's windows:
    # the points ahead of the source and the cold tail)
    L = 8 * stride
    total = w.n_points * ((w.n_steps + L - 1) // L)
    n_m, n_f = int(n_mlp.sum()), int(n_fixed.sum())
    assert st.surrogate_windows > 0.1 * total and n_f > 0
    assert abs(st.surrogate_windows - n_m) <= 1e-3 * total
    assert abs(st.ode_windows - (total - n_m - n_f)) <= 1e-3 * total
    assert st.judge_samples == st.surrogate_windows  # judge_frac = 1
    assert 0.0 < st.judge_max_err < 1.0
    ctx.close()
    s.close()


def test_zero_network_hybrid_ragged_row_tile(ms):
    """The hybrid kernel's far field on grids whose last row tile holds fewer
    than 128 points (lanes past the specimen's end): the zero network must
    still follow orc_run_track_windows on every point."""
    w = wl.block_256(dims=(200, 7, 3), n_tracks=4, n_steps=1800, T_thr=0.0)
    s = ms.Surrogate(np.zeros(omlp.N_PARAMS, dtype=np.float32), 1, 4)
    ctx, g = _run(ms, w, s, judge=0.0, steps_per_launch=128)
    sp = w.specimens[0]
    x, y, z = sp.grid.coords()
    o = orc.State.uniform(w.n_points, w.init_xas, w.init_xam)
    p = oracle_params()
    orc.run_track_windows(o, sp.source, x, y, z, 0, w.n_steps, w.dt, p=p, stride=4, group=128)
    T_last = orc.temperature(sp.source, x, y, z, w.n_steps * w.dt)[0]
    assert max_abs_diff(g, np.stack(orc.fractions(o, T_last, p))) <= RUN_TOL
    ctx.close()
    s.close()


def test_judge_sends_windows_back(ms):
    """ms_set_judge_tol.  A zero network (g only over each window: about
    1.6e-4 from the explicit oracle on this block) with every tile-window
    judged.  At tol = +inf the judge only measures: the result is the
    unjudged run's, bit for bit.  At tol = 0 every judged tile-window where
    the network's result differs from the explicit steps' takes theirs: the
    run then agrees with the FP64 explicit oracle to the FP32 path's run
    tolerance, and ms_stats counts the windows sent back."""
    w = wl.block_256(dims=(96, 96, 16), n_tracks=6, n_steps=4000)
    zero = ms.Surrogate(np.zeros(omlp.N_PARAMS, dtype=np.float32), 1, 8)

    def run(judge, tol):
        ctx = ms.Context(w.n_points, T_thr=w.T_thr)
        ctx.set_points([sp.grid for sp in w.specimens])
        ctx.fill_state(w.init_xas, w.init_xam)
        ctx.set_surrogate(zero, judge)
        ctx.set_judge_tol(tol)
        ctx.run_track([sp.source for sp in w.specimens], w.n_steps, w.dt)
        out = (ctx.fractions(), ctx.aux(), ctx.stats())
        ctx.close()
        return out

    g0, a0, s0 = run(0.0, float("inf"))
    gi, ai, si = run(1.0, float("inf"))
    gr, ar, sr = run(1.0, 0.0)
    for x, y in zip(g0, gi):
        assert np.array_equal(x, y)
    assert np.array_equal(a0, ai)
    assert si.judge_samples > 0 and si.judge_rejected == 0 and s0.judge_rejected == 0
    assert sr.judge_rejected > 0
    idx = np.random.default_rng(10).choice(w.n_points, 256, replace=False)
    idx = np.unique(np.concatenate([idx, np.arange(0, w.n_points, 9973)]))
    from tests._util import oracle_workload
    o = oracle_workload(w, idx)
    err_g = max_abs_diff(g0, o, idx)
    err_r = max_abs_diff(gr, o, idx)
    print(f"zero network {err_g:.3e}, judge sending back {sr.judge_rejected} windows {err_r:.3e}")
    assert err_r <= RUN_TOL
    assert err_r < 0.5 * err_g
    with pytest.raises(ms.MSError):
        c = ms.Context(16)
        try:
            c.set_judge_tol(float("nan"))
        finally:
            c.close()
    zero.close()


def test_hybrid_rejects_fp64_and_bad_fraction(ms):
    s = ms.Surrogate(np.zeros(omlp.N_PARAMS, dtype=np.float32))
    ctx = ms.Context(1000, precision=ms.MS_F64)
    with pytest.raises(ms.MSError, match="UNSUPPORTED"):
        ctx.set_surrogate(s, 0.0)
    ctx.close()
    ctx = ms.Context(1000)
    with pytest.raises(ms.MSError, match="INVALID_ARG"):
        ctx.set_surrogate(s, 1.5)
    ctx.set_surrogate(s, 0.5)
    ctx.set_surrogate(None)
    ctx.close()
    s.close()


@pytest.fixture(scope="module", params=[(0, 1), (1, 4), (1, 8)],
                ids=["gelu_r1", "relu_r4", "relu_r8"])
def trained(ms, torch, request):
    from paper_2402_17580_gb300 import surrogate
    act, stride = request.param
    w = wl.surrogate_lines(n_lines=64)
    data = surrogate.collect_windows(w.specimens, w.n_steps, w.dt, seed=1, stride=stride)
    s = surrogate.train(data.X, data.Y, iters=20000, batch=32768, lr=1e-3, seed=2,
                        activation=act, stride=stride)
    held = wl.surrogate_lines(seed=wl.SEED_BASE + 40, n_lines=16)
    hd = surrogate.collect_windows(held.specimens, held.n_steps, held.dt, seed=3, stride=stride)
    s.report = {"windows": len(data.X), "seen": data.windows_seen, "band": data.band_windows,
                "held_out": surrogate.evaluate(s, hd.X, hd.Y)}
    yield s
    s.close()


def test_trained_surrogate_held_out_error(trained):
    r = trained.report
    print("surrogate", trained.config(), r)
    assert r["windows"] > 10000
    h = r["held_out"]
    assert h["core_share"] > 0.999
    assert h["core_mae"] < (0.5 if trained.stride == 1 else 0.7) * h["core_target_mae"]
    if trained.stride == 1:
        assert h["rms"] < 0.5 * h["target_rms"]


def test_trained_hybrid_against_oracle(ms, trained):
    """A 96 x 96 x 16 block under 6 serpentine tracks (the 256^3 block's
    process parameters), 4000 steps, T_thr = 600 K: the hybrid path against
    the FP64 explicit oracle on 256 sampled points."""
    w = wl.block_256(dims=(96, 96, 16), n_tracks=6, n_steps=4000)
    ctx, g = _run(ms, w, trained, judge=0.01)
    st = ctx.stats()
    idx = np.random.default_rng(10).choice(w.n_points, 256, replace=False)
    # include the points the tracks pass over
    idx = np.unique(np.concatenate([idx, np.arange(0, w.n_points, 9973)]))
    from tests._util import oracle_workload
    o = oracle_workload(w, idx)
    err = max_abs_diff(g, o, idx)
    share = st.surrogate_windows / max(1, st.surrogate_windows + st.ode_windows)
    zero = ms.Surrogate(np.zeros(omlp.N_PARAMS, dtype=np.float32), *trained.config())
    zctx, zg = _run(ms, w, zero)
    err0 = max_abs_diff(zg, o, idx)
    print(f"hybrid {trained.config()} max|dX| {err:.3e} (zero network {err0:.3e}), "
          f"MLP share {share:.3f}, "
          f"judge {st.judge_samples} windows max {st.judge_max_err:.3e}")
    assert st.surrogate_windows > 0 and st.judge_samples > 0
    assert err <= HYBRID_TOL
    # what the trained network gains over the method without it (g only)
    assert err0 >= GAIN_MIN * err, (err, err0)
    zctx.close()
    zero.close()
    ctx.close()
