"""The window surrogate: training data, training loop and hybrid set-up.

The surrogate advances a point's fractions over 8 x stride explicit steps
with one MLP evaluation (see ``ms_set_surrogate`` in include/ms.h): the
network sees the temperatures of every stride-th level of the window (its 8
samples); the correction g at the samples gives the instantaneous part, the
network the diffusive residual.  Its
training windows come from this library's own full-FP64 path (``MS_F64``,
every step explicit, no skipping) on seeded synthetic thermal histories; the
network is trained on the GPU by the library's kernels (``ms_surrogate_*``).
PyTorch provides the device buffers and the stream only.

    from paper_2402_17580_gb300 import surrogate
    data = surrogate.collect_windows(w.specimens, w.n_steps, w.dt, stride=4)
    s = surrogate.train(data.X, data.Y, iters=4000, activation=B.MS_ACT_RELU, stride=4)
    ctx.set_surrogate(s, judge_frac=0.01)
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import _binding as B

T_SHIFT, T_SCALE, DT_SHIFT, OUT_SCALE = 1000.0, 1e-3, 5.0, 1.0e6
BAND_HALF_WIDTH = 40.0
CORE_RESIDUAL = 1e-4   # evaluate(): windows with larger residuals are reported apart
WINDOW = B.MS_MLP_WINDOW
N_IN, N_H, N_OUT = B.MS_MLP_IN, 64, B.MS_MLP_OUT


def band_mask(T: np.ndarray, p: B.Params, stride: int = 1) -> np.ndarray:
    """True where a window (rows of T: its start and its 8 samples) needs the
    explicit steps: a temperature within 40 K of T_am,start, T_as,end,
    T_as,start or T_as,start + T_reg, above T_s - 40 K, two consecutive
    temperatures more than 40 K apart, or (stride > 1) three consecutive
    temperatures whose parabola has a minimum below T_am,start or a maximum
    above T_as,end near them (extreme_between)."""
    edges = (p.T_am_start, p.T_as_end, p.T_as_start, p.T_as_start + p.T_reg)
    m = (T > p.T_s - BAND_HALF_WIDTH).any(axis=-1)
    for e in edges:
        m |= (np.abs(T - e) < BAND_HALF_WIDTH).any(axis=-1)
    d = np.diff(T, axis=-1)
    m |= ~(np.abs(d) <= BAND_HALF_WIDTH).all(axis=-1)
    if stride > 1:
        m |= extreme_between(T[..., :-2], T[..., 1:-1], T[..., 2:], p).any(axis=-1)
    return m


def extreme_between(a, b, c, p: B.Params):
    """Whether the parabola through three equally spaced temperatures a, b, c
    has its vertex within two sample spacings of b (between a and c, or up
    to one spacing beyond them: an abrupt turn can put the path's extreme
    between the samples while the parabola's lies past them) with a minimum
    below T_am,start or a maximum above T_as,end, where the correction g
    depends on the path's extreme."""
    k = a - 2.0 * b + c
    s = c - a
    inside = (k != 0) & (np.abs(s) <= 4.0 * np.abs(k))
    with np.errstate(divide="ignore", invalid="ignore"):
        v = b - s * s / (8.0 * k)
    return inside & np.where(k > 0, v < p.T_am_start, v > p.T_as_end)


def encode(xas, xam, T_new, dt) -> np.ndarray:
    """Network inputs (float32, [n, 12]) of windows starting at (xas, xam)
    with sampled temperatures T_new [n, 8]."""
    n = len(xas)
    x = np.empty((n, N_IN), dtype=np.float32)
    x[:, 0] = xas
    x[:, 1] = xam
    x[:, 2] = 1.0 - np.asarray(xas) - np.asarray(xam)
    x[:, 3:3 + WINDOW] = (np.asarray(T_new) - T_SHIFT) * T_SCALE
    x[:, 11] = math.log10(dt) + DT_SHIFT
    return x


def init_params(seed: int = 0) -> np.ndarray:
    """Seeded initial parameters: N(0, 1/fan_in) weights (last layer scaled
    by 0.1), zero biases, in the layout of include/ms.h."""
    rng = np.random.default_rng(seed)
    w1 = rng.normal(0.0, 1.0 / math.sqrt(N_IN), (N_H, N_IN))
    w2 = rng.normal(0.0, 1.0 / math.sqrt(N_H), (N_H, N_H))
    w3 = rng.normal(0.0, 0.1 / math.sqrt(N_H), (N_OUT, N_H))
    p = np.concatenate([w1.ravel(), np.zeros(N_H), w2.ravel(), np.zeros(N_H), w3.ravel(),
                        np.zeros(N_OUT)]).astype(np.float32)
    assert p.size == B.MS_MLP_PARAMS
    return p


@dataclass
class WindowSet:
    X: np.ndarray          # [n, 12] float32 inputs
    Y: np.ndarray          # [n, 3] float32 targets (1e6 x diffusive residuals)
    windows_seen: int      # windows before the band / change filter
    band_windows: int
    zero_windows: int      # windows without change (kept: a sample of them)


def collect_windows(specimens, n_steps: int, dt: float, keep_zero: float = 0.05, seed: int = 0,
                    params: B.Params | None = None, stride: int = 1) -> WindowSet:
    """Run the specimens with the full-FP64 explicit path and cut every
    point's history into windows of 8 x stride steps, sampling the
    temperature at every stride-th level; keep the windows the hybrid kernel
    would give the MLP (no band temperature or jump at the samples, no
    App. A initiation at the start), and of those without any change only a
    keep_zero sample.  Targets are 1e6 x (end fractions - G(start
    fractions)), G applying the correction g at the window's 8 samples in
    turn: the part of the window the correction does not supply."""
    if stride not in (1, 2, 4, 8, 16):
        raise ValueError("stride must be 1, 2, 4, 8 or 16")
    p = params or B.default_params()
    rng = np.random.default_rng(seed)
    n = sum(s.grid.n for s in specimens)
    ctx = B.Context(n, B.default_params(precision=B.MS_F64, T_thr=0.0))
    try:
        ctx.set_points([s.grid for s in specimens])
        ctx.fill_state(0.9, 0.0)
        srcs = [s.source for s in specimens]
        ctx.run_track(srcs, 0, dt)
        Tw = np.empty((n, WINDOW + 1))
        Xs, Ys = [], []
        seen = band = zero = 0
        K = WINDOW * stride
        for w0 in range(0, n_steps - K + 1, K):
            xas0, xam0 = ctx.fractions(with_beta=False)
            aux0 = ctx.aux()
            Tw[:, 0] = ctx.temperature()
            for l in range(WINDOW):
                ctx.run_track(srcs, stride, dt)
                Tw[:, l + 1] = ctx.temperature()
            xas1, xam1 = ctx.fractions(with_beta=False)
            seen += n
            bm = band_mask(Tw, p, stride) | (aux0 != 0.0)
            band += int(bm.sum())
            d_as, d_am = xas1 - xas0, xam1 - xam0
            still = (d_as == 0.0) & (d_am == 0.0)
            zero += int((still & ~bm).sum())
            keep = ~bm & (~still | (rng.random(n) < keep_zero))
            if not keep.any():
                continue
            Xs.append(encode(xas0[keep], xam0[keep], Tw[keep, 1:], dt))
            # residual: window end minus the correction g alone at the samples
            cas, cam = ctx.apply_correction(Tw[keep, 1:], xas0[keep], xam0[keep])
            r_as, r_am = xas1[keep] - cas, xam1[keep] - cam
            y = np.empty((int(keep.sum()), N_OUT), dtype=np.float32)
            y[:, 0] = OUT_SCALE * r_as
            y[:, 1] = OUT_SCALE * r_am
            y[:, 2] = -OUT_SCALE * (r_as + r_am)
            Ys.append(y)
    finally:
        ctx.close()
    X = np.concatenate(Xs) if Xs else np.zeros((0, N_IN), np.float32)
    Y = np.concatenate(Ys) if Ys else np.zeros((0, N_OUT), np.float32)
    return WindowSet(X, Y, seen, band, zero)


def train(X: np.ndarray, Y: np.ndarray, iters: int = 4000, batch: int = 16384, lr: float = 2e-3,
          lr_min: float = 2e-5, seed: int = 0, init: np.ndarray | None = None,
          log_every: int = 0, device: str = "cuda", activation: int = B.MS_ACT_GELU,
          stride: int = 1) -> B.Surrogate:
    """Adam with a cosine learning-rate decay on seeded minibatches; every
    step runs in the library's training kernels on a stream of its own.  The
    stride must be the one the windows (X, Y) were cut with."""
    import torch

    s = B.Surrogate(init if init is not None else init_params(seed), activation, stride)
    # one dedicated stream for torch's minibatch gathers and the library's
    # training kernels (a NULL handle would select the surrogate's own stream)
    stream = torch.cuda.Stream(device)
    s.set_stream(stream.cuda_stream)
    with torch.cuda.stream(stream):
        Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(device)
        Yd = torch.from_numpy(np.ascontiguousarray(Y, dtype=np.float32)).to(device)
        n = Xd.shape[0]
        if n == 0:
            raise ValueError("no training windows")
        b = min(batch, n)
        gen = torch.Generator(device=device)
        gen.manual_seed(seed)
        xb = torch.empty((b, N_IN), dtype=torch.float32, device=device)
        yb = torch.empty((b, N_OUT), dtype=torch.float32, device=device)
        history = []
        for it in range(iters):
            idx = torch.randint(0, n, (b,), generator=gen, device=device)
            torch.index_select(Xd, 0, idx, out=xb)
            torch.index_select(Yd, 0, idx, out=yb)
            a = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * it / max(1, iters - 1)))
            want = bool(log_every) and (it % log_every == 0 or it == iters - 1)
            loss = s.train_step(xb.data_ptr(), yb.data_ptr(), b, a, want_loss=want)
            if want:
                history.append((it, loss))
    stream.synchronize()
    s.set_stream(None)
    s.history = history
    return s


def evaluate(s: B.Surrogate, X: np.ndarray, Y: np.ndarray, device: str = "cuda") -> dict:
    """Inference on (X, Y): RMS, mean and max absolute error of the
    residuals (network output / 1e6), beside the residuals' own, and the
    mean absolute errors over the core windows, whose residuals stay within
    CORE_RESIDUAL (the rest come from temperature extremes between the
    samples that no function of the samples predicts)."""
    import torch

    stream = torch.cuda.Stream(device)
    s.set_stream(stream.cuda_stream)
    with torch.cuda.stream(stream):
        Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(device)
        out = torch.empty((Xd.shape[0], N_OUT), dtype=torch.float32, device=device)
        s.forward(Xd.data_ptr(), out.data_ptr(), Xd.shape[0])
    stream.synchronize()
    s.set_stream(None)
    err = (out.cpu().numpy() - Y) / OUT_SCALE
    tgt = np.asarray(Y, dtype=np.float64)[:, :2] / OUT_SCALE
    core = np.abs(tgt).max(axis=1) <= CORE_RESIDUAL
    return {"rms": float(np.sqrt(np.mean(err[:, :2] ** 2))),
            "mae": float(np.mean(np.abs(err[:, :2]))),
            "core_share": float(core.mean()) if len(core) else 1.0,
            "core_mae": float(np.mean(np.abs(err[core, :2]))) if core.any() else 0.0,
            "core_target_mae": float(np.mean(np.abs(tgt[core]))) if core.any() else 0.0,
            "max": float(np.abs(err[:, :2]).max()) if len(err) else 0.0,
            "target_rms": float(np.sqrt(np.mean(tgt ** 2))) if len(tgt) else 0.0,
            "target_mae": float(np.mean(np.abs(tgt))) if len(tgt) else 0.0,
            "target_max": float(np.abs(tgt).max()) if len(tgt) else 0.0}


__all__ = ["band_mask", "extreme_between", "encode", "init_params", "collect_windows", "train", "evaluate",
           "WindowSet"]
