"""The FMA-pipe exp2 / log2 (MS_FLAG_FMA_TRANSCENDENTALS; the paper's
polynomial transcendentals, Sec. 3.3) on the GPU.

The device functions are checked against the mathematics (numpy's FP64
exp2 and log2) over the whole FP32 range the kernels use, with the bounds
the fit states (exp2: relative error <= 1e-7 for the polynomial, plus the
FP32 rounding of the reduced argument; log2: absolute error <= 6e-8 on the
polynomial part plus the rounding of the result), beside the SFU's own error
on the same inputs.  The FP32 hot kernels built with them are then held to
the same parity bars as the SFU build: one step against the oracle on
random states in every branch, whole runs at 1e-4.
"""
import numpy as np
import pytest

import oracle as orc
import workloads as wl
from tests._util import gpu_workload, max_abs_diff, oracle_params, oracle_view, oracle_workload

pytestmark = pytest.mark.gpu

RUN_TOL = 1e-4
STEP_TOL = 2e-6
IMPL_STEP_TOL = 1e-5


@pytest.fixture(scope="module")
def ms():
    import paper_2402_17580_gb300 as m
    m.load()
    return m


FMA = 8   # MS_FLAG_FMA_TRANSCENDENTALS


def test_exp2_against_the_mathematics(ms):
    from paper_2402_17580_gb300 import _binding as B
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-125.9, 127.9, 400000), rng.uniform(-1, 1, 200000),
                        np.arange(-125, 128), np.arange(-125, 127) + 0.5]).astype(np.float32)
    ref = np.exp2(x.astype(np.float64))
    # the polynomial's bound, and a loose one for the SFU (its error is shown
    # beside the polynomial's, not pinned here)
    errs = {}
    for which, bound in (("fma_ex2", 3e-7), ("sfu_ex2", 2e-6)):
        y = B.eval_transcendental(which, x).astype(np.float64)
        rel = np.abs(y / ref - 1.0)
        errs[which] = float(rel.max())
        assert rel.max() <= bound, (which, float(rel.max()))
    print("exp2 relative error", errs)
    special = np.array([-np.inf, -200.0, -126.5, 0.0], dtype=np.float32)
    y = B.eval_transcendental("fma_ex2", special)
    np.testing.assert_array_equal(y, np.array([0.0, 0.0, 0.0, 1.0], dtype=np.float32))


def test_log2_against_the_mathematics(ms):
    from paper_2402_17580_gb300 import _binding as B
    rng = np.random.default_rng(2)
    x = np.concatenate([np.exp2(rng.uniform(-125.9, 127.9, 400000)), rng.uniform(0.5, 2.0, 200000),
                        rng.uniform(1e-6, 0.9, 100000)]).astype(np.float32)
    x = x[np.isfinite(x) & (x >= np.float32(1.17549435e-38))]
    ref = np.log2(x.astype(np.float64))
    for which, a, r in (("fma_lg2", 3e-7, 1.2e-7), ("sfu_lg2", 2e-6, 1e-6)):
        y = B.eval_transcendental(which, x).astype(np.float64)
        err = np.abs(y - ref)
        print(which, "max abs error", float(err.max()))
        assert np.all(err <= a + r * np.abs(ref)), (which, float(err.max()))
    special = np.array([0.0, 1e-40, np.inf, -1.0, 1.0, 2.0, 0.5], dtype=np.float32)
    y = B.eval_transcendental("fma_lg2", special)
    assert y[0] == -np.inf and y[1] == -np.inf and y[2] == np.inf and np.isnan(y[3])
    np.testing.assert_array_equal(y[4:], np.array([0.0, 1.0, -1.0], dtype=np.float32))


@pytest.mark.parametrize("dt,block,integrator,tol", [(1e-5, 1, 0, STEP_TOL),
                                                    (1e-3, 10, 0, STEP_TOL),
                                                    (1e-3, 1, 1, IMPL_STEP_TOL)])
def test_single_step_every_branch(ms, dt, block, integrator, tol):
    n = 6 * 128 + 37
    xas, xam, T0, T1 = wl.random_states(n, seed=21 + block, block=block)
    T0, T1 = T0.astype(np.float32), T1.astype(np.float32)
    ctx = ms.Context(n, flags=FMA, integrator=integrator)
    ctx.set_state(xas, xam)
    ctx.step(T0, T1, dt)
    g = ctx.fractions()
    p = oracle_params(ctx.params)
    st = orc.State.make(oracle_view(xas), oracle_view(xam))
    orc.step(st, T0.astype(np.float64), T1.astype(np.float64), dt, p)
    o = orc.fractions(st, T1.astype(np.float64), p)
    assert max_abs_diff(g, np.stack(o)) <= tol
    ctx.close()


@pytest.mark.parametrize("case", ["line_4096", "small_block"])
def test_runs_against_the_oracle(ms, case):
    """Whole runs through ms_run_track (the far-field kernel of the FMA
    build; the block with the active set on) against the oracle, and the
    App. A initiation below the FP32 range through ms_step."""
    if case == "line_4096":
        w = wl.line_4096()
    else:
        w = wl.block_256(dims=(256, 24, 8), n_tracks=4, n_steps=2500)
    ctx, g = gpu_workload(w, flags=FMA)
    assert max_abs_diff(g, oracle_workload(w)) <= RUN_TOL
    ctx.close()
    c = ms.Context(1, flags=FMA)
    c.set_state([0.9], [0.0])
    for _ in range(21):
        c.step(np.float32([1200.0]), np.float32([1200.0]), 1e-5)
    st = orc.State.make([0.9], [0.0])
    orc.run_temps(st, np.full(22, 1200.0), 1e-5)
    assert c.aux()[0] == pytest.approx(st.xt[0], rel=1e-4)
    c.close()


def test_flag_needs_fp32(ms):
    for prec in (ms.MS_F64ACC, ms.MS_KAHAN, ms.MS_F64):
        with pytest.raises(ms.MSError, match="UNSUPPORTED"):
            ms.Context(16, flags=FMA, precision=prec)
