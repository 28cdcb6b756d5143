"""ms_run_track_noalloc against ms_run_track, through the C ABI.

Some callers cannot allocate device memory while they run: their memory
belongs to a pre-sized pool, cudaMalloc's device-wide synchronisation is too
costly in their loop, or their GPU footprint must not grow.  For them the
library offers a no-alloc entry point that keeps its scratch in a static
device array and works on state arrays the caller already owns.  This test
gives it state arrays from the caller's allocator (torch here), runs the
same specimen as a context does, on two calls in a row, the first of them on
a torch side stream (non-blocking, so nothing orders it against the legacy
default stream), and checks that the fractions are bit-identical: both paths
launch the same kernels on the same tiles and steps per launch.  It sits in a
file of its own that pytest collects last.
"""
import math

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


def test_noalloc_matches_context_path_on_two_calls():
    torch = pytest.importorskip("torch")
    import paper_2402_17580_gb300 as ms
    from paper_2402_17580_gb300 import _binding as B

    w = wl.block_256(dims=(40, 24, 9), n_tracks=4, n_steps=600, T_thr=0.0)
    sp = w.specimens[0]
    n = w.n_points
    n_pad = math.ceil(n / 128) * 128
    params = ms.default_params(T_thr=0.0, steps_per_launch=32)

    ctx = ms.Context(n, ms.default_params(T_thr=0.0, steps_per_launch=32))
    ctx.set_points([sp.grid])
    ctx.fill_state(0.9, 0.0)

    dev = torch.device("cuda", 0)
    xas = torch.full((n_pad,), 0.9, dtype=torch.float32, device=dev)
    xam = torch.zeros(n_pad, dtype=torch.float32, device=dev)
    aux = torch.zeros(n_pad, dtype=torch.float32, device=dev)
    side = torch.cuda.Stream(dev)        # created non-blocking by torch
    torch.cuda.synchronize()

    for step0, k, stream in ((0, 300, side), (300, 300, torch.cuda.current_stream(dev))):
        ctx.run_track([sp.source], k, w.dt)
        ref_as, ref_am = ctx.fractions(with_beta=False)
        # the raw per-point initiation state, from the context's checkpoint
        # (a 64-byte header, then X_as, X_am and aux in the padded layout)
        ref_aux = np.frombuffer(ctx.checkpoint(), dtype=np.float32, offset=64 + 2 * 4 * n_pad,
                                count=n)
        # the call returns once its stream has finished the work
        B.run_track_noalloc(params, sp.grid, sp.source, xas.data_ptr(), xam.data_ptr(),
                            aux.data_ptr(), n, step0, k, w.dt, stream.cuda_stream)
        got_as = xas[:n].double().cpu().numpy()
        got_am = xam[:n].double().cpu().numpy()
        got_aux = aux[:n].cpu().numpy()
        assert np.array_equal(got_as, ref_as), (step0, float(np.max(np.abs(got_as - ref_as))))
        assert np.array_equal(got_am, ref_am), (step0, float(np.max(np.abs(got_am - ref_am))))
        assert np.array_equal(got_aux, ref_aux), step0
    # the run did work: alpha_s dissolved where the tracks melted the block
    assert float(np.min(xas[:n].cpu().numpy())) < 0.5
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_limits():
    pytest.importorskip("torch")
    import paper_2402_17580_gb300 as ms
    from paper_2402_17580_gb300 import _binding as B
    import torch

    w = wl.block_256(dims=(16, 8, 2), n_tracks=2, n_steps=10, T_thr=0.0)
    sp = w.specimens[0]
    buf = torch.zeros(256, dtype=torch.float32, device="cuda")
    p = ms.default_params(steps_per_launch=65)
    with pytest.raises(ms.MSError) as e:
        B.run_track_noalloc(p, sp.grid, sp.source, buf.data_ptr(), buf.data_ptr(),
                            buf.data_ptr(), sp.grid.n, 0, 1, w.dt)
    assert e.value.code == -1
    many = wl.HeatSource(np.repeat(sp.source.tracks[:1], 129, axis=0), sp.source.layers)
    with pytest.raises(ms.MSError) as e:
        B.run_track_noalloc(ms.default_params(), sp.grid, many, buf.data_ptr(), buf.data_ptr(),
                            buf.data_ptr(), sp.grid.n, 0, 1, w.dt)
    assert e.value.code == -1
