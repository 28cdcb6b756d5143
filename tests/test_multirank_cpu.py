"""Multi-rank path on CPU (gloo, world size 2).

The method shards with no exchange step: every rank advances its own
specimens.  These tests run the sharding and the timing reduction of the
multi-GPU bench as two gloo ranks on the CPU, with the FP64 oracle doing the
per-rank work, and check that (a) the merged result is bit-identical to the
unsharded run, (b) the max-over-ranks reduction is what bench.py reports,
and (c) a rank that fails before the barrier is detected by the other rank
within the process-group timeout instead of hanging it.
"""
import datetime
import os
import socket
import time

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2402_17580_gb300.shard import imbalance, shard_slabs, shard_specimens


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _oracle_specimen(w, s):
    import oracle as orc
    sp = w.specimens[s]
    x, y, z = sp.grid.coords()
    st = orc.State.uniform(sp.grid.n, 0.9, 0.0)
    T = orc.run_track(st, sp.source, x, y, z, 0, w.n_steps, w.dt)
    return np.stack(orc.fractions(st, T))


def _small_batch():
    import workloads as wl
    return wl.batch_64(n_specimens=6, n_lo=100, n_hi=900, n_steps=300, T_thr=0.0)


def _worker(rank, world, port, mode, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1")
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=8))
    try:
        if mode == "fail" and rank == 1:
            raise RuntimeError("rank 1 fails before the barrier")
        w = _small_batch()
        parts = shard_specimens([s.grid.n for s in w.specimens], world)
        mine = {s: _oracle_specimen(w, s) for s in parts[rank]}
        t_local = float(1.0 + rank)
        t = [None] * world
        dist.all_gather_object(t, t_local)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        dist.barrier()
        if rank == 0:
            merged = {}
            for g in gathered:
                merged.update(g)
            q.put(("ok", rank, merged, max(t)))
    except Exception as e:  # reported to the parent, never swallowed
        q.put(("error", rank, repr(e), None))
        raise
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    # drain the queue before joining: a child cannot exit while its queued
    # results are still buffered
    import queue
    out, deadline = [], time.time() + 120
    expected = 1 if mode == "ok" else 2
    while len(out) < expected and time.time() < deadline:
        try:
            out.append(q.get(timeout=1.0))
        except queue.Empty:
            if not any(p.is_alive() for p in procs):
                break
    for p in procs:
        p.join(timeout=max(1.0, deadline - time.time()))
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    while not q.empty():
        out.append(q.get())
    return codes, out


def test_shard_helpers():
    sizes = [5, 1, 9, 3, 3, 7, 2]
    parts = shard_specimens(sizes, 3)
    assert sorted(i for p in parts for i in p) == list(range(len(sizes)))
    assert imbalance(sizes, parts) < 1.2
    assert shard_slabs(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert shard_slabs(2, 4) == [(0, 1), (1, 2), (2, 2), (2, 2)]


def test_two_gloo_ranks_merge_bit_exact():
    codes, out = _run("ok")
    assert codes == [0, 0], out
    status, _, merged, tmax = out[0]
    assert status == "ok" and tmax == 2.0
    w = _small_batch()
    assert sorted(merged) == list(range(len(w.specimens)))
    for s in range(len(w.specimens)):
        assert np.array_equal(merged[s], _oracle_specimen(w, s))


def test_failed_rank_is_detected():
    codes, out = _run("fail")
    assert codes[1] != 0
    errs = {r: msg for status, r, msg, _ in out if status == "error"}
    assert 1 in errs and "rank 1 fails" in errs[1]
    assert codes[0] != 0 or 0 in errs   # rank 0 learns of it (error or timeout), no hang
