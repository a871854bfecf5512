"""The bench's multi-process path, run as two gloo ranks on the CPU.

Under torchrun every rank simulates its own circuit (replicas: the method has no
data-path exchange on one circuit).  The only collectives are the timing barrier and
the reductions that form the JSON line: the slowest rank's time (max) and the events of
all ranks (sum).  The reference arm runs on rank 0 alone; other ranks exit without work.
"""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = torch.multiprocessing


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    import torch.distributed as dist

    ws, r, local = bench._dist()
    assert dist.is_initialized() and dist.get_backend() == "gloo"
    bench._barrier(ws)
    secs = [0.25, 0.75][r]            # per-rank timed region
    events = [1000.0, 3000.0][r]      # per-rank events
    t = bench._max_over_ranks(secs, ws)
    e = bench._sum_over_ranks(events, ws)
    ref = None
    if r != 0:
        class A:  # the reference arm's arguments; rank 1 must not touch them
            pass
        ref = bench.run_reference(A())
    out.put((r, ws, local, t, e, ref))
    dist.destroy_process_group()


def test_two_rank_reductions_and_reference_arm():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for r, ws, local, t, e, ref in res:
        assert ws == 2 and local == r
        assert t == 0.75             # value = all ranks' events / the slowest rank's time
        assert e == 4000.0
    assert res[1][5] == 0            # rank 1 leaves the reference arm at once


def test_single_process_needs_no_process_group(monkeypatch):
    import bench

    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "0")
    ws, r, _ = bench._dist()
    assert (ws, r) == (1, 0)
    assert bench._max_over_ranks(1.5, ws) == 1.5 and bench._sum_over_ranks(2.0, ws) == 2.0
