"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): image
sharding for weak scaling and the max / sum reductions of the timed region."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        idx = bench.shard_indices(r, w, 5)
        t = torch.tensor(idx, dtype=torch.int64)
        gathered = [torch.zeros_like(t) for _ in range(w)]
        dist.all_gather(gathered, t)
        dev = torch.device("cpu")
        mx = bench.reduce_max(float(10 + rank), dist, dev)
        sm = bench.reduce_sum(float(rank + 1), dist, dev)
        out.put((rank, r, w, local, [g.tolist() for g in gathered], mx, sm))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_and_reductions():
    world = 2
    ctx = tmp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(world))
    for rank, r, w, local, gathered, mx, sm in res:
        assert (r, w, local) == (rank, world, rank)
        # ranks own disjoint, contiguous blocks of the seeded image sequence
        assert gathered == [[0, 1, 2, 3, 4], [5, 6, 7, 8, 9]]
        assert mx == 11.0 and sm == 3.0


def test_single_process_reductions_are_identity():
    assert bench.reduce_max(3.5) == 3.5
    assert bench.reduce_sum(2.0) == 2.0
    assert bench.shard_indices(0, 1) == list(range(bench.N_IMAGES))


def test_median_step_seconds_ignores_a_one_off_stall():
    import time
    calls = []

    def step():
        calls.append(1)
        time.sleep(0.06 if len(calls) == 2 else 0.002)  # one stall in the first run

    synced = []
    t = bench.median_step_seconds(step, steps=5, reps=3, sync=lambda: synced.append(1))
    assert len(calls) == 15 and len(synced) == 3
    assert 0.0015 < t < 0.008  # the stalled run (~14 ms per step) is not the median
