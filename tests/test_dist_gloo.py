"""The multi-process path of bench.py on CPU (gloo, world size 2): every rank runs its own
replica of the workload (trials are independent, so no data-path collective); the timed
region ends with a barrier and the maximum of the per-rank times is reported."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        t = bench.max_over_ranks(1.5 + rank, world)
        # replicas: rank-seeded YETs differ, the portfolio does not
        import synth
        y = synth.paper_scale_yet(seed=rank, n_trials=4)
        out[rank] = (t, int(y.event_ids[:8].sum()))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_and_max_over_ranks():
    ctx = mp.get_context("spawn")
    world, port = 2, _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0][0] == out[1][0] == 2.5
        assert out[0][1] != out[1][1]
