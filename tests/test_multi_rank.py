"""Multi-GPU host logic on CPU ranks (gloo, world size 2): images are
independent, so ranks solve disjoint seeds and the job time is the max over
ranks; no data-path collective exists."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist            # noqa: E402
import torch.multiprocessing as mp          # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seeds = bench.rank_seeds(rank, 5)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    t = bench.reduce_max(1.0 + rank)
    # each rank's inputs are generated locally from its own seeds
    import synth
    job = synth.custom(seeds[0], 6, 5, 4, 2, 100)
    hs = [None] * world
    dist.all_gather_object(hs, float(abs(job.R).sum()))
    if rank == 0:
        out.put((gathered, t, hs))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, t, hs = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert set(gathered[0]).isdisjoint(gathered[1])
    assert len(gathered[0]) == len(gathered[1]) == 5
    assert t == 2.0
    assert hs[0] != hs[1]


def test_single_rank_max_is_identity():
    import bench
    assert bench.reduce_max(3.5) == 3.5
