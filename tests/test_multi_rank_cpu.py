"""Host logic of the multi-GPU path on CPU: two gloo ranks shard the
frequencies (disjoint, together the full set, equal counts: weak scaling)
and take the max of their timings, with no data-path collective."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    om = bench.shard_frequencies(32, rank, world)
    mx = bench.barrier_max(dist, float(rank + 1) * 10.0)
    gathered = [None] * world
    dist.all_gather_object(gathered, om.tolist())
    if rank == 0:
        out.put((gathered, mx))
    dist.destroy_process_group()


def test_two_rank_frequency_sharding_and_max_timing():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, mx = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert mx == 20.0
    a, b = (np.array(x) for x in gathered)
    assert len(a) == len(b) == 32
    assert not set(a.round(12)) & set(b.round(12))
    import scenario as S
    np.testing.assert_allclose(np.sort(np.concatenate([a, b])), S.freq_list(64), rtol=0, atol=1e-15)
