"""Multi-rank logic of bench.py on CPU (gloo, world size 2): ranks take
disjoint energies (weak scaling, no data-path collective), and the timing
reductions return the max / sum over ranks."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist, r, local, w = bench.dist_init()
    assert (r, w) == (rank, world)
    idx = [bench.energy_index(r, w, k) for k in range(64)]
    import torch
    gathered = [None] * w
    dist.all_gather_object(gathered, idx)
    mx = bench.max_over_ranks(dist, float(rank + 1) * 1.5)
    sm = bench.sum_over_ranks(dist, float(rank + 1))
    out.put((rank, gathered, mx, sm))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_energy_sharding_and_reductions():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, mx, sm in results:
        assert mx == 3.0 and sm == 3.0
        a, b = gathered
        assert len(set(a)) == 64 and len(set(b)) == 64  # no energy repeats on a rank
        assert not set(a) & set(b)  # disjoint across ranks
        assert all(0 <= i < 128 for i in a + b)
