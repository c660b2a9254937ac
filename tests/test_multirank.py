"""The N > 1 path of bench.py on CPU: two gloo ranks.

Each rank computes the map of its own core site (independent, translation-equivalent
problems, no collective on the data path); the only collectives are the max over ranks
of the timed seconds and the barriers around the timed region.  Here two spawned ranks
check the rank logic of bench.py, and that the two ranks' problems are indeed equivalent:
the oracle's maps of sites 0 and 1 of a small ring agree."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    from oracle import rixs as orixs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds = bench.max_over_ranks(1.5 + rank, world)      # rank 1 is the slow one
        site = bench.rank_core_site(rank, 4)
        sites = [None] * world
        dist.all_gather_object(sites, site)
        value = bench.job_throughput(1000.0, world, seconds)
        ref = orixs.rixs_map(4, 2, 2, 1.0, 8.0, 4.0, site, 0.3, 0.1, np.linspace(-4, 12, 5),
                             np.linspace(-1, 10, 30), cf_tol=1e-13)
        maps = [None] * world
        dist.all_gather_object(maps, ref.I)
        q.put((rank, seconds, sites, value, float(np.max(np.abs(maps[0] - maps[1])) / np.max(maps[0]))))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_bench_logic():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        results = sorted(q.get(timeout=180) for _ in procs)
    finally:
        for p in procs:
            p.join(60)
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0, 0]
    for rank, seconds, sites, value, diff in results:
        assert seconds == 2.5                      # the slowest rank's time, on every rank
        assert sites == [0, 1]                     # distinct core sites per rank
        assert value == pytest.approx(2 * 1000.0 / 2.5)
        assert diff <= 1e-10                       # site 0 and site 1 maps: the same problem


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.rank_core_site(13, 12) == 1
    assert bench.job_throughput(400.0, 1, 2.0) == 200.0
