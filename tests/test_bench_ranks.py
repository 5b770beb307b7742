"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own
replica, combine into max elapsed time and total work."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(('127.0.0.1', 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ['MASTER_ADDR'] = '127.0.0.1'
    os.environ['MASTER_PORT'] = str(port)
    dist.init_process_group('gloo', rank=rank, world_size=world)
    import bench
    el, units = bench.combine_ranks(1.0 + rank, 10.0 * (rank + 1), dist)
    out.put((rank, el, units))
    dist.destroy_process_group()


def test_two_ranks_max_time_total_work():
    torch = pytest.importorskip('torch')
    mp = torch.multiprocessing.get_context('spawn')
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, el, units in res:
        assert el == 2.0 and units == 30.0


def test_single_process_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(3.0, 7.0, None) == (3.0, 7.0)
