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


def test_roofline_accounting():
    # the algorithmic FLOPs and cells of a launch follow from the hierarchy:
    # leaves only (a patch with children is restricted, not advanced)
    sys.path.insert(0, ROOT)
    import bench
    from synth import workload
    w = workload('blast3d')
    ppl = [512, 512, 512, 0, 0, 0, 0, 0]
    assert bench.leaf_patches(w, ppl) == 512 - 64 + 512 - 64 + 512
    cc = bench.cell_counts(w, ppl[:3])
    assert cc['leaf_cells'] == 1408 * 4096 and cc['all_patch_cells'] == 1536 * 4096
    assert cc['stage_updates_per_step'] == 3 * cc['leaf_cells']
    assert cc['fine_equivalent'] == 512 ** 3

    class Fake:
        def diag(self):
            return 0.0, None, ppl

    flops = bench.load_json(bench.FLOPS_FILE, None)
    f = flops['3']
    got = bench.rhs_flops_per_launch(Fake(), w, flops)
    assert got == 1408 * 3 * 16 * 16 * 17 * f['face'] + 1408 * 4096 * f['cell']
    wc = workload('shear2d', dim=3, base_cells=(128, 128, 128), levels=3, patch=16)
    got = bench.rhs_flops_per_launch(Fake(), wc, flops)
    rows = 1408 * 3 * 16 * 16
    assert got == rows * (19 * f['face_central'] + 17 * f['face_combine_central']) + 1408 * 4096 * f['cell']
    assert bench.rhs_flops_per_launch(Fake(), workload('blast3d', flux='hllc'), flops) is None
    # the recorded DRAM bytes apply to the default workload, and only while the
    # kernel's sources hash as they did at capture (else null)
    assert bench.rhs_traffic('blast3d', 0, 0) in (bench.RHS_TRAFFIC['bytes'][0], None)
    assert (bench.rhs_traffic('blast3d', 0, 0) is None) == (bench.rhs_source_hash() != bench.RHS_TRAFFIC['hash'])
    # per tile shape: a shape without a capture has none
    assert bench.rhs_traffic('blast3d', 0, 0, shape=1) is None
    assert bench.rhs_traffic('blast3d', 64, 0) is None
    assert bench.rhs_traffic('dmr', 0, 0) is None


def test_run_planning_and_traffic_scaling():
    # chunks of a run to t_end: capped, and one step at a time near the end so
    # that no step is spent after t_end (the last one is clipped to it)
    sys.path.insert(0, ROOT)
    import bench
    assert bench.plan_chunk(0.0, 1e-5, 25) == 0
    assert bench.plan_chunk(1.0, 1e-5, 25) == 25
    assert bench.plan_chunk(10.5e-5, 1e-5, 25) == 8
    assert bench.plan_chunk(2.5e-5, 1e-5, 25) == 1
    assert bench.plan_chunk(1.0, 0.0, 25) == 1
    # the captured launch's DRAM bytes, scaled per leaf patch to another launch
    for shape, b in bench.RHS_TRAFFIC['bytes'].items():
        if bench.rhs_traffic('blast3d', 0, 0, shape=shape) is not None:
            assert bench.rhs_traffic('blast3d', 0, 0, bench.RHS_TRAFFIC['leaves'], shape) == b
            assert bench.rhs_traffic('blast3d', 0, 0, 2 * bench.RHS_TRAFFIC['leaves'], shape) == 2 * b


def test_level0_assembly():
    # level 0's patches placed by their coordinates into one (z, y, x) array
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench

    class Fake:
        dim, N = 3, 2

        def get_level(self, l):
            coords = np.array([[x, y, z] for z in range(2) for y in range(3) for x in range(2)])
            data = np.zeros((len(coords), 5, 2, 2, 2))
            for i, (x, y, z) in enumerate(coords):
                data[i, 0] = 100 * z + 10 * y + x
            return coords, data
    a = bench.level0_rho(Fake())
    assert a.shape == (4, 6, 4)
    assert a[3, 5, 3] == 100 * 1 + 10 * 2 + 1 and a[0, 0, 0] == 0 and a[2, 1, 1] == 100
    assert bench.l1_rel(a + 1.0, a + 1.0) == 0.0
