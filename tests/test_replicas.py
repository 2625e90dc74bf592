"""The multi-GPU path is replicas only (one evaluation does not shard): the per-rank timings are
combined by a MAX all-reduce.  Checked here with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip('torch')

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ['MASTER_ADDR'] = '127.0.0.1'
    os.environ['MASTER_PORT'] = str(port)
    dist.init_process_group('gloo', rank=rank, world_size=world)
    ms, e2e = bench.combine_ranks(100.0 + 50.0 * rank, 300.0 - 10.0 * rank, dist, 'cpu')
    with open(os.path.join(out, 'r%d.txt' % rank), 'w') as f:
        f.write('%r %r' % (ms, e2e))
    dist.destroy_process_group()


def test_combine_ranks_takes_the_slowest(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        ms, e2e = map(float, open(tmp_path / ('r%d.txt' % r)).read().split())
        assert ms == 150.0 and e2e == 300.0


def test_combine_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(12.5, 20.0, None, 'cpu') == (12.5, 20.0)
