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


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores, a bounded sample per step)
    prints one JSON line with the contract's keys; its ms_per_step is the sample's measured time
    and the value scales the sample to a converged evaluation (a small workload here)."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, 'bench.py'), '--impl', 'reference',
                          '--steps', '1', '--warmup', '0', '--D', '2', '--chi', '6'],
                         cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ('impl', 'metric', 'value', 'unit', 'n_gpus', 'steps', 'warmup', 'ms_per_step',
                'higher_is_better', 'scaling', 'vs_baseline', 'dtype', 'data', 'config',
                'cpu_baseline', 'e2e'):
        assert key in line, key
    assert line['impl'] == 'reference' and line['unit'] == 'evals/s' and line['value'] > 0
    assert line['cpu_baseline']['value'] == line['value'] and line['cpu_baseline']['kind'] == 'oracle'
    assert line['e2e']['h2d_bytes_per_step'] == 0 and line['e2e']['d2h_bytes_per_step'] == 0
    # the step is the bounded sample, much shorter than the evaluation it is scaled to
    assert line['ms_per_step'] < 1000.0 * line['sec_per_eval_extrapolated']


def test_bench_option_logic():
    """The bench's defaults (FP64 emulation, randomized partial SVD, directional scheme, the
    cluster Jacobi kernel; the one-CTA kernel for the D2 scheme) and its stored oracle values: each
    method and projector-4 choice finds the golden file of its own reading at the workload size."""
    import importlib
    sys.path.insert(0, ROOT)
    bench = importlib.import_module('bench')
    saved = sys.argv
    try:
        sys.argv = ['bench.py']
        args = bench.parse()
        assert (args.precision, args.svd, args.method) == ('f64emu', 'partial-random', 'split')
        assert bench.jacobi_kernel(args) == 'cluster'
        args.method = 'split-d2'
        assert bench.jacobi_kernel(args) == 'cta'
        w = bench.workload(bench.parse())
        fs = {}
        for key in ('split', 'split-half-p4', 'split-d2'):
            g = bench.load_golden(w, key)
            assert g is not None, key
            rec = g['records'].get('converged') or g['records'].get('fixed')
            assert len(rec['g']) == 2 * w['D'] ** 4
            fs[key] = rec['f']
        # the two projector-4 readings agree in f to the bench's acceptance bound
        assert abs(fs['split'] - fs['split-half-p4']) <= bench.ACCEPT_DF
        assert bench.load_golden(dict(w, chi=32), 'split') is None
    finally:
        sys.argv = saved
