"""Benchmark: split-CTMRG free energy + gradient evaluations per second (arXiv:2506.19339).

One step = one f + grad f evaluation of the workload: the numerator <psi|T|psi> and norm <psi|psi>
environments are reset to the cold start and iterated (left, right, up, down moves per
iteration; Sec. III.B) for a fixed budget of iterations (or until ||dS||_2 < tol), then f and g
are evaluated (Sec. II).  Everything runs through the C ABI of libsctm.so.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--iters I] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun with N > 1 every rank runs an independent replica
(the single-instance path does not shard) and `value` is the sum over ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "split-CTMRG f+∇f evals/s at D=4 χ=64, mixed vs FP64 at |Δf|≤1e-8; % of peak"
WORKLOAD = dict(D=4, chi=64, T=4.5, seed=2)   # the configuration the metric is quoted on
NOMINAL_FP64_TFLOPS = 1.25                     # GB300 FP64 (vector and tensor), nominal
NOMINAL_BF16_TFLOPS = 2250.0
PRECISIONS = {'fp64': 0, 'tf32': 1, 'tf32x3': 2, 'bf16': 3, 'bf16x3': 4, 'f64emu': 5}
SVD_MODES = {'qr': 0, 'polar': 1, 'partial': 2, 'partial-random': 3}
SVD_NAMES = {'qr': 'cuSOLVER gesvd', 'polar': 'cuSOLVER gesvdp',
             'partial': 'partial SVD: gesvd cold solve, then warm-started subspace iteration + '
                        'one-CTA Jacobi',
             'partial-random': 'partial SVD: randomized cold solve (2 subspace steps), then '
                               'warm-started subspace iteration + one-CTA Jacobi'}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=3)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--iters', type=int, default=10, help='split-CTMRG iterations per evaluation')
    ap.add_argument('--tol', type=float, default=1e-10)
    ap.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--batch', type=int, default=0,
                    help='batched sweep: B contexts (T uniform in [4.40, 4.62], seeds 100..) '
                         'iterated concurrently; 0 = the single-instance workload')
    ap.add_argument('--svd', default='partial-random', choices=list(SVD_MODES),
                    help='FP64 SVD of the projectors: the partial SVD with a randomized cold '
                         'solve (partial-random) or a gesvd cold solve (partial), cuSOLVER gesvd '
                         '(qr) or gesvdp (polar)')
    ap.add_argument('--D', type=int, default=None,
                    help='override the PEPS bond dimension (small cases for profiler captures)')
    ap.add_argument('--chi', type=int, default=None, help='override chi (profiler captures)')
    ap.add_argument('--precision', default='fp64', choices=list(PRECISIONS),
                    help='arithmetic of the move contractions (mixed forms polish in FP64)')
    return ap.parse_args()


def workload_name(it, w=None):
    w = w or WORKLOAD
    return ('split-CTMRG f+grad, 3D Ising PEPO, PEPS D=%d N(0,1) seed %d, chi=%d, T=%g, '
            '%d iterations (num + norm networks) per evaluation, tol %g' %
            (w['D'], w['seed'], w['chi'], w['T'], it, 1e-10))


# ------------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
              'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
              'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, gpu=0):
        self.gpu = gpu
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(['nvidia-smi', '-i', str(self.gpu), '--query-gpu=' + self.FIELDS,
                                          '--format=csv,noheader,nounits', '-lms', '200'],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(',')]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)
        sm = [float(s[1]) for s in self.samples if s[1].replace('.', '').isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace('.', '').isdigit()]
        reasons = set()
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        for s in self.samples:
            for name, v in zip(names, s[5:9]):
                if v.lower().startswith('active'):
                    reasons.add(name)
        return {'sm_mhz': float(np.median(sm)) if sm else None,
                'sm_max_mhz': max(mx) if mx else None,
                'reasons': sorted(reasons), 'samples': len(self.samples)}


# ------------------------------------------------------------------------------------------------
# CPU baseline / reference arm: the FP64 oracle on the host cores
# ------------------------------------------------------------------------------------------------
def oracle_sample(A, T, chi, iters, budget_s=20.0):
    """Time the oracle on a bounded sample: moves of the numerator then the norm network (4 moves
    per iteration each) until `budget_s` of CPU work; scale to evaluations/s at `iters` iterations
    per evaluation."""
    from oracle import ising, split_ctmrg as sc
    D = A.shape[1]
    nets = [ising.ising_pepo(1.0 / T), ising.identity_pepo()]
    moves_done = [0, 0]
    secs = [0.0, 0.0]
    for n, O in enumerate(nets):
        env = sc.init_env(chi, D, O.shape[2])
        t0 = time.perf_counter()
        for w in 'LRUD':
            env = sc.move(env, A, O, A, w, chi)
            moves_done[n] += 1
            if time.perf_counter() - t0 > budget_s / 2:
                break
        secs[n] = time.perf_counter() - t0
    per_move = [secs[n] / moves_done[n] for n in range(2)]
    sec_per_eval = 4 * iters * (per_move[0] + per_move[1])
    sample = ('%d numerator + %d norm left/right/up/down moves of the FP64 oracle at the workload '
              'size (%.1f s), scaled to %d iterations x 4 moves x 2 networks per evaluation' %
              (moves_done[0], moves_done[1], secs[0] + secs[1], iters))
    return 1.0 / sec_per_eval, sample, secs[0] + secs[1]


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference(args):
    from paper_2506_19339_gb300 import inputs
    w = WORKLOAD
    rank = int(os.environ.get('RANK', '0'))
    if rank != 0:
        return
    A = inputs.random_peps(w['D'], w['seed'])
    budget = max(2.0, min(20.0, 150.0 / max(args.steps + args.warmup, 1)))
    for _ in range(args.warmup):
        oracle_sample(A, w['T'], w['chi'], args.iters, budget_s=budget / 4)
    vals = []
    samples = []
    for _ in range(args.steps):
        v, sample, secs = oracle_sample(A, w['T'], w['chi'], args.iters, budget_s=budget)
        vals.append(v)
        samples.append(secs)
    value = float(np.mean(vals))
    line = {
        'impl': 'reference', 'metric': METRIC, 'value': value, 'unit': 'evals/s',
        'n_gpus': args.gpus, 'steps': args.steps, 'warmup': args.warmup,
        'ms_per_step': 1000.0 / value, 'higher_is_better': True, 'scaling': 'weak',
        'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic',
        'config': {'workload': workload_name(args.iters), 'D': w['D'], 'chi': w['chi'],
                   'T': w['T'], 'seed': w['seed'], 'iterations_per_eval': args.iters},
        'cpu_baseline': {'value': value, 'unit': 'evals/s', 'cores': cpu_cores(), 'kind': 'oracle',
                         'sample': sample},
        'e2e': {'value': value, 'unit': 'evals/s', 'h2d_bytes_per_step': 0,
                'd2h_bytes_per_step': 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------
def combine_ranks(ms, e2e_ms, dist, device):
    """The timed totals of this rank (device-timed ms, end-to-end ms) -> the maximum over all
    ranks (every rank gets it).  Replicas run independently; the slowest rank sets the time of
    the whole job, and value = (evaluations of all ranks) / that time."""
    if not dist:
        return ms, e2e_ms
    import torch
    t = torch.tensor([ms, e2e_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0]), float(t[1])


def run_ours(args):
    import torch
    from paper_2506_19339_gb300 import build, inputs, sctm
    w = dict(WORKLOAD)
    if args.D:
        w['D'] = args.D
    if args.chi:
        w['chi'] = args.chi
    world = int(os.environ.get('WORLD_SIZE', '1'))
    rank = int(os.environ.get('RANK', '0'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group('nccl')
    dev = torch.device('cuda', local)
    torch.cuda.set_device(dev)
    build.build()
    sctm.load()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        A_cpu = inputs.random_peps(w['D'], w['seed'])
        v, sample, secs = oracle_sample(A_cpu, w['T'], w['chi'], args.iters, budget_s=20.0)
        cpu = {'value': v, 'unit': 'evals/s', 'cores': cpu_cores(), 'kind': 'oracle',
               'sample': sample}

    A_host = inputs.random_peps(w['D'], w['seed'])
    st, O = sctm.sctm_ising_pepo(w['T'])
    stream = torch.cuda.current_stream(dev)
    st, o = sctm.sctm_default_opts()
    o.T, o.D, o.p, o.d = w['T'], w['D'], 2, 2
    o.cuda_stream = stream.cuda_stream
    o.svd_mode = SVD_MODES[args.svd]
    o.precision = PRECISIONS[args.precision]
    A_dev = torch.from_numpy(A_host).to(dev)
    st, ctx = sctm.sctm_create(A_dev, np.ascontiguousarray(O), w['chi'], o)
    if st != sctm.SCTM_OK:
        raise RuntimeError('sctm_create failed: %s' % sctm.STATUS_NAMES[st])
    g_dev = torch.zeros_like(A_dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (126 MB)

    def evaluate(A_ptr, g_ptr):
        assert sctm.sctm_set_peps(ctx, A_ptr, 1) == sctm.SCTM_OK
        st, it, ds = sctm.sctm_iterate(ctx, args.iters, args.tol)
        assert st in (sctm.SCTM_OK, sctm.SCTM_ENOCONV), sctm.sctm_last_error(ctx)
        st, f = sctm.sctm_free_energy(ctx)
        st2 = sctm.sctm_grad(ctx, g_ptr)
        return f, it, ds, st

    # warm-up
    for _ in range(args.warmup):
        evaluate(A_dev, g_dev)
    torch.cuda.synchronize(dev)

    # ---- timed region, device-resident inputs
    sctm.sctm_profile(ctx, reset=True)
    sctm.sctm_set_profiling(ctx, True)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    step_ms = []
    its = []
    fs = []
    statuses = []
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f, it, ds, stf = evaluate(A_dev, g_dev)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        its.append(it)
        fs.append(f)
        statuses.append(stf)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    sctm.sctm_set_profiling(ctx, False)
    kern = {name: sctm.sctm_profile_kernel(ctx, k)[1] for name, k in
            (('ctr_f64_kernel', sctm.SCTM_KERNEL_F64), ('ctr_skinny_kernel', sctm.SCTM_KERNEL_SKINNY),
             ('ctr_tc_kernel', sctm.SCTM_KERNEL_TC), ('emu_ctr_kernel', sctm.SCTM_KERNEL_F64EMU))}
    st, prof = sctm.sctm_profile(ctx, reset=True)
    ms = float(np.sum(step_ms))

    # ---- e2e: host buffers through the C ABI, host<->device copies inside the timed region
    A_pin = torch.from_numpy(A_host).pin_memory()
    g_pin = torch.zeros(A_host.shape, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize(dev)
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        evaluate(A_pin.numpy(), g_pin.numpy())
        torch.cuda.synchronize(dev)
        e2e_ms.append(1000.0 * (time.perf_counter() - t0))
    st, prof_e2e = sctm.sctm_profile(ctx, reset=True)

    # FP64 matrix-multiply rate of this GPU (cuBLAS through torch), context for the roofline
    a = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    torch.matmul(a, a)
    torch.cuda.synchronize(dev)
    best = 1e9
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, a)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    dgemm_tflops = 2 * 4096 ** 3 / (best * 1e-3) / 1e12
    sctm.sctm_destroy(ctx)

    # max over ranks
    ms, e2e_total = combine_ranks(ms, float(np.sum(e2e_ms)), dist, dev)
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, 'MEASURED_PEAKS.json')))
    except (OSError, ValueError):
        pass
    if 'bf16_tflops_sustained' in peaks:
        fp64_peak = peaks['bf16_tflops_sustained'] * NOMINAL_FP64_TFLOPS / NOMINAL_BF16_TFLOPS
        peak_note = 'measured bf16 sustained x nominal FP64/BF16 ratio (1.25/2250)'
    else:
        fp64_peak = 1700.0 * NOMINAL_FP64_TFLOPS / NOMINAL_BF16_TFLOPS
        peak_note = 'fallback bf16 sustained x nominal FP64/BF16 ratio'
    kf = kern['ctr_f64_kernel']
    achieved = (kf['flops'] / (kf['ms'] * 1e-3) / 1e12) if kf['ms'] > 0 else None
    hbm = peaks.get('hbm_gbs', 6800.0)
    kernels = {}
    for name, kv in kern.items():
        if kv['launches'] == 0:
            continue
        sec = kv['ms'] * 1e-3
        kernels[name] = {'launches_per_step': kv['launches'] / args.steps,
                         'ms_per_step': kv['ms'] / args.steps,
                         'tflops': kv['flops'] / sec / 1e12 if sec > 0 else None,
                         'min_gbs': kv['bytes'] / sec / 1e9 if sec > 0 else None}
    if 'ctr_skinny_kernel' in kernels and kernels['ctr_skinny_kernel']['min_gbs']:
        kernels['ctr_skinny_kernel']['frac_of_hbm'] = kernels['ctr_skinny_kernel']['min_gbs'] / hbm
    # the step is FP64-bound as a whole: FP64 contraction FLOPs of the step over its device time
    f64_flops = sum(kern[k]['flops'] for k in ('ctr_f64_kernel', 'ctr_skinny_kernel'))
    gpu_wide = f64_flops / (ms * 1e-3) / 1e12 if ms > 0 else None
    n_steps = args.steps * world
    value = n_steps / (ms * 1e-3)
    total_its = int(np.sum(its))
    line = {
        'metric': METRIC, 'value': value, 'unit': 'evals/s', 'n_gpus': world,
        'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': ms / args.steps,
        'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None,
        'dtype': 'f64' if args.precision == 'fp64' else args.precision + '+f64',
        'data': 'synthetic',
        'config': {'workload': workload_name(args.iters, w), 'D': w['D'], 'chi': w['chi'],
                   'T': w['T'], 'seed': w['seed'], 'iterations_per_eval': args.iters,
                   'precision': '%s move contractions, FP64 SVD (%s)' % (
                       args.precision.upper(), SVD_NAMES[args.svd]),
                   'parallelism': 'replicas',
                   'l2': 'flushed before every step (256 MiB write, outside the step events)'},
        'iterations_per_s': total_its * world / (ms * 1e-3),
        'f': fs[-1], 'status': [sctm.STATUS_NAMES[s] for s in statuses][-1],
        'roofline': {'bound': 'alu', 'kernel': 'ctr_f64_kernel', 'achieved': achieved,
                     'peak': fp64_peak, 'unit': 'TFLOP/s',
                     'frac': (achieved / fp64_peak) if achieved else None, 'traffic': None,
                     'peak_note': peak_note, 'dgemm_torch_tflops': dgemm_tflops,
                     'kernels': kernels,
                     'step_fp64_contraction_tflops': gpu_wide,
                     'step_fp64_contraction_frac': (gpu_wide / fp64_peak) if gpu_wide else None,
                     'ctr_ms_per_step': prof['ctr_ms'] / args.steps,
                     'svd_ms_per_step': prof['svd_ms'] / args.steps,
                     'ctr_launches_per_step': prof['ctr_launches'] / args.steps,
                     'svd_calls_per_step': prof['svd_calls'] / args.steps},
        'cpu_baseline': cpu,
        'e2e': {'value': n_steps / (e2e_total * 1e-3), 'unit': 'evals/s',
                'h2d_bytes_per_step': int(A_host.nbytes),
                'd2h_bytes_per_step': int(A_host.nbytes + 8)},
        'clocks': clk,
        'gpu_launches': int(prof['kernel_launches']),
        'wall_s': wall,
    }
    print(json.dumps(line), flush=True)


def run_batch(args):
    """The batched sweep: B independent evaluations of (D=4, chi=64) at B temperatures, iterated
    concurrently through sctm_iterate_batch; value = evaluations per second of the whole batch."""
    import torch
    from paper_2506_19339_gb300 import build, inputs, sctm
    w = WORKLOAD
    B = args.batch
    dev = torch.device('cuda', 0)
    build.build()
    sctm.load()
    Ts = inputs.temperature_sweep(B)
    streams = [torch.cuda.Stream(dev) for _ in range(B)]
    ctxs, As, gs = [], [], []
    for i, T in enumerate(Ts):
        A = torch.from_numpy(inputs.random_peps(w['D'], 100 + i)).to(dev)
        st, O = sctm.sctm_ising_pepo(T)
        st, o = sctm.sctm_default_opts()
        o.T, o.D, o.p, o.d = float(T), w['D'], 2, 2
        o.cuda_stream = streams[i].cuda_stream
        o.svd_mode = SVD_MODES[args.svd]
        o.precision = PRECISIONS[args.precision]
        st, ctx = sctm.sctm_create(A, np.ascontiguousarray(O), w['chi'], o)
        if st != sctm.SCTM_OK:
            raise RuntimeError('sctm_create failed for batch member %d: %s' % (i, sctm.STATUS_NAMES[st]))
        ctxs.append(ctx)
        As.append(A)
        gs.append(torch.zeros_like(A))
    mem = sum(sctm.sctm_device_bytes(c) for c in ctxs)

    def step():
        for c, A in zip(ctxs, As):
            assert sctm.sctm_set_peps(c, A, 1) == sctm.SCTM_OK
        st, sts, its, dss = sctm.sctm_iterate_batch(ctxs, args.iters, args.tol)
        for c, g in zip(ctxs, gs):
            sctm.sctm_free_energy(c)
            sctm.sctm_grad(c, g)
        return its

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(0)
    clocks.start()
    ms = []
    for _ in range(args.steps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        its = step()
        torch.cuda.synchronize(dev)
        ms.append(1000.0 * (time.perf_counter() - t0))
    clk = clocks.stop()
    for c in ctxs:
        sctm.sctm_destroy(c)
    total = float(np.sum(ms))
    line = {
        'metric': METRIC, 'value': B * args.steps / (total * 1e-3), 'unit': 'evals/s', 'n_gpus': 1,
        'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': total / args.steps,
        'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64',
        'data': 'synthetic',
        'config': {'workload': 'batched sweep: %d contexts, T uniform in [4.40, 4.62], PEPS D=%d '
                               'N(0,1) seeds 100..%d, chi=%d, %d iterations per evaluation, '
                               '%s, SVD %s, iterated concurrently (one host thread and stream '
                               'set per context)' % (B, w['D'], 99 + B, w['chi'], args.iters,
                                                     args.precision.upper(), args.svd),
                   'batch': B, 'iterations_per_eval': args.iters, 'device_bytes': mem,
                   'timing': 'host wall clock around each step with device synchronisation'},
        'clocks': clk,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.batch > 0:
        run_batch(args)
        return
    if args.impl == 'reference':
        run_reference(args)
    else:
        run_ours(args)


if __name__ == '__main__':
    main()
