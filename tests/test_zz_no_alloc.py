"""The allocation-free contraction entry point (sctm_gemm_noalloc), for callers that cannot
allocate device memory.  It is checked against the context-based entry points: Z00 of an
environment (the trace of the corner product, Sec. II) computed with it must equal what
sctm_local_values returns for the same environment, on two calls in a row (the shared scratch
keeps the first call's contents)."""
import numpy as np
import pytest

from paper_2506_19339_gb300 import build, inputs, sctm

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _gemm(X, Y):
    import torch
    M, K = X.shape
    N = Y.shape[1]
    O = torch.full((M, N), float('nan'), dtype=torch.float64, device='cuda')
    st = sctm.sctm_gemm_noalloc(X, Y, O, M, N, K)
    torch.cuda.synchronize()
    assert st == sctm.SCTM_OK, sctm.STATUS_NAMES[st]
    return O


def test_no_alloc_matches_local_values():
    build.build()
    sctm.load()
    T, chi, D = 4.6, 24, 2          # chi^2 = 576 > 256: the final sum runs split-K
    A = inputs.perturbed_product_peps(D, 7)
    st, O = sctm.sctm_ising_pepo(T)
    r = sctm.SplitCTMRG(A, O, chi, T)
    try:
        r.iterate(2)
        st, vals = sctm.sctm_local_values(r.ctx, sctm.SCTM_NET_NUM)
        assert st == sctm.SCTM_OK
        env = r.env(sctm.SCTM_NET_NUM)
    finally:
        r.close()
    z00_ref = vals[0]
    C1, C2, C3, C4 = (env[k] for k in ('C1', 'C2', 'C3', 'C4'))
    for call in range(2):
        P = _gemm(_dev(C1.T), _dev(C2))               # C1^T C2
        Q = _gemm(_dev(C4.T), _dev(C3))               # C4^T C3
        z = _gemm(P.reshape(1, chi * chi), Q.reshape(chi * chi, 1))
        z00 = float(z.cpu().numpy()[0, 0])
        assert abs(z00 - z00_ref) <= 1e-12 * abs(z00_ref), (call, z00, z00_ref)


def test_no_alloc_general_shapes_and_limits():
    """Split-K and single-pass shapes against numpy, and the documented size limit."""
    import torch
    build.build()
    sctm.load()
    rng = np.random.default_rng(3)
    for (M, N, K) in [(5, 7, 20000), (300, 200, 500), (1, 1, 1)]:
        X = rng.standard_normal((M, K))
        Y = rng.standard_normal((K, N))
        for _ in range(2):
            got = _gemm(_dev(X), _dev(Y)).cpu().numpy()
            assert np.abs(got - X @ Y).max() <= 1e-12 * np.abs(X).max() * np.abs(Y).max() * K
    M, N = (1 << 11) + 1, 1 << 10          # M*N = 2^21 + 2^10 doubles: above the scratch limit
    X = torch.zeros(M, 1, dtype=torch.float64, device='cuda')
    Y = torch.zeros(1, N, dtype=torch.float64, device='cuda')
    O = torch.zeros(M, N, dtype=torch.float64, device='cuda')
    assert sctm.sctm_gemm_noalloc(X, Y, O, M, N, 1) == sctm.SCTM_EINVAL
    host = np.zeros((2, 2))
    assert sctm.sctm_gemm_noalloc(host, host, host, 2, 2, 2) == sctm.SCTM_EINVAL


def test_no_alloc_warm_calls_leave_free_memory_unchanged():
    """After one warm call (which loads the module and looks up the scratch address), further
    calls -- single-pass and split-K shapes -- must not change the device's free memory: the
    entry point allocates nothing.  Every tensor is allocated before the first reading."""
    import torch
    build.build()
    sctm.load()
    rng = np.random.default_rng(5)
    shapes = [(5, 7, 20000), (300, 200, 500), (64, 64, 4096)]
    ops = []
    for (M, N, K) in shapes:
        X, Y = _dev(rng.standard_normal((M, K))), _dev(rng.standard_normal((K, N)))
        O = torch.zeros((M, N), dtype=torch.float64, device='cuda')
        ops.append((X, Y, O, M, N, K))
    X, Y, O, M, N, K = ops[0]
    assert sctm.sctm_gemm_noalloc(X, Y, O, M, N, K) == sctm.SCTM_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        for (X, Y, O, M, N, K) in ops:
            assert sctm.sctm_gemm_noalloc(X, Y, O, M, N, K) == sctm.SCTM_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
