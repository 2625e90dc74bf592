"""GPU: the mixed-precision forms of the contractions (tensor cores, tcgen05) against FP64.

The kernel test bounds the elementwise error by c (|X||Y|)_ij, c from the operand format: the hi
part of x keeps the format's significand (11 bits TF32, 8 bits BF16), the hi/lo pair about twice
that, and the FP32 accumulator adds ~sqrt(K) 2^-24 on random data.  The iteration tests check
that a mixed-form run followed by the FP64 polish reaches the FP64 fixed point (f to 1e-10), and
that a run of mixed-form iterations alone lands within the form's error of the FP64 one."""
import numpy as np
import pytest

from oracle import ising, split_ctmrg as sc
from paper_2506_19339_gb300 import build, inputs, sctm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip('torch')

FORMS = {
    # precision: (elementwise c in |O - XY| <= c |X||Y|, relative Frobenius error bound)
    sctm.SCTM_PREC_FP64: (1e-13, 1e-14),
    sctm.SCTM_PREC_TF32: (2e-3, 1e-3),
    sctm.SCTM_PREC_TF32X3: (2e-5, 2e-6),
    sctm.SCTM_PREC_BF16: (1.6e-2, 8e-3),
    sctm.SCTM_PREC_BF16X3: (1e-4, 3e-5),
    # eight 7-bit digits per element: 56 bits against each row's (column's) maximum
    sctm.SCTM_PREC_F64EMU: (1e-13, 1e-13),
}


@pytest.fixture(scope='module', autouse=True)
def lib():
    build.build()
    return sctm.load()


def _gemm(X, Y, prec):
    M, K = X.shape
    N = Y.shape[1]
    dX = torch.from_numpy(X).cuda()
    dY = torch.from_numpy(Y).cuda()
    dO = torch.full((M, N), float('nan'), dtype=torch.float64, device='cuda')
    torch.cuda.synchronize()
    st = sctm.sctm_gemm(dX, dY, dO, M, N, K, prec, torch.cuda.current_stream().cuda_stream)
    assert st == sctm.SCTM_OK, st
    return dO.cpu().numpy()


@pytest.mark.parametrize('M,N,K', [
    (1, 1, 1),          # one element, one partial K chunk
    (129, 65, 33),      # ragged in every dimension: two M tiles, two N tiles, two K chunks
    (300, 200, 1000),   # several tiles and K chunks
    (64, 64, 5000),     # one tile: K split across CTAs, FP64 split-K reduction
    (1000, 1000, 64),   # grid of 8 x 16 tiles, short K
])
@pytest.mark.parametrize('prec', sorted(FORMS))
def test_gemm_forms(M, N, K, prec):
    X = inputs.random_matrix(M, K, 11)
    Y = inputs.random_matrix(K, N, 12)
    O = _gemm(X, Y, prec)
    ref = X @ Y
    bound = np.abs(X) @ np.abs(Y)
    c, rel = FORMS[prec]
    assert np.all(np.isfinite(O))
    assert np.all(np.abs(O - ref) <= c * bound + 1e-300), np.max(np.abs(O - ref) / bound)
    assert np.linalg.norm(O - ref) <= rel * np.linalg.norm(ref)


@pytest.mark.parametrize('prec', [sctm.SCTM_PREC_FP64, sctm.SCTM_PREC_F64EMU])
def test_gemm_long_k_fp64_accurate_forms(prec):
    """K = 20000 (over a hundred K blocks of the emulation accumulated in one output): the
    FP64-accurate forms keep their K-independent elementwise bound (the FP32-accumulating forms'
    error grows with K and is covered at the sizes above)."""
    M, N, K = 130, 70, 20000
    X = inputs.random_matrix(M, K, 13)
    Y = inputs.random_matrix(K, N, 14)
    O = _gemm(X, Y, prec)
    ref = X @ Y
    bound = np.abs(X) @ np.abs(Y)
    c, rel = FORMS[prec]
    assert np.all(np.abs(O - ref) <= c * bound), np.max(np.abs(O - ref) / bound)
    assert np.linalg.norm(O - ref) <= rel * np.linalg.norm(ref)


def test_split_products_are_used():
    """The hi/lo forms must be far more accurate than the plain ones (the lo terms are added)."""
    X = inputs.random_matrix(256, 512, 21)
    Y = inputs.random_matrix(512, 192, 22)
    ref = X @ Y
    err = {p: np.linalg.norm(_gemm(X, Y, p) - ref) / np.linalg.norm(ref) for p in FORMS}
    assert err[sctm.SCTM_PREC_TF32X3] < err[sctm.SCTM_PREC_TF32] / 100
    assert err[sctm.SCTM_PREC_BF16X3] < err[sctm.SCTM_PREC_BF16] / 50
    assert err[sctm.SCTM_PREC_TF32] < err[sctm.SCTM_PREC_BF16]
    assert err[sctm.SCTM_PREC_FP64] < 1e-14
    assert err[sctm.SCTM_PREC_F64EMU] < 1e-14


def test_gemm_rejects_bad_arguments():
    X = torch.zeros(4, 4, dtype=torch.float64, device='cuda')
    h = np.zeros((4, 4))
    assert sctm.sctm_gemm(X, X, X, 4, 4, 4, 7, None) == sctm.SCTM_EINVAL
    assert sctm.sctm_gemm(X, X, X, 0, 4, 4, 0, None) == sctm.SCTM_EINVAL
    assert sctm.sctm_gemm(h, X, X, 4, 4, 4, 0, None) == sctm.SCTM_EINVAL


def _ctx(A, T, chi, prec):
    st, O = sctm.sctm_ising_pepo(T)
    return sctm.SplitCTMRG(A, O, chi, T, precision=prec)


@pytest.mark.parametrize('prec', [sctm.SCTM_PREC_TF32, sctm.SCTM_PREC_TF32X3,
                                  sctm.SCTM_PREC_BF16, sctm.SCTM_PREC_BF16X3])
def test_mixed_then_polish_reaches_fp64_fixed_point(prec):
    """Mixed-form iterations until the spectrum change stalls, then FP64 iterations to the
    tolerance: the converged f equals the oracle's converged f (contractive input).  A spectrum
    change below tol does not bound f's distance to the fixed point as tightly: the oracle's own f
    moves by 6.4e-11 (relative) between stopping at ||dS|| < 1e-11 and < 1e-13 on this input, and
    a trajectory that comes from the mixed form approaches along other directions, so the two
    converged values are compared at 1e-9.  The GPU run stops at 1e-11: its FP64 spectrum change
    levels off near 1e-12 on this input."""
    T, D, chi = 4.6, 2, 16
    A = inputs.perturbed_product_peps(D, 7)
    r = _ctx(A, T, chi, prec)
    try:
        st, it, ds = r.iterate(400, 1e-11)
        assert st == sctm.SCTM_OK and ds < 1e-11, (st, it, ds)
        f = r.free_energy()
    finally:
        r.close()
    ref = sc.evaluate(A, ising.ising_pepo(1 / T), ising.identity_pepo(), T, chi, 400, 1e-13)
    assert abs(f - ref['f']) <= 1e-9 * abs(ref['f']), (f, ref['f'])


# pseudo-inverse cutoff floors of the mixed forms (Engine::cutoff_floor)
FLOORS = {sctm.SCTM_PREC_TF32: 1e-3, sctm.SCTM_PREC_TF32X3: 1e-4, sctm.SCTM_PREC_BF16: 1e-2,
          sctm.SCTM_PREC_BF16X3: 1e-3}


@pytest.mark.parametrize('prec,tol', [(sctm.SCTM_PREC_TF32X3, 2e-4), (sctm.SCTM_PREC_BF16X3, 2e-5),
                                      (sctm.SCTM_PREC_TF32, 2e-4), (sctm.SCTM_PREC_BF16, 3e-3)])
def test_mixed_moves_against_fp64(prec, tol):
    """Three iterations of moves (left, right, up, down) in the mixed form against the same moves
    in FP64 with the same pseudo-inverse cutoff (the form's floor): ln kappa of both networks
    agrees to the form's error (tolerances 10x the largest difference measured on this input:
    2.1e-5 TF32 hi/lo, 1.1e-6 BF16 hi/lo, 2.3e-5 TF32, 3.1e-4 BF16), and not exactly (the
    tensor-core kernel ran)."""
    T, D, chi = 4.6, 2, 16
    A = inputs.perturbed_product_peps(D, 7)
    st, O = sctm.sctm_ising_pepo(T)
    rm = sctm.SplitCTMRG(A, O, chi, T, precision=prec)
    rf = sctm.SplitCTMRG(A, O, chi, T, cutoff=FLOORS[prec])
    try:
        for net in (sctm.SCTM_NET_NUM, sctm.SCTM_NET_DEN):
            for _ in range(3):
                for d in range(4):
                    assert sctm.sctm_move(rm.ctx, net, d) == sctm.SCTM_OK
                    assert sctm.sctm_move(rf.ctx, net, d) == sctm.SCTM_OK
                a = sctm.sctm_local_values(rm.ctx, net)[1][4]
                b = sctm.sctm_local_values(rf.ctx, net)[1][4]
                assert 0.0 < abs(a - b) <= tol * abs(b), (net, a, b)
    finally:
        rm.close()
        rf.close()


@pytest.mark.parametrize('prec', [sctm.SCTM_PREC_TF32X3, sctm.SCTM_PREC_F64EMU])
def test_mixed_full_size_moves(prec):
    """D=4, chi=64: the projector matrices (~1e-35 for this normalised N(0,1) PEPS) are below
    the FP32 range without the operands' power-of-two (row) scaling; two moves of each network
    complete with finite local values."""
    A = inputs.random_peps(4, 2)
    st, O = sctm.sctm_ising_pepo(4.5)
    r = sctm.SplitCTMRG(A, O, 64, 4.5, precision=prec, svd_mode=sctm.SCTM_SVD_PARTIAL)
    try:
        for net in (sctm.SCTM_NET_NUM, sctm.SCTM_NET_DEN):
            for d in (sctm.SCTM_MOVE_LEFT, sctm.SCTM_MOVE_RIGHT):
                assert sctm.sctm_move(r.ctx, net, d) == sctm.SCTM_OK
            st, out = sctm.sctm_local_values(r.ctx, net)
            assert np.all(np.isfinite(out[:4]))
    finally:
        r.close()


@pytest.mark.parametrize('D,chi,T,seed,eps,iters', [
    (2, 16, 4.6, 7, 0.3, 40),
    (3, 10, 4.4, 4, 0.1, 30),
])
def test_f64emu_parity_with_oracle(D, chi, T, seed, eps, iters):
    """SCTM_PREC_F64EMU at small sizes: no contraction here reaches the emulation's K >= 512 gate,
    so every contraction runs on the FP64 kernels and the FP64 tolerances (f 1e-10, g 1e-8
    against the oracle) must hold unchanged.  The emulation kernel itself is held to the same
    tolerances at full size in tests/test_gpu_configs.py, where it launches."""
    A = inputs.perturbed_product_peps(D, seed, eps=eps)
    r = _ctx(A, T, chi, sctm.SCTM_PREC_F64EMU)
    try:
        r.iterate(iters, 0.0)
        f, g = r.free_energy(), r.grad()
    finally:
        r.close()
    ref = sc.evaluate(A, ising.ising_pepo(1 / T), ising.identity_pepo(), T, chi, iters)
    assert abs(f - ref['f']) <= 1e-10 * abs(ref['f']), (f, ref['f'])
    assert np.linalg.norm(g - ref['g']) <= 1e-8 * np.linalg.norm(ref['g'])


@pytest.mark.parametrize('prec', [sctm.SCTM_PREC_TF32X3, sctm.SCTM_PREC_F64EMU])
def test_bounded_wait_timeout_is_reported(prec, monkeypatch):
    """Failure detection without a fault: with the test switch SCTM_TEST_FIRST_WAIT_ZERO=1 the
    first mbarrier wait of every tensor-core CTA gives up at once; the kernel drains its copies and
    MMAs with the normal bounded waits, frees its tensor memory, sets the error flag and returns,
    so sctm_gemm reports SCTM_ETIMEOUT.  The next call, without the switch, succeeds and is
    correct: the context is intact."""
    X = inputs.random_matrix(300, 200, 31)
    Y = inputs.random_matrix(200, 130, 32)
    dX, dY = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    dO = torch.zeros((300, 130), dtype=torch.float64, device='cuda')
    s = torch.cuda.current_stream().cuda_stream
    monkeypatch.setenv('SCTM_TEST_FIRST_WAIT_ZERO', '1')
    assert sctm.sctm_gemm(dX, dY, dO, 300, 130, 200, prec, s) == sctm.SCTM_ETIMEOUT
    monkeypatch.delenv('SCTM_TEST_FIRST_WAIT_ZERO')
    assert sctm.sctm_gemm(dX, dY, dO, 300, 130, 200, prec, s) == sctm.SCTM_OK
    c, rel = FORMS[prec]
    O = dO.cpu().numpy()
    assert np.all(np.abs(O - X @ Y) <= c * (np.abs(X) @ np.abs(Y)) + 1e-300)
