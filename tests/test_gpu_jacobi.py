"""GPU: the Jacobi SVD that closes each warm step of the partial SVD (Sec. III: the leading
singular triplets of the projector matrix by an iterative solver), in its two kernels -- one CTA,
and the rows of the iterated matrices split over a cluster of 8 CTAs -- called through the C ABI
(sctm_jacobi_svd) on k x k matrices of the kinds the subspace iteration produces: dense Gaussian
(cold solves), graded to 1e-12 (the Rayleigh-Ritz matrix of a converged subspace), nearly diagonal
(warm solves near the fixed point), exact multiplets (the D2-symmetric scheme's spectra), zero
columns (rank-deficient subspaces) and the zero matrix.

Each result is checked against LAPACK's singular values and by its own identities (B = U S W^T,
W^T W = I, U^T U = I on the columns with S above 1e-6 S_0), and the two kernels against each
other.  Bounds: a k-term FP64 dot product rounds at k 2^-53 ~ 1e-14 of the operands' norms, so
values and reconstruction are held to 1e-13 of |B|.  U's columns of a multiplet are determined
only up to a rotation inside it, so they are held to orthogonality alone, and to a looser bound:
both kernels stop after the FP64 sweep that started below 1e-6, which leaves rounding level where
Jacobi converges quadratically (distinct values) but not inside an exact multiplet, where
convergence is linear (measured with the one-CTA kernel at k = 80, four-fold multiplets:
||U^T U - I||_F = 3.8e-8)."""
import numpy as np
import pytest

from paper_2506_19339_gb300 import build, sctm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip('torch')


@pytest.fixture(scope='module', autouse=True)
def lib():
    build.build()
    return sctm.load()


def _matrix(kind, k, seed):
    rng = np.random.default_rng(seed)
    if kind == 'zero':
        return np.zeros((k, k))
    if kind == 'gaussian':
        return rng.standard_normal((k, k))
    q1 = np.linalg.qr(rng.standard_normal((k, k)))[0]
    q2 = np.linalg.qr(rng.standard_normal((k, k)))[0]
    s = np.logspace(0, -12, k)
    if kind == 'graded':
        return (q1 * s) @ q2.T
    if kind == 'near_diagonal':
        return np.diag(s) + 1e-7 * np.triu(rng.standard_normal((k, k)), 1) * s[None, :]
    if kind == 'multiplets':
        m = np.repeat(np.logspace(0, -3, (k + 3) // 4), 4)[:k]
        return (q1 * m) @ q2.T
    if kind == 'zero_columns':
        b = (q1 * s) @ q2.T
        b[:, [1, k // 2, k - 1]] = 0.0
        return b
    raise ValueError(kind)


def _svd(B, variant):
    k = B.shape[0]
    dev = torch.device('cuda', 0)
    Bd = torch.from_numpy(np.asfortranarray(B).ravel(order='F').copy()).to(dev)
    S = torch.full((k,), -1.0, dtype=torch.float64, device=dev)
    U = torch.full((k * k,), np.nan, dtype=torch.float64, device=dev)
    W = torch.full((k * k,), np.nan, dtype=torch.float64, device=dev)
    st = sctm.sctm_jacobi_svd(Bd, k, S, U, W, variant)
    return (st, S.cpu().numpy(), U.cpu().numpy().reshape(k, k, order='F'),
            W.cpu().numpy().reshape(k, k, order='F'))


def _check(B, S, U, W, kind):
    k = B.shape[0]
    nb = max(np.linalg.norm(B, 2), 1e-300)
    ref = np.linalg.svd(B, compute_uv=False)
    assert np.all(np.diff(S) <= 0.0)
    assert np.max(np.abs(S - ref)) <= 1e-13 * nb
    assert np.linalg.norm(B - (U * S) @ W.T) <= 1e-13 * max(np.linalg.norm(B), 1e-300) + 1e-300
    assert np.linalg.norm(W.T @ W - np.eye(k)) <= 1e-12
    big = S > 1e-6 * S[0] if S[0] > 0 else np.zeros(k, bool)
    Ub = U[:, big]
    tol = 1e-6 if kind == 'multiplets' else 1e-10
    assert np.linalg.norm(Ub.T @ Ub - np.eye(Ub.shape[1])) <= tol


CASES = [('gaussian', 80), ('gaussian', 79), ('gaussian', 34), ('gaussian', 31), ('gaussian', 125),
         ('gaussian', 128), ('gaussian', 64), ('graded', 80), ('near_diagonal', 80),
         ('multiplets', 80), ('multiplets', 46), ('zero_columns', 80), ('zero', 80)]


@pytest.mark.parametrize('kind,k', CASES)
def test_both_kernels_against_lapack_and_each_other(kind, k):
    B = _matrix(kind, k, seed=k)
    st0, S0, U0, W0 = _svd(B, sctm.SCTM_JACOBI_CTA)
    st1, S1, U1, W1 = _svd(B, sctm.SCTM_JACOBI_CLUSTER)
    assert st0 == sctm.SCTM_OK and st1 == sctm.SCTM_OK, (st0, st1)
    _check(B, S0, U0, W0, kind)
    _check(B, S1, U1, W1, kind)
    nb = max(np.linalg.norm(B, 2), 1e-300)
    assert np.max(np.abs(S0 - S1)) <= 1e-13 * nb
    if kind in ('gaussian', 'graded', 'near_diagonal'):
        # distinct singular values: the same singular pairs up to sign, where the gap to the
        # neighbours bounds the angle (the pairs of the graded tail below 1e-6 S_0 are left out)
        sel = S0 > 1e-6 * S0[0]
        d = np.abs(np.sum(W0[:, sel] * W1[:, sel], axis=0))
        assert np.all(d >= 1.0 - 1e-8), d.min()


def test_repeated_calls_are_deterministic():
    """The cluster kernel's sums are taken in a fixed order: the same input gives the same bits."""
    B = _matrix('gaussian', 80, seed=5)
    a = _svd(B, sctm.SCTM_JACOBI_CLUSTER)
    b = _svd(B, sctm.SCTM_JACOBI_CLUSTER)
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(x, y)


def test_orders_outside_the_cluster_kernel_are_rejected():
    dev = torch.device('cuda', 0)
    buf = torch.zeros(200 * 200, dtype=torch.float64, device=dev)
    for k in (29, 30, 129, 160):
        assert sctm.sctm_jacobi_svd(buf, k, buf, buf, buf, sctm.SCTM_JACOBI_CLUSTER) == sctm.SCTM_EINVAL
    assert sctm.sctm_jacobi_svd(buf, 161, buf, buf, buf, sctm.SCTM_JACOBI_CTA) == sctm.SCTM_EINVAL
    assert sctm.sctm_jacobi_svd(buf, 8, buf, buf, buf, 2) == sctm.SCTM_EINVAL
