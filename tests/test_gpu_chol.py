"""GPU: the column-scaled, shifted Cholesky-QR pass that orthonormalises the partial SVD's subspace
bases (Sec. III: the leading singular triplets of the projector matrix by an iterative solver), in
its two kernels -- one CTA, and the rows of the Gram matrix split over a cluster of 8 CTAs --
called through the C ABI (sctm_chol_orth).

The cluster kernel applies each pivot's rank-one update to every element in pivot order as one
fused multiply-add, and the same back substitution for the inverse factor, so its result must be
the one-CTA kernel's bit for bit.  Inputs: Gram matrices of n x k bases of the kinds the subspace
iteration produces -- Gaussian, graded by singular values down to 1e-12 (a warm subspace
Y ~ U S), with nearly dependent tail columns, with a zero column -- with and without the shift
11 (n k + k (k + 1)) 2^-53 of the engine's first two passes.  For a well-conditioned basis the
unshifted pass must also orthonormalise: (Y T)^T (Y T) = I to 1e-12."""
import numpy as np
import pytest

from paper_2506_19339_gb300 import build, sctm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip('torch')
N = 512


@pytest.fixture(scope='module', autouse=True)
def lib():
    build.build()
    return sctm.load()


def _basis(kind, k, seed):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((N, k))
    if kind == 'gaussian':
        return Y
    if kind == 'graded':
        q = np.linalg.qr(Y)[0]
        return q * np.logspace(0, -12, k)
    if kind == 'dependent_tail':
        q = np.linalg.qr(Y)[0]
        Y = q * np.logspace(0, -3, k)
        Y[:, -4:] = Y[:, :4] @ rng.standard_normal((4, 4)) + 1e-14 * rng.standard_normal((N, 4))
        return Y
    if kind == 'zero_column':
        Y[:, k // 3] = 0.0
        return Y
    raise ValueError(kind)


def _pass(G, k, shift, variant):
    dev = torch.device('cuda', 0)
    Gd = torch.from_numpy(G.ravel(order='F').copy()).to(dev)
    T = torch.full((k * k,), np.nan, dtype=torch.float64, device=dev)
    st = sctm.sctm_chol_orth(Gd, k, shift, T, variant)
    return st, T.cpu().numpy().reshape(k, k, order='F')


@pytest.mark.parametrize('k', [32, 33, 45, 64, 80, 100, 125, 128])
@pytest.mark.parametrize('kind', ['gaussian', 'graded', 'dependent_tail', 'zero_column'])
@pytest.mark.parametrize('shifted', [False, True])
def test_cluster_kernel_is_bit_identical(k, kind, shifted):
    Y = _basis(kind, k, seed=k)
    G = Y.T @ Y
    G = 0.5 * (G + G.T)  # symmetric bit for bit, like the engine's Gram contraction
    shift = 11.0 * (N * k + k * (k + 1)) * 2.0 ** -53 if shifted else 0.0
    st0, T0 = _pass(G, k, shift, sctm.SCTM_CHOL_CTA)
    st1, T1 = _pass(G, k, shift, sctm.SCTM_CHOL_CLUSTER)
    assert st0 == sctm.SCTM_OK and st1 == sctm.SCTM_OK
    assert np.all(np.isfinite(T1))
    assert np.array_equal(T0, T1), np.max(np.abs(T0 - T1))
    assert np.all(np.tril(T1, -1) == 0.0)
    if kind == 'gaussian' and not shifted:
        Q = Y @ T1
        assert np.linalg.norm(Q.T @ Q - np.eye(k)) <= 1e-12


def test_orders_outside_the_cluster_kernel_are_rejected():
    dev = torch.device('cuda', 0)
    buf = torch.zeros(200 * 200, dtype=torch.float64, device=dev)
    for k in (31, 129):
        assert sctm.sctm_chol_orth(buf, k, 0.0, buf, sctm.SCTM_CHOL_CLUSTER) == sctm.SCTM_EINVAL
    assert sctm.sctm_chol_orth(buf, 161, 0.0, buf, sctm.SCTM_CHOL_CTA) == sctm.SCTM_EINVAL
    assert sctm.sctm_chol_orth(buf, 40, -1.0, buf, sctm.SCTM_CHOL_CTA) == sctm.SCTM_EINVAL
    assert sctm.sctm_chol_orth(buf, 40, 0.0, buf, 2) == sctm.SCTM_EINVAL
