"""GPU: the variational optimisation loop of Sec. IV.B (L-BFGS over the PEPS tensor, each
evaluation warm-started from the previous environment): f must decrease from a perturbed
product state, with the paper's environment gradient and with the fixed-point adjoint."""
import numpy as np
import pytest

from paper_2506_19339_gb300 import build, inputs, sctm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module', autouse=True)
def lib():
    build.build()
    return sctm.load()


@pytest.mark.parametrize('grad_mode', [sctm.SCTM_GRAD_ENV, sctm.SCTM_GRAD_ADJOINT])
def test_lbfgs_lowers_the_free_energy(grad_mode):
    from paper_2506_19339_gb300 import optimize
    T, D, chi = 4.6, 2, 6
    A0 = inputs.perturbed_product_peps(D, 7)
    A, hist = optimize.lbfgs_minimize(A0, T, chi, steps=4, grad_mode=grad_mode,
                                      svd_mode=sctm.SCTM_SVD_QR, tol=1e-11)
    fs = [h[0] for h in hist]
    print('L-BFGS (grad mode %d): f %s' % (grad_mode, ['%.10f' % f for f in fs]))
    assert np.all(np.isfinite(fs))
    assert min(fs) < fs[0] - 1e-6
    assert np.all(np.isfinite(A))
