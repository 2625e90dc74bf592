"""GPU: the partial SVD (Sec. III's iterative solver for the largest chi singular triplets) against
the FP64 oracle, whose projectors come from a full SVD.

The first solve of every projector after a cold start is a full SVD (SCTM_SVD_PARTIAL) or two
subspace steps from a pseudo-random subspace (SCTM_SVD_PARTIAL_RANDOM); later solves are one
warm-started subspace-iteration step, whose subspace error decays geometrically with the
iterations.  At a fixed point the two methods have the same projectors, so converged values
agree to the convergence level; after a fixed number of iterations from the cold start they agree
to the decayed subspace error of the first warm solves (f to 1e-10, g to 1e-5 on the contractive
inputs below, measured 3e-11 and 1e-6 at worst in both modes)."""
import numpy as np
import pytest

from oracle import ising, split_ctmrg as sc
from paper_2506_19339_gb300 import build, inputs, sctm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module', autouse=True)
def lib():
    build.build()
    return sctm.load()


def _ctx(A, T, chi, mode=sctm.SCTM_SVD_PARTIAL):
    st, O = sctm.sctm_ising_pepo(T)
    return sctm.SplitCTMRG(A, O, chi, T, svd_mode=mode)


def _oracle(A, T, chi, iters, tol=None):
    return sc.evaluate(A, ising.ising_pepo(1.0 / T), ising.identity_pepo(), T, chi, iters, tol)


MODES = [sctm.SCTM_SVD_PARTIAL, sctm.SCTM_SVD_PARTIAL_RANDOM]


@pytest.mark.parametrize('mode', MODES)
@pytest.mark.parametrize('D,chi,T,seed,eps,iters', [
    (2, 16, 4.6, 7, 0.3, 40),
    (3, 10, 4.4, 4, 0.1, 30),
    (2, 7, 4.4, 3, 0.3, 30),
])
def test_partial_svd_parity_fixed_iterations(D, chi, T, seed, eps, iters, mode):
    A = inputs.perturbed_product_peps(D, seed, eps=eps)
    r = _ctx(A, T, chi, mode)
    try:
        r.iterate(iters, 0.0)
        f, g = r.free_energy(), r.grad()
    finally:
        r.close()
    ref = _oracle(A, T, chi, iters)
    assert abs(f - ref['f']) <= 1e-10 * abs(ref['f']), (f, ref['f'])
    assert np.linalg.norm(g - ref['g']) <= 1e-5 * np.linalg.norm(ref['g'])


@pytest.mark.parametrize('mode', MODES)
def test_partial_svd_converged_fixed_point(mode):
    """Converged f against the oracle's converged f (1e-9: the oracle's own f moves by 6.4e-11
    between stopping at 1e-11 and 1e-13 on this input) and converged g (1e-8), and the partial
    run's fixed point is a fixed point of the full-SVD iteration: ten full-SVD iterations from it
    move f by less than 1e-10."""
    T, chi = 4.6, 16
    A = inputs.perturbed_product_peps(2, 7)
    rp, rq = _ctx(A, T, chi, mode), _ctx(A, T, chi, sctm.SCTM_SVD_QR)
    try:
        st, it, ds = rp.iterate(400, 1e-11)
        assert st == sctm.SCTM_OK, (st, it, ds)
        f = rp.free_energy()
        g = rp.grad()
        for net in (sctm.SCTM_NET_NUM, sctm.SCTM_NET_DEN):
            st, buf = sctm.sctm_env_export(rp.ctx, net)
            assert sctm.sctm_env_import(rq.ctx, net, buf) == sctm.SCTM_OK
        rq.iterate(10, 0.0)
        fq = rq.free_energy()
    finally:
        rp.close()
        rq.close()
    ref = _oracle(A, T, chi, 400, 1e-13)
    assert abs(f - ref['f']) <= 1e-9 * abs(ref['f']), (f, ref['f'])
    # the environment gradient at the partial SVD's fixed point is the full SVD's
    assert np.linalg.norm(g - ref['g']) <= 1e-8 * np.linalg.norm(ref['g'])
    assert abs(fq - f) <= 1e-10 * abs(f), (fq, f)


@pytest.mark.parametrize('mode', MODES)
def test_partial_svd_full_size_runs(mode):
    """D=4, chi=64 (subspace 80 of 512): a cold and three warm iterations complete without an
    error status, and the spectrum change is finite."""
    A = inputs.random_peps(4, 2)
    r = _ctx(A, 4.5, 64, mode)
    try:
        st, it, ds = r.iterate(4, 0.0)
        assert st in (sctm.SCTM_OK, sctm.SCTM_ENOCONV) and it == 4 and np.isfinite(ds)
    finally:
        r.close()


def test_partial_svd_large_subspace_stays_on_full_svd():
    """chi = 161 at D = 1: every subspace (161 columns at the alpha cut, whose dimension is 161;
    169 at the kappa and iota cuts) is above the 160-column limit of the one-CTA kernels, so every
    projector keeps the full SVD and the result equals the full-SVD mode's bit for bit."""
    A = inputs.product_plus_peps(1)
    fs = []
    for mode in (sctm.SCTM_SVD_QR, sctm.SCTM_SVD_PARTIAL):
        st, O = sctm.sctm_ising_pepo(10.0)
        r = sctm.SplitCTMRG(A, O, 161, 10.0, svd_mode=mode)
        try:
            r.iterate(2, 0.0)
            fs.append(r.free_energy())
        finally:
            r.close()
    assert fs[0] == fs[1]


def test_partial_svd_large_subspace_matches_full_svd():
    """chi = 100 at D = 2: subspaces of 125 columns, above the 112 that fit the one-CTA kernels'
    shared memory, so one k x k matrix of the Cholesky-QR and Jacobi kernels lives in global
    scratch.  Twenty iterations from the cold start on a contractive input agree with the full
    SVD path (measured 1.1e-14 in f, 7e-9 in g)."""
    T, D, chi = 4.6, 2, 100
    A = inputs.perturbed_product_peps(D, 7)
    res = {}
    for mode in (sctm.SCTM_SVD_QR, sctm.SCTM_SVD_PARTIAL_RANDOM):
        r = _ctx(A, T, chi, mode)
        try:
            r.iterate(20, 0.0)
            res[mode] = (r.free_energy(), r.grad())
        finally:
            r.close()
    f0, g0 = res[sctm.SCTM_SVD_QR]
    f1, g1 = res[sctm.SCTM_SVD_PARTIAL_RANDOM]
    assert abs(f1 - f0) <= 1e-10 * abs(f0), (f1, f0)
    assert np.linalg.norm(g1 - g0) <= 1e-6 * np.linalg.norm(g0)
