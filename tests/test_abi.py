"""The C ABI without a GPU: the library builds for sm_103a, loads, exports every entry point that
include/sctm.h declares, and its host-only entry points behave as documented."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import ising
from paper_2506_19339_gb300 import build, sctm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope='module')
def lib():
    build.build()
    return sctm.load()


def declared_functions():
    src = open(os.path.join(ROOT, 'include', 'sctm.h')).read()
    src = re.sub(r'/\*.*?\*/', '', src, flags=re.S)
    return sorted(set(re.findall(r'\b(sctm_[a-z_]+)\s*\(', src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ('sctm_create', 'sctm_iterate', 'sctm_free_energy', 'sctm_grad',
                     'sctm_destroy', 'sctm_ising_pepo', 'sctm_last_error'):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_ising_pepo_matches_oracle(lib):
    """The library's closed-form sqrt(W) (Sec. IV) against the oracle's eigendecomposition."""
    for T in (4.4, 4.5115, 4.6, 10.0):
        st, O = sctm.sctm_ising_pepo(T)
        assert st == sctm.SCTM_OK
        assert np.allclose(O, ising.ising_pepo(1.0 / T), rtol=1e-14, atol=1e-15)
    st, O = sctm.sctm_ising_pepo(float('inf'))
    assert st == sctm.SCTM_OK and np.allclose(O, 0.25, atol=1e-15)
    assert sctm.sctm_ising_pepo(0.0)[0] == sctm.SCTM_EINVAL
    assert sctm.sctm_ising_pepo(-4.0)[0] == sctm.SCTM_EINVAL


def test_host_side_error_paths(lib):
    st, o = sctm.sctm_default_opts()
    assert st == sctm.SCTM_OK and o.D == 2 and o.p == 2 and o.d == 2 and o.svd_cutoff == 1e-12
    assert sctm.sctm_destroy(None) == sctm.SCTM_OK
    assert sctm.sctm_last_error(None) != ''
    assert sctm.sctm_env_size(None, 0) == 0
    A = np.zeros((2, 2, 2, 2, 2))
    O = np.zeros((2, 2, 2, 2, 2, 2))
    for chi in (0, -3, 5000):
        st, ctx = sctm.sctm_create(A, O, chi, o)
        assert st == sctm.SCTM_EINVAL and not ctx.value
    bad = sctm.SctmOpts.from_buffer_copy(o)
    bad.batch = 2
    assert sctm.sctm_create(A, O, 4, bad)[0] == sctm.SCTM_EINVAL
    assert o.jacobi == sctm.SCTM_JACOBI_CTA
    bad = sctm.SctmOpts.from_buffer_copy(o)
    bad.jacobi = 2
    assert sctm.sctm_create(A, O, 4, bad)[0] == sctm.SCTM_EINVAL
    assert ctypes.sizeof(sctm.SctmOpts) == 80  # the header's struct: 13 fields + jacobi, padded
    assert lib.sctm_iterate(None, 1, 0.0, None, None) == sctm.SCTM_EINVAL
    assert lib.sctm_free_energy(None, None) == sctm.SCTM_EINVAL


@pytest.mark.parametrize('D,d,chi,svd', [(1, 2, 1, 0), (2, 2, 5, 0), (3, 2, 10, 0), (4, 2, 64, 0),
                                         (2, 3, 7, 0), (2, 2, 5, 2), (4, 2, 64, 2), (3, 2, 100, 2),
                                         (3, 2, 36, 3), (5, 2, 100, 3)])
def test_plans_build_without_gpu(lib, D, d, chi, svd):
    """SCTM_DRYRUN=1 builds every plan (four moves, convergence, local contractions) of both
    networks with placeholder pointers: every contraction's labels, dimensions and ranks are
    checked on the CPU, for the full (svd 0) and the partial (svd 2) SVD plans; chi = 100 has
    subspaces above the one-CTA limit, which stay on the full SVD.  SCTM_DRYRUN_ADJOINT=1 also
    builds the reverse-mode (adjoint) plans from the tapes, checking every backward contraction."""
    import subprocess
    import sys
    code = ('import numpy as np\n'
            'from paper_2506_19339_gb300 import sctm\n'
            'st, o = sctm.sctm_default_opts()\n'
            'o.D, o.d, o.svd_mode = %d, %d, %d\n'
            'A = np.zeros((2,) + (%d,) * 4); O = np.zeros((2, 2) + (%d,) * 4)\n'
            'st, ctx = sctm.sctm_create(A, O, %d, o)\n'
            'print(st)\n') % (D, d, svd, D, d, chi)
    env = dict(os.environ, SCTM_DRYRUN='1', SCTM_DRYRUN_ADJOINT='1')
    out = subprocess.run([sys.executable, '-c', code], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == '0', out.stdout + out.stderr


def test_binding_constants_match_header():
    """The ctypes binding's enum values are the header's (status codes, precisions, SVD modes,
    networks, moves, profiled kernels)."""
    import re
    text = open(os.path.join(ROOT, 'include', 'sctm.h')).read()
    values = {}
    for name, val in re.findall(r'\b(SCTM_[A-Z0-9_]+)\s*=\s*(\d+)', text):
        values[name] = int(val)
    assert len(values) > 20
    for name, val in values.items():
        if hasattr(sctm, name):
            assert getattr(sctm, name) == val, name
    for name in ('SCTM_PREC_F64EMU', 'SCTM_SVD_PARTIAL_RANDOM', 'SCTM_KERNEL_F64EMU', 'SCTM_ETIMEOUT'):
        assert getattr(sctm, name) == values[name], name


@pytest.mark.parametrize('D,chi,svd', [(2, 6, 0), (4, 16, 3), (3, 9, 2)])
def test_reduced_plans_build_without_gpu(lib, D, chi, svd):
    """SCTM_DRYRUN=1 with the reduced method (Sec. II, Fig. 3): the fused-tensor plan, the four
    moves, the spectrum and the local contractions build with every label and dimension checked."""
    import subprocess
    import sys
    code = ('import numpy as np\n'
            'from paper_2506_19339_gb300 import sctm\n'
            'st, o = sctm.sctm_default_opts()\n'
            'o.D, o.d, o.svd_mode, o.method = %d, 2, %d, sctm.SCTM_METHOD_REDUCED\n'
            'A = np.zeros((2,) + (%d,) * 4); O = np.zeros((2, 2) + (2,) * 4)\n'
            'st, ctx = sctm.sctm_create(A, O, %d, o)\n'
            'print(st)\n') % (D, svd, D, chi)
    env = dict(os.environ, SCTM_DRYRUN='1')
    out = subprocess.run([sys.executable, '-c', code], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == '0', out.stdout + out.stderr


@pytest.mark.parametrize('D,chi,svd,p4', [(2, 6, 0, 0), (4, 64, 3, 0), (3, 36, 2, 1), (5, 100, 3, 1),
                                          (4, 64, 3, 1)])
def test_symmetric_plans_build_without_gpu(lib, D, chi, svd, p4):
    """SCTM_DRYRUN=1 with the D2-symmetric split method (Sec. III.B): the one-update iteration
    (this boundary's stage-1 projectors, the opposite boundary's as their mirrored views, the
    full or half projector 4, T4, and both corners from their enlarged forms), the spectrum and
    the local contractions over the strided views of the derived environment slots build with
    every label and dimension checked."""
    import subprocess
    import sys
    code = ('import numpy as np\n'
            'from paper_2506_19339_gb300 import sctm\n'
            'st, o = sctm.sctm_default_opts()\n'
            'o.D, o.d, o.svd_mode, o.method = %d, 2, %d, sctm.SCTM_METHOD_SPLIT_D2\n'
            'o.p4_mode = %d\n'
            'A = np.zeros((2,) + (%d,) * 4); O = np.zeros((2, 2) + (2,) * 4)\n'
            'st, ctx = sctm.sctm_create(A, O, %d, o)\n'
            'print(st)\n') % (D, svd, p4, D, chi)
    env = dict(os.environ, SCTM_DRYRUN='1')
    out = subprocess.run([sys.executable, '-c', code], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == '0', out.stdout + out.stderr


@pytest.mark.parametrize('D,chi,svd', [(2, 6, 0), (3, 10, 2), (4, 64, 3)])
def test_directional_half_p4_plans_build_without_gpu(lib, D, chi, svd):
    """SCTM_DRYRUN=1 with the directional split method and the half projector 4 (Appendix,
    projector 4(b)): each move's plan adds the up and down moves' projector-1 pipelines (their
    one-column alpha patches in their own frames) and the 2x1-cell patch renormalised by them;
    every label and dimension of all four moves is checked."""
    import subprocess
    import sys
    code = ('import numpy as np\n'
            'from paper_2506_19339_gb300 import sctm\n'
            'st, o = sctm.sctm_default_opts()\n'
            'o.D, o.d, o.svd_mode, o.method = %d, 2, %d, sctm.SCTM_METHOD_SPLIT\n'
            'o.p4_mode = sctm.SCTM_P4_HALF\n'
            'A = np.zeros((2,) + (%d,) * 4); O = np.zeros((2, 2) + (2,) * 4)\n'
            'st, ctx = sctm.sctm_create(A, O, %d, o)\n'
            'print(st)\n') % (D, svd, D, chi)
    env = dict(os.environ, SCTM_DRYRUN='1')
    out = subprocess.run([sys.executable, '-c', code], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == '0', out.stdout + out.stderr


def test_symmetric_method_option_checks(lib):
    """The D2-symmetric method has the environment gradient only: the adjoint is rejected on
    entry, before any device work."""
    A = np.zeros((2, 2, 2, 2, 2))
    O = np.zeros((2, 2, 2, 2, 2, 2))
    st, o = sctm.sctm_default_opts()
    o.method = sctm.SCTM_METHOD_SPLIT_D2
    o.grad_mode = sctm.SCTM_GRAD_ADJOINT
    assert sctm.sctm_create(A, O, 4, o)[0] == sctm.SCTM_EINVAL
    o.grad_mode = sctm.SCTM_GRAD_ENV
    o.method = 3
    assert sctm.sctm_create(A, O, 4, o)[0] == sctm.SCTM_EINVAL
    o.method = sctm.SCTM_METHOD_REDUCED        # the half projector 4 is a split-method patch
    o.p4_mode = sctm.SCTM_P4_HALF
    assert sctm.sctm_create(A, O, 4, o)[0] == sctm.SCTM_EINVAL
    o.method = sctm.SCTM_METHOD_SPLIT          # and has the environment gradient only
    o.grad_mode = sctm.SCTM_GRAD_ADJOINT
    assert sctm.sctm_create(A, O, 4, o)[0] == sctm.SCTM_EINVAL
    o.grad_mode = sctm.SCTM_GRAD_ENV
    o.method = sctm.SCTM_METHOD_SPLIT_D2
    o.p4_mode = 2
    assert sctm.sctm_create(A, O, 4, o)[0] == sctm.SCTM_EINVAL


def test_reduced_method_option_checks(lib):
    """The reduced method is FP64 with the environment gradient only: other combinations are
    rejected on entry."""
    A = np.zeros((2, 2, 2, 2, 2))
    O = np.zeros((2, 2, 2, 2, 2, 2))
    st, o = sctm.sctm_default_opts()
    o.method = sctm.SCTM_METHOD_REDUCED
    o.precision = sctm.SCTM_PREC_TF32
    assert sctm.sctm_create(A, O, 4, o)[0] == sctm.SCTM_EINVAL
    o.precision = sctm.SCTM_PREC_FP64
    o.grad_mode = sctm.SCTM_GRAD_ADJOINT
    assert sctm.sctm_create(A, O, 4, o)[0] == sctm.SCTM_EINVAL
    o.grad_mode = sctm.SCTM_GRAD_ENV
    o.method = 7
    assert sctm.sctm_create(A, O, 4, o)[0] == sctm.SCTM_EINVAL
