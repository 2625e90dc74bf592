"""Thin Python binding of libsctm.so (include/sctm.h), argument marshalling only.

Every function has the name of the C entry point it calls and returns its sctm_status (plus the
outputs the C call writes).  All computation happens in the library's CUDA kernels; there is no
Python or CPU fallback: if the compiled library is missing, ``load()`` raises.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, 'libsctm.so')

SCTM_OK, SCTM_EINVAL, SCTM_ECUDA, SCTM_ECUSOLVER, SCTM_ENOMEM, SCTM_ENOCONV, SCTM_ENUMERIC, \
    SCTM_ETIMEOUT = range(8)
STATUS_NAMES = ['SCTM_OK', 'SCTM_EINVAL', 'SCTM_ECUDA', 'SCTM_ECUSOLVER', 'SCTM_ENOMEM',
                'SCTM_ENOCONV', 'SCTM_ENUMERIC', 'SCTM_ETIMEOUT']
SCTM_PREC_FP64, SCTM_PREC_TF32, SCTM_PREC_TF32X3, SCTM_PREC_BF16, SCTM_PREC_BF16X3, SCTM_PREC_F64EMU = range(6)
SCTM_GRAD_ENV, SCTM_GRAD_ADJOINT = 0, 1
SCTM_SVD_QR, SCTM_SVD_POLAR, SCTM_SVD_PARTIAL, SCTM_SVD_PARTIAL_RANDOM = 0, 1, 2, 3
SCTM_NET_NUM, SCTM_NET_DEN = 0, 1
SCTM_METHOD_SPLIT, SCTM_METHOD_REDUCED, SCTM_METHOD_SPLIT_D2 = 0, 1, 2
SCTM_P4_FULL, SCTM_P4_HALF = 0, 1
SCTM_JACOBI_CTA, SCTM_JACOBI_CLUSTER = 0, 1
SCTM_CHOL_CTA, SCTM_CHOL_CLUSTER = 0, 1
SCTM_MOVE_LEFT, SCTM_MOVE_RIGHT, SCTM_MOVE_UP, SCTM_MOVE_DOWN = range(4)


class SctmOpts(ctypes.Structure):
    _fields_ = [('T', ctypes.c_double), ('D', ctypes.c_int), ('p', ctypes.c_int),
                ('d', ctypes.c_int), ('precision', ctypes.c_int), ('grad_mode', ctypes.c_int),
                ('svd_cutoff', ctypes.c_double), ('init_seed', ctypes.c_ulonglong),
                ('batch', ctypes.c_int), ('cuda_stream', ctypes.c_void_p),
                ('svd_mode', ctypes.c_int), ('method', ctypes.c_int), ('p4_mode', ctypes.c_int),
                ('jacobi', ctypes.c_int)]


class SctmError(RuntimeError):
    def __init__(self, status, msg=''):
        super().__init__('%s: %s' % (STATUS_NAMES[status] if 0 <= status < 8 else status, msg))
        self.status = status


_lib = None


def load():
    """Load libsctm.so from the package directory (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError('libsctm.so not found at %s: build it first '
                          '(python -c "import __graft_entry__ as g; g.build()")' % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    D = ctypes.c_double
    I = ctypes.c_int
    S = ctypes.c_size_t
    sig = {
        'sctm_default_opts': (I, [ctypes.POINTER(SctmOpts)]),
        'sctm_create': (I, [P, P, I, ctypes.POINTER(SctmOpts), ctypes.POINTER(P)]),
        'sctm_set_peps': (I, [P, P, I]),
        'sctm_iterate': (I, [P, I, D, ctypes.POINTER(I), ctypes.POINTER(D)]),
        'sctm_free_energy': (I, [P, ctypes.POINTER(D)]),
        'sctm_grad': (I, [P, P]),
        'sctm_destroy': (I, [P]),
        'sctm_ising_pepo': (I, [D, P]),
        'sctm_last_error': (ctypes.c_char_p, [P]),
        'sctm_env_size': (S, [P, I]),
        'sctm_env_export': (I, [P, I, P, S]),
        'sctm_env_import': (I, [P, I, P, S]),
        'sctm_move': (I, [P, I, I]),
        'sctm_spectrum': (I, [P, I, P]),
        'sctm_local_values': (I, [P, I, P]),
        'sctm_gemm_noalloc': (I, [P, P, P, I, I, I, P]),
        'sctm_gemm': (I, [P, P, P, I, I, I, I, P]),
        'sctm_jacobi_svd': (I, [P, I, P, P, P, I, P]),
        'sctm_chol_orth': (I, [P, I, D, P, I, P]),
        'sctm_profile_kernel': (I, [P, I, P, P, P, P]),
        'sctm_iterate_batch': (I, [ctypes.POINTER(P), I, I, D, ctypes.POINTER(I),
                                   ctypes.POINTER(I), ctypes.POINTER(D)]),
        'sctm_device_bytes': (S, [P]),
        'sctm_set_grad_mode': (I, [P, I, D, I, D]),
        'sctm_autotune_info': (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I)]),
        'sctm_adjoint_info': (I, [P, ctypes.POINTER(I), ctypes.POINTER(D)]),
        'sctm_set_profiling': (I, [P, I]),
        'sctm_profile': (I, [P, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_longlong),
                             ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(D),
                             ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                             I]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(x):
    """Device pointer of a torch tensor, or host pointer of a float64 C-contiguous ndarray."""
    if hasattr(x, 'data_ptr'):
        if x.dtype.__str__() != 'torch.float64' or not x.is_contiguous():
            raise TypeError('expected a contiguous float64 tensor')
        return ctypes.c_void_p(x.data_ptr())
    if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags['C_CONTIGUOUS']):
        raise TypeError('expected a C-contiguous float64 ndarray')
    return x.ctypes.data_as(ctypes.c_void_p)


def sctm_default_opts():
    o = SctmOpts()
    st = load().sctm_default_opts(ctypes.byref(o))
    return st, o


def sctm_ising_pepo(T):
    out = np.zeros(64)
    st = load().sctm_ising_pepo(float(T), _ptr(out))
    return st, out.reshape(2, 2, 2, 2, 2, 2)


def sctm_create(peps, pepo, chi, opts):
    ctx = ctypes.c_void_p()
    st = load().sctm_create(_ptr(peps), _ptr(pepo), int(chi), ctypes.byref(opts), ctypes.byref(ctx))
    return st, ctx


def sctm_set_peps(ctx, peps, reset_env):
    return load().sctm_set_peps(ctx, _ptr(peps), int(reset_env))


def sctm_iterate(ctx, max_it, tol):
    it = ctypes.c_int(0)
    ds = ctypes.c_double(0.0)
    st = load().sctm_iterate(ctx, int(max_it), float(tol), ctypes.byref(it), ctypes.byref(ds))
    return st, it.value, ds.value


def sctm_free_energy(ctx):
    f = ctypes.c_double(0.0)
    st = load().sctm_free_energy(ctx, ctypes.byref(f))
    return st, f.value


def sctm_grad(ctx, g):
    """g: float64 ndarray (host) or torch tensor (device) of p*D^4 entries, written in place."""
    return load().sctm_grad(ctx, _ptr(g))


def sctm_destroy(ctx):
    return load().sctm_destroy(ctx)


def sctm_last_error(ctx):
    msg = load().sctm_last_error(ctx)
    return msg.decode() if msg else ''


def sctm_env_size(ctx, network):
    return int(load().sctm_env_size(ctx, int(network)))


def sctm_env_export(ctx, network):
    n = sctm_env_size(ctx, network)
    buf = np.zeros(max(n, 1))
    st = load().sctm_env_export(ctx, int(network), _ptr(buf), n)
    return st, buf[:n]


def sctm_env_import(ctx, network, buf):
    buf = np.ascontiguousarray(buf, dtype=np.float64)
    return load().sctm_env_import(ctx, int(network), _ptr(buf), buf.size)


def sctm_move(ctx, network, direction):
    return load().sctm_move(ctx, int(network), int(direction))


def sctm_spectrum(ctx, network, chi):
    S = np.zeros(chi)
    st = load().sctm_spectrum(ctx, int(network), _ptr(S))
    return st, S


def sctm_local_values(ctx, network):
    out = np.zeros(5)
    st = load().sctm_local_values(ctx, int(network), _ptr(out))
    return st, out


def sctm_gemm_noalloc(X, Y, O, M, N, K, stream=None):
    """O = X Y (row-major device tensors, FP64) without any device allocation in the library."""
    return load().sctm_gemm_noalloc(_ptr(X), _ptr(Y), _ptr(O), int(M), int(N), int(K),
                                    ctypes.c_void_p(stream))


def sctm_chol_orth(G, k, shift, T, variant, stream=None):
    """One Cholesky-QR pass on the k x k column-major device Gram matrix G (SCTM_CHOL_CTA or
    _CLUSTER kernel) into T; returns the status."""
    return load().sctm_chol_orth(_ptr(G), int(k), float(shift), _ptr(T), int(variant),
                                 ctypes.c_void_p(stream))


def sctm_jacobi_svd(B, k, S, U, W, variant, stream=None):
    """Jacobi SVD of the k x k column-major device matrix B (SCTM_JACOBI_CTA or _CLUSTER kernel);
    returns the status."""
    return load().sctm_jacobi_svd(_ptr(B), int(k), _ptr(S), _ptr(U), _ptr(W), int(variant),
                                  ctypes.c_void_p(stream))


def sctm_gemm(X, Y, O, M, N, K, precision, stream=None):
    """O = X Y (row-major device matrices) in the given SCTM_PREC_* form; returns the status."""
    return load().sctm_gemm(_ptr(X), _ptr(Y), _ptr(O), int(M), int(N), int(K), int(precision),
                            ctypes.c_void_p(stream))


def sctm_iterate_batch(ctxs, max_it, tol):
    n = len(ctxs)
    arr = (ctypes.c_void_p * n)(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    st = (ctypes.c_int * n)()
    it = (ctypes.c_int * n)()
    ds = (ctypes.c_double * n)()
    s = load().sctm_iterate_batch(arr, n, int(max_it), float(tol), st, it, ds)
    return s, list(st), list(it), list(ds)


def sctm_set_grad_mode(ctx, mode, tol=1e-10, max_matvecs=400, svd_grad_cutoff=1e-6):
    return load().sctm_set_grad_mode(ctx, int(mode), float(tol), int(max_matvecs),
                                     float(svd_grad_cutoff))


def sctm_adjoint_info(ctx):
    mv = (ctypes.c_int * 2)()
    res = (ctypes.c_double * 2)()
    st = load().sctm_adjoint_info(ctx, mv, res)
    return st, list(mv), list(res)


def sctm_autotune_info(ctx, network):
    emu, total = ctypes.c_int(0), ctypes.c_int(0)
    st = load().sctm_autotune_info(ctx, int(network), ctypes.byref(emu), ctypes.byref(total))
    return st, emu.value, total.value


def sctm_device_bytes(ctx):
    return int(load().sctm_device_bytes(ctx))


def sctm_set_profiling(ctx, mode):
    """mode 0 off, 1 events around launches (concurrent streams), 2 serialised execution."""
    return load().sctm_set_profiling(ctx, int(mode))


def sctm_profile(ctx, reset=False):
    ctr_ms, svd_ms = ctypes.c_double(0), ctypes.c_double(0)
    cl, cf, sc_, kl = (ctypes.c_longlong(0) for _ in range(4))
    st = load().sctm_profile(ctx, ctypes.byref(ctr_ms), ctypes.byref(cl), ctypes.byref(cf),
                             ctypes.byref(svd_ms), ctypes.byref(sc_), ctypes.byref(kl), int(reset))
    return st, {'ctr_ms': ctr_ms.value, 'ctr_launches': cl.value, 'ctr_flops': cf.value,
                'svd_ms': svd_ms.value, 'svd_calls': sc_.value, 'kernel_launches': kl.value}


SCTM_KERNEL_F64, SCTM_KERNEL_SKINNY, SCTM_KERNEL_TC, SCTM_KERNEL_F64EMU, SCTM_KERNEL_JACOBI, \
    SCTM_KERNEL_CHOL = range(6)


def sctm_profile_kernel(ctx, kernel):
    ms = ctypes.c_double(0)
    ln, fl, by = (ctypes.c_longlong(0) for _ in range(3))
    st = load().sctm_profile_kernel(ctx, int(kernel), ctypes.byref(ms), ctypes.byref(ln),
                                    ctypes.byref(fl), ctypes.byref(by))
    return st, {'ms': ms.value, 'launches': ln.value, 'flops': fl.value, 'bytes': by.value}


def unpack_env(buf, chi, D, d):
    """Split an exported environment into {'C1'..'C4': (chi,chi), 'T1'..'T4': [ket,int,bra]}."""
    env = {}
    off = 0
    for c in ('C1', 'C2', 'C3', 'C4'):
        env[c] = buf[off:off + chi * chi].reshape(chi, chi)
        off += chi * chi
    for t in ('T1', 'T2', 'T3', 'T4'):
        lst = []
        for m in (D, d, D):
            lst.append(buf[off:off + chi * chi * m].reshape(chi, chi, m))
            off += chi * chi * m
        env[t] = lst
    return env


def unpack_env_reduced(buf, chi, m):
    """The reduced method's environment: {'C1'..'C4': (chi, chi), 'T1'..'T4': (chi, chi, m)}."""
    env = {}
    off = 0
    for c in ('C1', 'C2', 'C3', 'C4'):
        env[c] = buf[off:off + chi * chi].reshape(chi, chi)
        off += chi * chi
    for t in ('T1', 'T2', 'T3', 'T4'):
        env[t] = buf[off:off + chi * chi * m].reshape(chi, chi, m)
        off += chi * chi * m
    return env


class SplitCTMRG:
    """Convenience owner of one context: create / iterate / f / g / destroy."""

    def __init__(self, peps, pepo, chi, T, precision=SCTM_PREC_FP64, cutoff=1e-12, seed=0,
                 svd_mode=SCTM_SVD_QR, method=SCTM_METHOD_SPLIT, p4_mode=SCTM_P4_FULL,
                 jacobi=SCTM_JACOBI_CTA):
        st, o = sctm_default_opts()
        p, D = peps.shape[0], peps.shape[1]
        o.T, o.D, o.p, o.d = float(T), D, p, pepo.shape[2]
        o.precision, o.svd_cutoff, o.init_seed = precision, cutoff, seed
        o.svd_mode = svd_mode
        o.method = method
        o.p4_mode = p4_mode
        o.jacobi = jacobi
        self.method = method
        self.chi, self.D, self.p, self.d = chi, D, p, pepo.shape[2]
        st, self.ctx = sctm_create(np.ascontiguousarray(peps, dtype=np.float64),
                                   np.ascontiguousarray(pepo, dtype=np.float64), chi, o)
        if st != SCTM_OK:
            raise SctmError(st, 'sctm_create failed')

    def _check(self, st, allow=(SCTM_OK,)):
        if st not in allow:
            raise SctmError(st, sctm_last_error(self.ctx))
        return st

    def iterate(self, max_it, tol=0.0):
        st, it, ds = sctm_iterate(self.ctx, max_it, tol)
        self._check(st, (SCTM_OK, SCTM_ENOCONV))
        return st, it, ds

    def free_energy(self):
        st, f = sctm_free_energy(self.ctx)
        self._check(st, (SCTM_OK, SCTM_ENOCONV))
        return f

    def grad(self):
        g = np.zeros((self.p,) + (self.D,) * 4)
        self._check(sctm_grad(self.ctx, g), (SCTM_OK, SCTM_ENOCONV))
        return g

    def env(self, network):
        st, buf = sctm_env_export(self.ctx, network)
        self._check(st)
        d = self.d if network == SCTM_NET_NUM else 1
        if self.method == SCTM_METHOD_REDUCED:
            return unpack_env_reduced(buf, self.chi, self.D * d * self.D)
        return unpack_env(buf, self.chi, self.D, d)

    def close(self):
        if self.ctx:
            sctm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
