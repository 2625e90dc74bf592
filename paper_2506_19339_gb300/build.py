"""Build libsctm.so in-tree with nvcc for sm_103a (GB300).

The translation units are compiled in parallel and linked against cuSOLVER / cuBLAS.  The
result (paper_2506_19339_gb300/libsctm.so) and the objects (paper_2506_19339_gb300/_build/)
are not tracked by git; every machine builds its own.
"""
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, 'csrc')
INCLUDE = os.path.join(ROOT, 'include')
BUILD = os.path.join(PKG, '_build')
LIB = os.path.join(PKG, 'libsctm.so')
SOURCES = ['kernels.cu', 'ctr_tc.cu', 'ctr_emu.cu', 'psvd.cu', 'engine.cu', 'adjoint.cu',
           'reduced.cu', 'api.cu', 'noalloc.cu']
ARCH = ['-gencode', 'arch=compute_103a,code=sm_103a']


def nvcc():
    for cand in (os.environ.get('NVCC'), shutil.which('nvcc'), '/usr/local/cuda/bin/nvcc'):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError('nvcc not found')


def _flags():
    return ['-O3', '-std=c++17', '-lineinfo', '-Xcompiler', '-fPIC', '-I', INCLUDE, '-I', CSRC] + ARCH


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, 'sctm.h'),
                                                               os.path.abspath(__file__)]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force=False, verbose=False):
    """Compile (if any source is newer than the library) and return the library path."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(BUILD, src.replace('.cu', '.o'))
        objs.append(obj)
        cmd = [cc, '-c', os.path.join(CSRC, src), '-o', obj] + _flags()
        if verbose:
            print(' '.join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(' '.join(cmd) + '\n' + out.decode(errors='replace'))
        elif verbose and out:
            print(out.decode(errors='replace'), file=sys.stderr)
    if errors:
        raise RuntimeError('nvcc failed:\n' + '\n'.join(errors))
    tmp = LIB + '.tmp'
    cmd = [cc, '-shared', '-o', tmp] + objs + ARCH + ['-lcusolver', '-lcublas']
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError('link failed:\n' + r.stdout.decode(errors='replace'))
    os.replace(tmp, LIB)
    return LIB


if __name__ == '__main__':
    print(build(force='--force' in sys.argv, verbose=True))
