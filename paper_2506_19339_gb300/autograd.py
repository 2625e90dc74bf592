"""torch.autograd interface of the split-CTMRG free energy: f(A) with d f / d A from the library's
fixed-point adjoint (sctm_grad in SCTM_GRAD_ADJOINT mode).

Argument marshalling only: the forward pass is sctm_set_peps + sctm_iterate + sctm_free_energy,
the backward pass sctm_grad, all on the GPU through the C ABI.  A context is reused across calls,
so each forward pass starts from the previous environment (warm start), as an optimiser of A
would use it.
"""
import numpy as np
import torch

from . import sctm


class FreeEnergyContext:
    """Owns one context for PEPS tensors of one shape.  grad_mode: SCTM_GRAD_ADJOINT (d f / d A,
    the default) or SCTM_GRAD_ENV (the paper's environment gradient)."""

    def __init__(self, pepo, chi, T, D, p=2, svd_mode=sctm.SCTM_SVD_PARTIAL_RANDOM,
                 max_it=400, tol=1e-10, adjoint_tol=1e-10, max_matvecs=400, seed_peps=None,
                 grad_mode=sctm.SCTM_GRAD_ADJOINT, precision=sctm.SCTM_PREC_FP64,
                 svd_grad_cutoff=1e-6):
        st, o = sctm.sctm_default_opts()
        o.T, o.D, o.p, o.d = float(T), int(D), int(p), int(pepo.shape[2])
        o.svd_mode = svd_mode
        o.precision = precision
        o.grad_mode = grad_mode
        o.cuda_stream = torch.cuda.current_stream().cuda_stream
        A0 = seed_peps if seed_peps is not None else np.ones((p,) + (D,) * 4) / np.sqrt(p * D ** 4)
        st, self.ctx = sctm.sctm_create(np.ascontiguousarray(A0, dtype=np.float64),
                                        np.ascontiguousarray(pepo, dtype=np.float64), chi, o)
        if st != sctm.SCTM_OK:
            raise sctm.SctmError(st, 'sctm_create failed')
        st = sctm.sctm_set_grad_mode(self.ctx, grad_mode, adjoint_tol, max_matvecs,
                                     svd_grad_cutoff)
        if st != sctm.SCTM_OK:
            raise sctm.SctmError(st, sctm.sctm_last_error(self.ctx))
        self.max_it, self.tol, self.cold = max_it, tol, True
        self.last_iterations = 0

    def close(self):
        if self.ctx:
            sctm.sctm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 -- interpreter shutdown
            pass


class SplitCTMRGFreeEnergy(torch.autograd.Function):
    """f = SplitCTMRGFreeEnergy.apply(A, fctx): A a float64 CUDA tensor (p, D, D, D, D)."""

    @staticmethod
    def forward(ctx, A, fctx):
        A = A.detach().contiguous()
        st = sctm.sctm_set_peps(fctx.ctx, A, 1 if fctx.cold else 0)
        if st != sctm.SCTM_OK:
            raise sctm.SctmError(st, sctm.sctm_last_error(fctx.ctx))
        fctx.cold = False
        st, it, ds = sctm.sctm_iterate(fctx.ctx, fctx.max_it, fctx.tol)
        if st not in (sctm.SCTM_OK, sctm.SCTM_ENOCONV):
            raise sctm.SctmError(st, sctm.sctm_last_error(fctx.ctx))
        fctx.last_iterations = it
        st, f = sctm.sctm_free_energy(fctx.ctx)
        if st not in (sctm.SCTM_OK, sctm.SCTM_ENOCONV):
            raise sctm.SctmError(st, sctm.sctm_last_error(fctx.ctx))
        ctx.fctx = fctx
        ctx.shape = A.shape
        return torch.tensor(f, dtype=torch.float64, device=A.device)

    @staticmethod
    def backward(ctx, grad_f):
        g = torch.empty(ctx.shape, dtype=torch.float64, device=grad_f.device)
        st = sctm.sctm_grad(ctx.fctx.ctx, g)
        if st not in (sctm.SCTM_OK, sctm.SCTM_ENOCONV):
            raise sctm.SctmError(st, sctm.sctm_last_error(ctx.fctx.ctx))
        return grad_f * g, None


def free_energy(A, fctx):
    return SplitCTMRGFreeEnergy.apply(A, fctx)
