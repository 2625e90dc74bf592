"""Variational optimisation of the PEPS (Sec. IV.B): minimise the free-energy density f(A), an
upper bound of the exact one, with L-BFGS, each evaluation warm-started from the previous
environment.

The optimiser is torch.optim.LBFGS (host-side bookkeeping of a few p D^4 vectors); every f and
gradient comes from the library on the GPU through paper_2506_19339_gb300.autograd.  The paper
drives L-BFGS with its environment gradient (Eq. "gradient expression"); SCTM_GRAD_ADJOINT uses
the derivative of the converged f instead.
"""
import numpy as np
import torch

from . import autograd as sag
from . import sctm


def lbfgs_minimize(A0, T, chi, steps=10, grad_mode=sctm.SCTM_GRAD_ENV, lr=1.0, history_size=10,
                   svd_mode=sctm.SCTM_SVD_PARTIAL_RANDOM, max_it=400, tol=1e-10):
    """Minimise f over A from A0 (numpy, (p, D, D, D, D)) for the Ising PEPO at temperature T.
    Returns (A, history) with history a list of (f, |g|) per evaluation."""
    st, O = sctm.sctm_ising_pepo(T)
    if st != sctm.SCTM_OK:
        raise sctm.SctmError(st, 'sctm_ising_pepo')
    D, p = A0.shape[1], A0.shape[0]
    fctx = sag.FreeEnergyContext(O, chi, T, D, p=p, svd_mode=svd_mode, max_it=max_it, tol=tol,
                                 grad_mode=grad_mode)
    A = torch.from_numpy(np.ascontiguousarray(A0, dtype=np.float64)).cuda().requires_grad_(True)
    opt = torch.optim.LBFGS([A], lr=lr, history_size=history_size, max_iter=1,
                            line_search_fn='strong_wolfe')
    history = []

    def closure():
        opt.zero_grad()
        f = sag.free_energy(A, fctx)
        f.backward()
        history.append((float(f.detach()), float(A.grad.norm())))
        return f

    try:
        for _ in range(steps):
            opt.step(closure)
    finally:
        fctx.close()
    return A.detach().cpu().numpy(), history
