"""Ising model tensors, FP64 (oracle; test infrastructure only).

Follows arXiv:2506.19339 Sec. II (delta tensor with split bond weights, Fig. 1, Eq. "SVD" and
Eq. "TN for partition function") and Sec. IV (3D Ising: W, its eigendecomposition and the
matrix square root sqrt(W)).
"""
import numpy as np


def boltzmann_matrix(beta, J=1.0):
    """Bond weight W(s_i, s_j) = exp(beta J s_i s_j) with spin up = index 0, spin down = index 1
    (Sec. IV, the 2x2 matrix W written below the Hamiltonian H = -sum s_i s_j)."""
    e = np.exp(beta * J)
    ie = np.exp(-beta * J)
    return np.array([[e, ie], [ie, e]], dtype=np.float64)


def sqrt_boltzmann(beta):
    """sqrt(W) = U lambda^(1/2) U^-1 by eigendecomposition of the real symmetric positive
    semi-definite W (Sec. IV).  Eigenvalues below zero from rounding are clipped (beta = 0
    makes W singular)."""
    W = boltzmann_matrix(beta)
    lam, U = np.linalg.eigh(W)
    lam = np.clip(lam, 0.0, None)
    return (U * np.sqrt(lam)) @ U.T


def ising_pepo(beta):
    """The uniform PEPO tensor O[s_up, s_dn, u, l, d, r] (Sec. II, Fig. 1(c)): the six-leg delta
    tensor with one sqrt(W) on each leg,
        O = sum_k Q[k,s_up] Q[k,s_dn] Q[k,u] Q[k,l] Q[k,d] Q[k,r],  Q = sqrt(W).
    s_dn contracts with the ket PEPS A, s_up with the bra PEPS (A-bar); d = 2."""
    Q = sqrt_boltzmann(beta)
    return np.einsum('ka,kb,kc,kd,ke,kf->abcdef', Q, Q, Q, Q, Q, Q)


def identity_pepo(p=2):
    """The operator of the norm network <psi|psi> written as a PEPO: delta(s_up, s_dn) with four
    in-plane legs of dimension 1.  With it the triple-layer engine contracts the double-layer
    network of Sec. III.A (the int layer becomes trivial)."""
    O = np.zeros((p, p, 1, 1, 1, 1))
    for s in range(p):
        O[s, s, 0, 0, 0, 0] = 1.0
    return O
