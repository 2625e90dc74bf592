"""Exact reference contractions on tiny periodic systems, FP64 (oracle; test infrastructure only).

These pin the network conventions of the oracle independently of any CTMRG:
* the tensor trace of the PEPO network equals the 3D Ising partition function
  (Sec. II, Eq. "TN for partition function");
* the transfer-matrix overlap <psi|T|psi> built by explicit enumeration equals the tensor trace of
  the reduced site tensor a = A-bar O A (Sec. II, Eq. "free energy expression" and Fig. 3(a)).
"""
import itertools

import numpy as np

from .ising import boltzmann_matrix, sqrt_boltzmann


def ising_Z_enumeration(beta, L):
    """Z = sum_{s} prod_<ij> W(s_i, s_j) on a periodic Lx x Ly x Lz cubic lattice by summing over
    all 2^N spin configurations (Sec. II, the product of bond weights).  Periodic directions of
    length 2 carry two distinct bonds between the same pair of sites, as the tensor trace does."""
    Lx, Ly, Lz = L
    N = Lx * Ly * Lz
    idx = np.arange(N).reshape(Lx, Ly, Lz)
    cfg = ((np.arange(2 ** N)[:, None] >> np.arange(N)[None, :]) & 1)
    spin = 1 - 2 * cfg  # index 0 -> +1, index 1 -> -1
    E = np.zeros(2 ** N)
    for x in range(Lx):
        for y in range(Ly):
            for z in range(Lz):
                i = idx[x, y, z]
                for j in (idx[(x + 1) % Lx, y, z], idx[x, (y + 1) % Ly, z], idx[x, y, (z + 1) % Lz]):
                    E += spin[:, i] * spin[:, j]
    return float(np.sum(np.exp(beta * E)))


def pepo_network_trace(O, L):
    """tTr of the uniform PEPO network on a periodic Lx x Ly x Lz lattice (Sec. II,
    Eq. "TN for partition function"), evaluated as Tr(T^Lz) where T is the plane-to-plane
    transfer matrix of one layer of O tensors (rows: the s_dn legs, columns: the s_up legs).
    O's legs are (s_up, s_dn, u, l, d, r) = (z+, z-, y-, x-, y+, x+)."""
    Lx, Ly, Lz = L
    N = Lx * Ly
    sites = [(x, y) for x in range(Lx) for y in range(Ly)]
    hb = {}
    vb = {}
    c = 2 * N
    for (x, y) in sites:
        hb[(x, y)] = c; c += 1
        vb[(x, y)] = c; c += 1
    ops = []
    for n, (x, y) in enumerate(sites):
        legs = [N + n, n, vb[(x, (y - 1) % Ly)], hb[((x - 1) % Lx, y)], vb[(x, y)], hb[(x, y)]]
        ops += [O, legs]
    layer = np.einsum(*ops, list(range(2 * N)), optimize='greedy').reshape(2 ** N, 2 ** N)
    return float(np.trace(np.linalg.matrix_power(layer, Lz)))


def peps_torus_amplitudes(A, Lx, Ly):
    """psi(s_1..s_N) of the periodic Lx x Ly PEPS built from A[s,u,l,d,r] (Sec. II, Fig. 2(a)),
    returned as a vector over the 2^N physical configurations (site n = x*Ly + y, the bit of
    site n is the slowest-varying for n = 0)."""
    N = Lx * Ly
    ops = []
    phys = list(range(N))
    h = {}
    v = {}
    c = N
    for x in range(Lx):
        for y in range(Ly):
            h[(x, y)] = c; c += 1
            v[(x, y)] = c; c += 1
    for x in range(Lx):
        for y in range(Ly):
            n = x * Ly + y
            legs = [phys[n], v[(x, (y - 1) % Ly)], h[((x - 1) % Lx, y)], v[(x, y)], h[(x, y)]]
            ops += [A, legs]
    psi = np.einsum(*ops, phys, optimize='greedy')
    return psi.reshape(-1)


def transfer_matrix_torus(beta, Lx, Ly):
    """The plane-to-plane transfer matrix T(s, s') of the 3D Ising model for a periodic Lx x Ly
    plane, by enumeration: T(s,s') = sum_k prod_i Q(k_i,s_i) Q(k_i,s'_i) prod_<ij> W(k_i,k_j)
    with Q = sqrt(W) (Sec. II: one plane of uniform O tensors; the in-plane bond between two O is
    Q Q^T = W).  Configurations are ordered as in peps_torus_amplitudes."""
    N = Lx * Ly
    W = boltzmann_matrix(beta)
    Q = sqrt_boltzmann(beta)
    cfg = ((np.arange(2 ** N)[:, None] >> (N - 1 - np.arange(N))[None, :]) & 1)
    w = np.ones(2 ** N)
    for x in range(Lx):
        for y in range(Ly):
            i = x * Ly + y
            for j in (((x + 1) % Lx) * Ly + y, x * Ly + (y + 1) % Ly):
                w *= W[cfg[:, i], cfg[:, j]]
    Qn = np.ones((1, 1))
    for _ in range(N):
        Qn = np.kron(Qn, Q)
    return Qn.T @ (w[:, None] * Qn)


def reduced_site_tensor(A, O, B):
    """a[(ua,uo,ub),(la,lo,lb),(da,do,db),(ra,ro,rb)] = sum_{s,s'} A[s,..] O[s',s,..] B[s',..]:
    the single-layer tensor of the reduced method (Sec. II, Fig. 3(a)), bond D*d*D."""
    a = np.einsum('sabcd,tsefgh,tijkl->aeibfjcgkdhl', A, O, B)
    D1, d1, D2 = A.shape[1], O.shape[2], B.shape[1]
    m = D1 * d1 * D2
    return a.reshape(m, m, m, m)


def torus_trace_site(a, Lx, Ly):
    """tTr of the periodic Lx x Ly network of a single-layer tensor a[u,l,d,r]."""
    ops = []
    h = {}
    v = {}
    c = 0
    for x in range(Lx):
        for y in range(Ly):
            h[(x, y)] = c; c += 1
            v[(x, y)] = c; c += 1
    for x in range(Lx):
        for y in range(Ly):
            ops += [a, [v[(x, (y - 1) % Ly)], h[((x - 1) % Lx, y)], v[(x, y)], h[(x, y)]]]
    return float(np.einsum(*ops, [], optimize='greedy'))
