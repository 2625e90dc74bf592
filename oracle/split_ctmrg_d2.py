"""D2-symmetric split-CTMRG, plain FP64 NumPy (oracle; test infrastructure only).

Follows arXiv:2506.19339 Sec. III.B, the passage on lattice symmetries with Eq. "Symmetry
constraints" and the figure of symmetric corner absorption (absent from the source, so it is
read as stated below).

Symmetry.  For a real PEPS A whose virtual legs are invariant under the square's group D4 and
a PEPO invariant under the cube's group, the nested triple-layer network (A up-left, O in the
middle, the bra B = A down-right of each cell) keeps the subgroup D2 generated by
  * the reflection about the main diagonal (``split_ctmrg.frame_transpose``), and
  * the rotation by 180 degrees together with the exchange ket <-> bra
    (``split_ctmrg.frame_rotate``).
An environment invariant under both is fixed by C1, C4 and the left edge T4^{ket,int,bra}; in
the leg conventions of ``split_ctmrg``
    C3 = C1 = C1^T,    C2 = C4 = C4^T,    T1^X = T4^X,
    T2 = T3 = rev(T4),  rev: (ket, int, bra) -> (bra, int, ket), each with its two chain bonds
                        exchanged,
which is the paper's Eq. "Symmetry constraints" written in these conventions.

Iteration (reading of the symmetric scheme).  One set of projectors per iteration, the six
pairs of the left move of the current (symmetric) environment, updates every tensor:
  * the left edge T4 is renormalised exactly as in the directional left move;
  * each corner absorbs one column and one row at once -- C1: itself, the top edge of the
    column, the left edge of the row and the site; C4 the same with the bottom edge -- and both
    of its legs are truncated by the one alpha pair, the second leg read in the reflected frame
    (about the main diagonal for C1, about the anti-diagonal for C4);
  * C1 and C4 are symmetrised, C <- (C + C^T) / 2 (a no-op up to rounding: the update is
    symmetric by construction), and every tensor is divided by its Frobenius norm.
The other eight edge tensors and two corners follow from the constraints above.  At a fixed
point of the directional scheme that is invariant up to gauge, the same environment is a fixed
point of this iteration: both give the same f.

The PEPS and its gradient are kept in the symmetric subspace by the group average
``d4_project`` (Sec. III.B: both A and g are projected at each optimisation step).
"""
import numpy as np

from . import split_ctmrg as sc

KET, INT, BRA = sc.KET, sc.INT, sc.BRA


# ----------------------------------------------------------------------------------------------
# the symmetric subspace of the PEPS (Sec. III.B)
# ----------------------------------------------------------------------------------------------

def d4_permutations():
    """The eight elements of D4 acting on the virtual legs (u, l, d, r) = axes 1..4 of A[s,u,l,d,r],
    as axis permutations of A: the four rotations of the cyclic order u -> l -> d -> r and the
    four reflections (each rotation followed by the exchange u <-> l, d <-> r)."""
    rot = [1, 2, 3, 4]
    perms = []
    for k in range(4):
        r = rot[k:] + rot[:k]
        perms.append((0,) + tuple(r))
        refl = [r[1], r[0], r[3], r[2]]
        perms.append((0,) + tuple(refl))
    return perms


def d4_project(A):
    """Group average (1/8) sum_g g.A: the orthogonal projection onto the D4-invariant tensors."""
    A = np.asarray(A, dtype=np.float64)
    return sum(A.transpose(p) for p in d4_permutations()) / 8.0


# ----------------------------------------------------------------------------------------------
# symmetric environment
# ----------------------------------------------------------------------------------------------

def _rev(lst):
    return [sc._swapab(lst[BRA]), sc._swapab(lst[INT]), sc._swapab(lst[KET])]


def sym_env(C1, C4, T4):
    """The full environment (all sixteen slots) that the constraints give from C1, C4, T4."""
    T4 = list(T4)
    return {'C1': C1, 'C2': C4, 'C3': C1, 'C4': C4,
            'T1': list(T4), 'T2': _rev(T4), 'T3': _rev(T4), 'T4': T4}


def sym_init_env(chi, D, d, seed=0):
    """Cold start: C1, C4 and T4 drawn as in ``split_ctmrg.init_env`` (same counters), the two
    corners symmetrised; the rest from the constraints."""
    e = sc.init_env(chi, D, d, seed)
    C1 = 0.5 * (e['C1'] + e['C1'].T)
    C4 = 0.5 * (e['C4'] + e['C4'].T)
    return sym_env(C1, C4, e['T4'])


def constraint_residual(env):
    """Largest deviation of a full environment from Eq. "Symmetry constraints" (relative to the
    largest entry of the slot compared), used to check the directional scheme's own fixed point
    shape and this module's bookkeeping."""
    def rel(X, Y):
        return float(np.max(np.abs(X - Y)) / max(np.max(np.abs(Y)), 1e-300))
    r = [rel(env['C1'], env['C1'].T), rel(env['C4'], env['C4'].T),
         rel(env['C3'], env['C1']), rel(env['C2'], env['C4'])]
    for x in range(3):
        r.append(rel(env['T1'][x], env['T4'][x]))
    rv = _rev(env['T4'])
    for x in range(3):
        r.append(rel(env['T2'][x], rv[x]))
        r.append(rel(env['T3'][x], rv[x]))
    return max(r)


# ----------------------------------------------------------------------------------------------
# one symmetric iteration
# ----------------------------------------------------------------------------------------------

# the enlarged corners (a corner with one column and one row absorbed) are the directional
# module's; the symmetric corner update below truncates both of their legs
enlarged_c1 = sc.enlarged_c1
enlarged_c4 = sc.enlarged_c4


# the opposite boundary's stage-1 pairs as the 180-degree-rotation images of this boundary's (the
# geometry is the directional scheme's; the D2 symmetry makes them the opposite boundary's pairs
# of the same environment)
mirror_stage1 = sc.opposite_stage1


# the half projector 4's patch: with the D2 symmetry the up / down moves' projector 1 are this
# move's own P_1T / P_1B (the defaults of ``split_ctmrg.half_p4_halves``)
half_p4_halves = sc.half_p4_halves


def sym_projectors(env, A, O, B, chi, cutoff=1e-12, p4='full', pr='mirror', info=None):
    """The six composite projector pairs of one symmetric iteration (the left move's cuts,
    Sec. III.C and Appendix): stage 1 (P1, P2, P3) from the one-column patches; the opposite
    boundary's stage-1 pairs by symmetry (pr='mirror', the paper's D2 scheme) or by their own SVDs
    (pr='svd', as in the directional scheme); stage 2: P5, P6 from the 1x2-cell patches, P4 from
    the 2x2-cell patch (p4='full') or the 2x1-cell patch (p4='half')."""
    halves = sc.one_column_halves(env, A, O, B)
    left = {cut: sc.projector_pair(U, L, sc.T_AXES_LEFT[cut], chi, cutoff)
            for cut, (U, L) in halves.items()}
    if pr == 'mirror':
        right = mirror_stage1(left)
    else:
        right = {cut: sc.projector_pair(U, L, sc.T_AXES_RIGHT[cut], chi, cutoff)
                 for cut, (U, L) in halves.items()}
    halves2 = sc.two_column_halves(env, A, O, B, left, right, alpha=(p4 != 'half'))
    if p4 == 'half':
        halves2['alpha'] = half_p4_halves(env, A, O, B, left)
    stage2 = {cut: sc.projector_pair(U2, L2, (0, 1, 2), chi, cutoff)
              for cut, (U2, L2) in halves2.items()}
    if info is not None:
        info['left'], info['right'], info['stage2'] = left, right, stage2
    return sc.composite_projectors(left, stage2)


def sym_iteration(env, A, O, B, chi, cutoff=1e-12, symmetrise=True, info=None, p4='full',
                  pr='mirror'):
    """One iteration of the symmetric scheme on a symmetric environment (module docstring).
    The projectors are the left move's; the edge is the left move's T4'.  Each corner absorbs
    its column and row at once (``enlarged_c1`` / ``enlarged_c4``) and both of its legs are
    truncated by the alpha pair: C1 (above the row cut, left of the column cut) takes P_T on
    both legs; C4 (below the row cut) takes P_B on both, its column-cut leg read in the frame
    reflected about the anti-diagonal, where ket and bra trade places, so that P_B's
    (bond, A_v, O_v, B_v) meets (bond, B.r, O.r, A.r).
    symmetrise=False leaves out the final C <- (C + C^T) / 2 (to measure how symmetric the
    update comes out by itself).  Returns the new symmetric environment (``sym_env``)."""
    pinfo = {}
    P = sym_projectors(env, A, O, B, chi, cutoff, p4, pr, pinfo)
    _, T4n, _ = sc.renormalise(env, A, O, B, P)
    PaB, PaT = P['alpha']                            # [xl, A_v, O_v, B_v, k], [k, xl, ...]
    Ct1 = enlarged_c1(env, A, O, B)
    X = sc._c2('hpqrvabc,kvabc->hpqrk', Ct1, PaT)
    C1n = sc._c2('hpqrk,jhpqr->jk', X, PaT)
    Ct4 = enlarged_c4(env, A, O, B)
    X = sc._c2('vabchpqr,vabck->hpqrk', Ct4, PaB)
    C4n = sc._c2('hpqrk,hrqpj->jk', X, PaB)
    if info is not None:
        info['asym'] = (float(np.linalg.norm(C1n - C1n.T) / np.linalg.norm(C1n)),
                        float(np.linalg.norm(C4n - C4n.T) / np.linalg.norm(C4n)))
        info['projectors'] = P
        info.update(pinfo)
    if symmetrise:
        C1n = 0.5 * (C1n + C1n.T)
        C4n = 0.5 * (C4n + C4n.T)
    C1n = C1n / np.linalg.norm(C1n)
    C4n = C4n / np.linalg.norm(C4n)
    T4n = [t / np.linalg.norm(t) for t in T4n]
    return sym_env(C1n, C4n, T4n)


def sym_iterate(env, A, O, B, chi, max_iter, tol=None, cutoff=1e-12, trace=None, p4='full',
                pr='mirror'):
    """Iterate to ||S[i+1] - S[i]||_2 < tol with the convergence measure of Sec. III.D
    (``split_ctmrg.ctm_spectrum``).  Returns (env, iterations, last dS, spectrum)."""
    S_old = np.zeros(chi)
    dS = np.inf
    it = 0
    for it in range(1, max_iter + 1):
        env = sym_iteration(env, A, O, B, chi, cutoff, p4=p4, pr=pr)
        S = np.zeros(chi)
        s = sc.ctm_spectrum(env)
        S[:len(s)] = s[:chi]
        dS = float(np.linalg.norm(S - S_old))
        S_old = S
        if trace is not None:
            trace.append(dS)
        if tol is not None and dS < tol:
            break
    return env, it, dS, S_old


def sym_evaluate(A, O_num, O_den, T, chi, max_iter, tol=None, cutoff=1e-12, seed=0, p4='full',
                 pr='mirror'):
    """f and the projected environment gradient of the D4-projected PEPS (Eqs. "free energy
    expression" and "gradient expression", Sec. III.B for the projections), both networks
    iterated from the symmetric cold start."""
    A = d4_project(A)
    p, D = A.shape[0], A.shape[1]
    res = {}
    for name, O in (('num', O_num), ('den', O_den)):
        d = O.shape[2]
        env = sym_init_env(chi, D, d, seed)
        env, it, dS, S = sym_iterate(env, A, O, A, chi, max_iter, tol, cutoff, p4=p4, pr=pr)
        loc = sc.local_contractions(env, A, O, A)
        E = sc.bra_environment(env, loc)
        res[name] = {'env': env, 'iters': it, 'dS': dS, 'S': S, 'lnk': sc.ln_kappa(loc),
                     'Z11': loc['Z11'], 'E': E}
    beta_f = -(res['num']['lnk'] - res['den']['lnk'])
    g = -2.0 * (res['num']['E'] / res['num']['Z11'] - res['den']['E'] / res['den']['Z11'])
    res['beta_f'] = beta_f
    res['f'] = T * beta_f
    res['g'] = d4_project(T * g)
    res['A'] = A
    return res
