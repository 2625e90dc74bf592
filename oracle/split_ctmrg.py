"""Split-CTMRG for the triple-layer PEPS-PEPO-PEPS network, plain FP64 NumPy
(oracle; test infrastructure only).

Follows arXiv:2506.19339 Sec. III (split-CTM environment, left move, six-projector scheme,
projector construction of Eqs. "projector construction" / "projector construction 2",
convergence criterion), the Appendix (the patches of projectors 1-6) and Sec. II
(Eqs. "free energy expression" and "gradient expression").  Steps that the paper defines only in
its figures (absent from the source) follow one fixed reading, restated where it is used.

Conventions
-----------
Site tensors (Sec. II): ket A[s,u,l,d,r], PEPO O[s_up,s_dn,u,l,d,r] (s_dn joins A.s, s_up joins
the bra), bra B[s,u,l,d,r] (B = A-bar = A for a real PEPS).

Nested planar embedding (Sec. III.A, Fig. 4(a) reading): in every unit cell A sits up-left, O in
the middle, B down-right.  Hence every boundary carries its three edge tensors in the order
ket, int, bra -- top to bottom on the left/right boundaries, left to right on the top/bottom ones.

Environment E = {C1..C4, T1..T4 x (ket, int, bra)} (Sec. III.A):
  C1[h,v] top-left  (h -> top chain, v -> left chain)    C2[h,v] top-right (h -> top, v -> right)
  C3[h,v] bottom-right (h -> bottom, v -> right)         C4[h,v] bottom-left (h -> bottom, v -> left)
  T1^X[a,b,m] top chain, a = left bond, b = right bond, m = down into X.u
  T2^X[a,b,m] right chain, a = up, b = down, m = left into X.r
  T3^X[a,b,m] bottom chain, a = left, b = right, m = up into X.d
  T4^X[a,b,m] left chain, a = up, b = down, m = right into X.l

Cuts of the left boundary after a column is absorbed (reading of Fig. 5):
  alpha (between rows)         legs (xl, A_v, O_v, B_v, xr)
  kappa (inside a row, k | i)  legs (xl, A.d, s, O.u, B.u, xr)
  iota  (inside a row, i | b)  legs (xl, A.d, O.d, s', B.u, xr)
(xl / xr: the left / right environment bonds of a patch.)
"""
import numpy as np

KET, INT, BRA = 0, 1, 2


def _c(spec, *ops):
    return np.einsum(spec, *ops, optimize='greedy')


# ----------------------------------------------------------------------------------------------
# environment
# ----------------------------------------------------------------------------------------------

_MASK64 = (1 << 64) - 1
ENV_SLOTS = ('C1', 'C2', 'C3', 'C4', 'T1k', 'T1i', 'T1b', 'T2k', 'T2i', 'T2b',
             'T3k', 'T3i', 'T3b', 'T4k', 'T4i', 'T4b')


def splitmix64_uniform(seed, counters):
    """Uniform doubles in [0, 1) from the SplitMix64 generator (Steele, Lea & Flood, OOPSLA 2014):
    the output for counter c is the generator's (c+1)-th output from state `seed`, i.e.
        z = seed + (c + 1) * 0x9E3779B97F4A7C15   (mod 2^64)
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9;  z = (z ^ (z >> 27)) * 0x94D049BB133111EB
        z = z ^ (z >> 31);                          u = (z >> 11) * 2^-53."""
    out = np.empty(len(counters))
    for n, c in enumerate(counters):
        z = (seed + (int(c) + 1) * 0x9E3779B97F4A7C15) & _MASK64
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        z = z ^ (z >> 31)
        out[n] = (z >> 11) * (1.0 / 9007199254740992.0)
    return out


def init_env(chi, D, d, seed=0):
    """Deterministic cold start at the full bond dimension chi (the paper gives none).  Entry j
    (row-major) of environment slot q (order C1..C4, T1^{k,i,b}, T2^{k,i,b}, T3^{k,i,b},
    T4^{k,i,b}) is splitmix64_uniform(seed, q * 2^32 + j).  A full-rank start is needed: the
    all-ones rank-1 boundary leaves the kappa / iota bonds of a product PEPS at rank 1 forever,
    because their stage-1 patches see the rest of the lattice only through the opposite
    boundary's bond."""
    shapes = [(chi, chi)] * 4 + [(chi, chi, m) for _ in range(4) for m in (D, d, D)]
    vals = []
    for q, shp in enumerate(shapes):
        n = int(np.prod(shp))
        vals.append(splitmix64_uniform(seed, (q << 32) + np.arange(n)).reshape(shp))
    env = {'C1': vals[0], 'C2': vals[1], 'C3': vals[2], 'C4': vals[3]}
    for k, t in enumerate(('T1', 'T2', 'T3', 'T4')):
        env[t] = vals[4 + 3 * k: 7 + 3 * k]
    return env


def copy_env(env):
    return {k: ([t.copy() for t in v] if isinstance(v, list) else v.copy()) for k, v in env.items()}


# ----------------------------------------------------------------------------------------------
# frames: the right, up and down moves are the left move in a relabelled network
# ----------------------------------------------------------------------------------------------

def _swapab(T):
    return T.transpose(1, 0, 2)


def frame_transpose(env, A, O, B):
    """Reflection about the main diagonal (x <-> y).  It maps the nested cell onto itself (A
    stays up-left), so the up move is the left move in this frame."""
    e = {
        'C1': env['C1'].T, 'C2': env['C4'].T, 'C3': env['C3'].T, 'C4': env['C2'].T,
        'T1': list(env['T4']), 'T2': list(env['T3']), 'T3': list(env['T2']), 'T4': list(env['T1']),
    }
    return (e, A.transpose(0, 2, 1, 4, 3), O.transpose(0, 1, 3, 2, 5, 4), B.transpose(0, 2, 1, 4, 3))


def frame_rotate(env, A, O, B):
    """Rotation by 180 degrees combined with the exchange ket <-> bra.  The rotation moves A to
    the down-right corner of the cell, where B was; relabelling the layers restores the nested
    cell, so the right move is the left move in this frame.  Chains reverse direction (a <-> b)
    and their ket/bra entries trade places; O exchanges s_up <-> s_dn."""
    def rev(lst):
        return [_swapab(lst[BRA]), _swapab(lst[INT]), _swapab(lst[KET])]
    e = {
        'C1': env['C3'], 'C2': env['C4'], 'C3': env['C1'], 'C4': env['C2'],
        'T1': rev(env['T3']), 'T2': rev(env['T4']), 'T3': rev(env['T1']), 'T4': rev(env['T2']),
    }
    return (e, B.transpose(0, 3, 4, 1, 2), O.transpose(1, 0, 4, 5, 2, 3), A.transpose(0, 3, 4, 1, 2))


def to_frame(move, env, A, O, B):
    if move == 'L':
        return dict(env), A, O, B
    if move == 'U':
        return frame_transpose(env, A, O, B)
    if move == 'R':
        return frame_rotate(env, A, O, B)
    if move == 'D':
        return frame_transpose(*frame_rotate(env, A, O, B))
    raise ValueError(move)


def from_frame(move, env_f):
    """Inverse relabelling (both primitive frames are involutions)."""
    dummy = np.zeros((1, 1, 1, 1, 1))
    dO = np.zeros((1, 1, 1, 1, 1, 1))
    if move == 'L':
        return env_f
    if move == 'U':
        return frame_transpose(env_f, dummy, dO, dummy)[0]
    if move == 'R':
        return frame_rotate(env_f, dummy, dO, dummy)[0]
    if move == 'D':
        e = frame_transpose(env_f, dummy, dO, dummy)[0]
        return frame_rotate(e, dummy, dO, dummy)[0]
    raise ValueError(move)


# ----------------------------------------------------------------------------------------------
# projector construction (Sec. III.C)
# ----------------------------------------------------------------------------------------------

def projector_pair(U, L, t_axes, chi, cutoff):
    """Projectors for one cut from its upper half U (rho_T) and lower half L (rho_B), Sec. III.C.

    U and L carry the same cut legs in the same order.  t_axes are the legs to be truncated; the
    rest are the remaining (non-truncated) legs r.  As matrices rho_T = U[t, r] and
    rho_B = L[t, r]^T, so rho_B rho_T = L^T U is contracted over t and is a matrix on the
    remaining legs (the SVD runs on the non-truncated indices, Sec. V / Appendix).
        rho_B rho_T = U_s S V_s^T,   keep the largest chi singular values,
        P_B = rho_T V~ (S~^1/2)^+    (t x chi, attached to the tensors below the cut),
        P_T = (S~^1/2)^+ U~^T rho_B  (chi x t, attached to the tensors above the cut),
    Eq. "projector construction 2"; P_T P_B = I on the kept (non-zero) part.  The pseudo-inverse
    zeroes s_k / s_1 < cutoff.  Sign gauge: each pair (u_k, v_k) is flipped so that the entry of
    u_k with the largest magnitude (first such index) is positive.

    Returns P_B with shape t_dims + (chi,), P_T with shape (chi,) + t_dims, and the full spectrum.
    chi=None keeps every singular value (no truncation; used by the exactness tests).
    """
    r_axes = [i for i in range(U.ndim) if i not in t_axes]
    perm = list(t_axes) + r_axes
    tdims = [U.shape[i] for i in t_axes]
    rdims = [U.shape[i] for i in r_axes]
    nt = int(np.prod(tdims))
    nr = int(np.prod(rdims))
    Um = U.transpose(perm).reshape(nt, nr)
    Lm = L.transpose(perm).reshape(nt, nr)
    M = Lm.T @ Um
    _count(float(nr) * nr * nt)
    Us, S, Vh = np.linalg.svd(M)
    if chi is None:
        chi = S.shape[0]
    k = min(chi, S.shape[0])
    Ut = Us[:, :k].copy()
    Vt = Vh[:k, :].T.copy()
    s = S[:k]
    for j in range(k):
        i = int(np.argmax(np.abs(Ut[:, j])))
        if Ut[i, j] < 0:
            Ut[:, j] *= -1.0
            Vt[:, j] *= -1.0
    inv = np.where(s > cutoff * S[0], 1.0 / np.sqrt(np.where(s > 0, s, 1.0)), 0.0)
    PB = np.zeros((nt, chi))
    PT = np.zeros((chi, nt))
    PB[:, :k] = (Um @ Vt) * inv[None, :]
    PT[:k, :] = ((Lm @ Ut) * inv[None, :]).T
    _count(2.0 * nt * nr * k)
    return PB.reshape(tdims + [chi]), PT.reshape([chi] + tdims), S


# ----------------------------------------------------------------------------------------------
# insertion and absorption (Sec. III.B, Fig. 5(a),(b))
# ----------------------------------------------------------------------------------------------

# Algorithmic FLOP count of the contractions evaluated so far: 2 x the product of the dimensions
# of every distinct label of a pairwise contraction (its multiply-adds), and 2 M N K for the
# projector matrix products.  reset_flops() zeroes it; SVDs are not counted.
FLOPS = {'contractions': 0}


def reset_flops():
    FLOPS['contractions'] = 0


def _count(n_macs):
    FLOPS['contractions'] += 2 * int(n_macs)


def _c2(spec, X, Y):
    """Pairwise contraction written as an einsum spec and evaluated with a BLAS matrix product
    (numpy.tensordot): every label shared by X and Y and absent from the output is summed."""
    ins, out = spec.split('->')
    a, b = ins.split(',')
    dims = dict(zip(a, X.shape))
    dims.update(zip(b, Y.shape))
    _count(np.prod([dims[c] for c in dims], dtype=np.float64))
    shared = [c for c in a if c in b and c not in out]
    for c in a + b:
        if c not in out and (c in a) == (c in b):
            continue
        if c not in out:
            raise ValueError('label %r of %r is neither shared nor kept' % (c, spec))
    if any(c in b and c in out for c in a):
        return np.einsum(spec, X, Y)
    R = np.tensordot(X, Y, axes=([a.index(c) for c in shared], [b.index(c) for c in shared]))
    rest = [c for c in a if c not in shared] + [c for c in b if c not in shared]
    return R.transpose([rest.index(c) for c in out])


def absorbed_corners(env):
    """Each corner with the edge tensors of one inserted column (Fig. 5(b)):
        Ct1[h, v, ua, uo, ub] = C1 T1^ket T1^int T1^bra   (h -> right, v -> down)
        Ct2[h, w, ua, uo, ub] = T1^ket T1^int T1^bra C2   (h -> left,  w -> down)
        Ct4[h, v, da, do, db] = C4 T3^ket T3^int T3^bra   (h -> right, v -> up)
        Ct3[h, w, da, do, db] = T3^ket T3^int T3^bra C3   (h -> left,  w -> up)"""
    T1k, T1i, T1b = env['T1']
    T3k, T3i, T3b = env['T3']
    X = _c2('av,acp->vcp', env['C1'], T1k)
    X = _c2('vcp,ceo->vepo', X, T1i)
    Ct1 = _c2('vepo,ehb->hvpob', X, T1b)
    X = _c2('egb,gw->ewb', T1b, env['C2'])
    X = _c2('ceo,ewb->cwob', T1i, X)
    Ct2 = _c2('hcp,cwob->hwpob', T1k, X)
    X = _c2('av,acE->vcE', env['C4'], T3k)
    X = _c2('vcE,cef->veEf', X, T3i)
    Ct4 = _c2('veEf,ehg->hvEfg', X, T3b)
    X = _c2('egG,gw->ewG', T3b, env['C3'])
    X = _c2('cef,ewG->cwfG', T3i, X)
    Ct3 = _c2('hcE,cwfG->hwEfG', T3k, X)
    return Ct1, Ct2, Ct3, Ct4


def top_block(C1, T1, C2):
    """C1 T1^ket T1^int T1^bra C2 -> [v1, ua, uo, ub, v2] (the top boundary of a one-column patch)."""
    X = _c2('av,abx->vbx', C1, T1[KET])
    X = _c2('vbx,bcy->vcxy', X, T1[INT])
    X = _c2('vcxy,cez->vexyz', X, T1[BRA])
    return _c2('vexyz,ew->vxyzw', X, C2)


def bottom_block(C4, T3, C3):
    """C4 T3^ket T3^int T3^bra C3 -> [v4, da, do, db, v3]."""
    return top_block(C4, T3, C3)


def upper_halves(Ctop, T4, T2, A, O, B):
    """Upper halves of the one-column patch at the kappa, iota and alpha cuts of one row: the top
    boundary plus the row's tensors above the cut (A with its T^ket; then O with T^int; then B
    with T^bra).  Canonical leg orders as in the module docstring."""
    X = _c2('vaobw,vxl->xaoblw', Ctop, T4[KET])
    X = _c2('xaoblw,saler->xobwser', X, A)
    Uk = _c2('xobwser,wyr->xesoby', X, T2[KET])
    X = _c2('xesoby,xXl->Xesobyl', Uk, T4[INT])
    X = _c2('Xesobyl,tsolfr->Xebyftr', X, O)
    Ui = _c2('Xebyftr,yYr->XeftbY', X, T2[INT])
    X = _c2('xeftby,xXl->Xeftbyl', Ui, T4[BRA])
    X = _c2('Xeftbyl,tblgr->Xefygr', X, B)
    Ua = _c2('Xefygr,yYr->XefgY', X, T2[BRA])
    return Uk, Ui, Ua


def lower_halves(Cbot, T4, T2, A, O, B):
    """Lower halves at the iota, kappa and alpha cuts: the bottom boundary plus the row's tensors
    below the cut (B with T^bra; then O with T^int; then A with T^ket)."""
    X = _c2('vefgw,xvl->xefgwl', Cbot, T4[BRA])
    X = _c2('xefgwl,tblgr->xefwtbr', X, B)
    Li = _c2('xefwtbr,ywr->xeftby', X, T2[BRA])
    X = _c2('XeftbY,xXl->xeftbYl', Li, T4[INT])
    X = _c2('xeftbYl,tsolfr->xebYsor', X, O)
    Lk = _c2('xebYsor,yYr->xesoby', X, T2[INT])
    X = _c2('XesobY,xXl->xesobYl', Lk, T4[KET])
    X = _c2('xesobYl,saler->xobYar', X, A)
    La = _c2('xobYar,yYr->xaoby', X, T2[KET])
    return Li, Lk, La


def one_column_halves(env, A, O, B):
    """(rho_T, rho_B) of the one-column patches used by the stage-1 projectors, keyed by cut:
    1 row for kappa / iota (paper: 1x1 cells), 2 rows for alpha (paper: 1x2 cells).  Each patch is
    closed by the left and right environment columns and by the top / bottom boundaries."""
    Ctop = top_block(env['C1'], env['T1'], env['C2'])
    Cbot = bottom_block(env['C4'], env['T3'], env['C3'])
    Uk, Ui, Ua = upper_halves(Ctop, env['T4'], env['T2'], A, O, B)
    Li, Lk, La = lower_halves(Cbot, env['T4'], env['T2'], A, O, B)
    return {'alpha': (Ua, La), 'kappa': (Uk, Lk), 'iota': (Ui, Li)}


# truncated legs of each stage-1 projector, as axes of the canonical cut orders
#   left column (this move): the bra-related legs plus xl            (P1, P2, P3)
#   right column (the opposite boundary): the ket-related legs plus xr
#   alpha: left (xl, B_v)        right (xr, A_v)
#   kappa: left (xl, s, B.u)     right (xr, A.d, s)
#   iota:  left (xl, s', B.u)    right (xr, A.d, s')
# The O vertical line is always left to stage 2.  (Putting O.u into the kappa stage-1 group makes
# the kappa bond rank of each boundary bounded by the opposite boundary's, a loop in which a lost
# singular value never returns: a product PEPS then stays at rank 2.)
T_AXES_LEFT = {'alpha': (0, 3), 'kappa': (0, 2, 4), 'iota': (0, 3, 4)}
T_AXES_RIGHT = {'alpha': (4, 1), 'kappa': (5, 1, 2), 'iota': (5, 1, 3)}


def stage1_projectors(halves, chi, cutoff):
    """P1 (alpha), P2 (kappa), P3 (iota) on the bra-related legs of this move's column, and the
    mirror-image stage-1 pairs of the opposite boundary on the ket-related legs of the next column
    (Fig. 5(c) and Appendix; the paper takes the latter from the right move)."""
    left, right = {}, {}
    for cut, (U, L) in halves.items():
        left[cut] = projector_pair(U, L, T_AXES_LEFT[cut], chi, cutoff)
        right[cut] = projector_pair(U, L, T_AXES_RIGHT[cut], chi, cutoff)
    return left, right


# ----------------------------------------------------------------------------------------------
# two-column patches (stage 2)
# ----------------------------------------------------------------------------------------------

def two_column_halves(env, A, O, B, left, right, alpha=True):
    """(rho_T, rho_B) of the two-column patches used by the stage-2 projectors P4 (alpha, 2x2
    cells), P5 (kappa, 1x2 cells) and P6 (iota, 1x2 cells).  Column x belongs to this move and is
    renormalised on its bra-related legs by the stage-1 pair; column x+1 is renormalised on its
    ket-related legs by the opposite boundary's stage-1 pair.  Leg orders:
        kappa: (k2, A.d, O.u | O.u', B.u', kR)   iota: (k3, A.d, O.d | O.d', B.u', kR)
        alpha: (k1, A_v, O_v | O_v', B_v', kR)
    alpha=False leaves out the alpha patch (the half projector 4 uses its own, 2x1 cells)."""
    Ct1, Ct2, Ct3, Ct4 = absorbed_corners(env)
    T4k, T4i, T4b = env['T4']
    T2k, T2i, T2b = env['T2']
    PBk, PTk, _ = left['kappa']
    PBi, PTi, _ = left['iota']
    PBa, PTa, _ = left['alpha']
    QBk, QTk, _ = right['kappa']
    QBi, QTi, _ = right['iota']
    QBa, QTa, _ = right['alpha']
    out = {}

    # ---- kappa (one row)
    X = _c2('hvpob,vxl->hpobxl', Ct1, T4k)
    X = _c2('hpobxl,splEr->hobxsEr', X, A)
    UL = _c2('hobxsEr,kxsb->hkEor', X, PTk)
    X = _c2('hwpob,wyr->hpobyr', Ct2, T2k)
    X = _c2('hpobyr,splEr->hobysEl', X, A)
    UR = _c2('hobysEl,kyEs->hlobk', X, QTk)
    U2 = _c2('hkEor,hrOBK->kEoOBK', UL, UR)
    X = _c2('hvEfg,Xvm->hEfgXm', Ct4, T4b)
    X = _c2('hEfgXm,tbmgQ->hEfXtbQ', X, B)
    X = _c2('hEfXtbQ,xXl->hEftbQxl', X, T4i)
    X = _c2('hEftbQxl,tsolfR->hEbQxsoR', X, O)
    LL = _c2('hEbQxsoR,xsbk->hkEoRQ', X, PBk)
    X = _c2('hwEfG,Ywm->hEfGYm', Ct3, T2b)
    X = _c2('hEfGYm,tbMGm->hEfYtbM', X, B)
    X = _c2('hEfYtbM,yYl->hEftbMyl', X, T2i)
    X = _c2('hEftbMyl,tsoLfl->hEbMysoL', X, O)
    LR = _c2('hEbMysoL,yEsk->hLMobk', X, QBk)
    L2 = _c2('hkEoRQ,hRQOBK->kEoOBK', LL, LR)
    out['kappa'] = (U2, L2)

    # ---- iota (one row)
    X = _c2('hvpob,vxl->hpobxl', Ct1, T4k)
    X = _c2('hpobxl,splEr->hobxsEr', X, A)
    X = _c2('hobxsEr,xXL->hobsErXL', X, T4i)
    X = _c2('hobsErXL,tsoLfR->hbErXtfR', X, O)
    UL = _c2('hbErXtfR,kXtb->hkEfrR', X, PTi)
    X = _c2('hwpob,wyr->hpobyr', Ct2, T2k)
    X = _c2('hpobyr,splEr->hobysEl', X, A)
    X = _c2('hobysEl,yYR->hobsElYR', X, T2i)
    X = _c2('hobsElYR,tsoLfR->hbElYtfL', X, O)
    UR = _c2('hbElYtfL,kYEt->hlLfbk', X, QTi)
    U2 = _c2('hkEfrR,hrRFBK->kEfFBK', UL, UR)
    X = _c2('hvEfg,xvm->hEfgxm', Ct4, T4b)
    X = _c2('hEfgxm,tbmgQ->hEfxtbQ', X, B)
    LL = _c2('hEfxtbQ,xtbk->hkEfQ', X, PBi)
    X = _c2('hwEfG,ywm->hEfGym', Ct3, T2b)
    X = _c2('hEfGym,tbMGm->hEfytbM', X, B)
    LR = _c2('hEfytbM,yEtk->hMfbk', X, QBi)
    L2 = _c2('hkEfQ,hQFBK->kEfFBK', LL, LR)
    out['iota'] = (U2, L2)

    if not alpha:
        return out
    # ---- alpha (two rows): quarters Q1 (upper-left), Q2 (upper-right), Q4, Q3
    X = _c2('hvpob,vxl->hpobxl', Ct1, T4k)
    X = _c2('hpobxl,splEr->hobxsEr', X, A)
    X = _c2('hobxsEr,xXL->hobsErXL', X, T4i)
    X = _c2('hobsErXL,tsoLfR->hbErXtfR', X, O)
    X = _c2('hbErXtfR,XZM->hbErtfRZM', X, T4b)
    X = _c2('hbErtfRZM,tbMgS->hErfRZgS', X, B)
    Q1 = _c2('hErfRZgS,kZg->hkEfrRS', X, PTa)
    X = _c2('hwpob,wyr->hpobyr', Ct2, T2k)
    X = _c2('hpobyr,splEr->hobysEl', X, A)
    X = _c2('hobysEl,yYR->hobsElYR', X, T2i)
    X = _c2('hobsElYR,tsoLfR->hbElYtfL', X, O)
    X = _c2('hbElYtfL,YWS->hbElWtfLS', X, T2b)
    X = _c2('hbElWtfLS,tbMgS->hElWfLMg', X, B)
    Q2 = _c2('hElWfLMg,kWE->hlLMfgk', X, QTa)
    U2 = _c2('hkEfrRS,hrRSFGK->kEfFGK', Q1, Q2)
    X = _c2('hvEfg,YvM->hEfgYM', Ct4, T4b)
    X = _c2('hEfgYM,tbMgS->hEfYtbS', X, B)
    X = _c2('hEfYtbS,XYL->hEftbSXL', X, T4i)
    X = _c2('hEftbSXL,tsoLfR->hEbSXsoR', X, O)
    X = _c2('hEbSXsoR,xXl->hEbSsoRxl', X, T4k)
    X = _c2('hEbSsoRxl,splEr->hbSoRxpr', X, A)
    Q4 = _c2('hbSoRxpr,xbk->hkporRS', X, PBa)
    X = _c2('hwEfg,WwS->hEfgWS', Ct3, T2b)
    X = _c2('hEfgWS,tbMgS->hEfWtbM', X, B)
    X = _c2('hEfWtbM,ZWR->hEftbMZR', X, T2i)
    X = _c2('hEftbMZR,tsoLfR->hEbMZsoL', X, O)
    X = _c2('hEbMZsoL,yZr->hEbMsoLyr', X, T2k)
    X = _c2('hEbMsoLyr,splEr->hbMoLypl', X, A)
    Q3 = _c2('hbMoLypl,ypk->hlLMobk', X, QBa)
    L2 = _c2('hkporRS,hrRSOBK->kpoOBK', Q4, Q3)
    out['alpha'] = (U2, L2)
    return out


# ----------------------------------------------------------------------------------------------
# enlarged corners and the half projector 4 (Appendix, projector 4(b))
# ----------------------------------------------------------------------------------------------

def enlarged_c1(env, A, O, B):
    """C1 with one column and one row absorbed: C1, the top edge T1^{k,i,b} of the column, the left
    edge T4^{k,i,b} of the row and the site's three layers, as
        Ct[h, A.r, O.r, B.r, v, A.d, O.d, B.d]
    (h: the top chain's bond right of the column; v: the left chain's bond below the row)."""
    T1k, T1i, T1b = env['T1']
    T4k, T4i, T4b = env['T4']
    X = _c2('aw,acp->wcp', env['C1'], T1k)
    X = _c2('wcp,ceo->wepo', X, T1i)
    X = _c2('wepo,ehq->whpoq', X, T1b)
    X = _c2('whpoq,wxl->hpoqxl', X, T4k)
    X = _c2('hpoqxl,splDR->hoqxsDR', X, A)
    X = _c2('hoqxsDR,xym->hoqsDRym', X, T4i)
    X = _c2('hoqsDRym,tsomEF->hqDRytEF', X, O)
    X = _c2('hqDRytEF,yvn->hqDRtEFvn', X, T4b)
    X = _c2('hqDRtEFvn,tqnGH->hDREFvGH', X, B)
    return X.transpose(0, 2, 4, 7, 5, 1, 3, 6)


def enlarged_c4(env, A, O, B):
    """C4 with one column and one row absorbed: C4, the bottom edge T3^{k,i,b} of the column, the
    left edge T4^{k,i,b} of the row and the site, as
        Ct[v, A.u, O.u, B.u, h, A.r, O.r, B.r]
    (v: the left chain's bond above the row; h: the bottom chain's bond right of the column)."""
    T3k, T3i, T3b = env['T3']
    T4k, T4i, T4b = env['T4']
    X = _c2('aw,acp->wcp', env['C4'], T3k)
    X = _c2('wcp,ceo->wepo', X, T3i)
    X = _c2('wepo,ehq->whpoq', X, T3b)
    X = _c2('whpoq,ywn->hpoqyn', X, T4b)
    X = _c2('hpoqyn,tUnqR->hpoytUR', X, B)
    X = _c2('hpoytUR,xym->hpotURxm', X, T4i)
    X = _c2('hpotURxm,tsVmoS->hpURxsVS', X, O)
    X = _c2('hpURxsVS,vxl->hpURsVSvl', X, T4k)
    X = _c2('hpURsVSvl,sWlpQ->hURVSvWQ', X, A)
    return X.transpose(5, 6, 3, 1, 0, 7, 4, 2)


def half_p4_halves(env, A, O, B, left, col_T=None, col_B=None):
    """(rho_T, rho_B) of the half projector 4 (Appendix, projector 4(b)): the 2x1 patch of the
    two enlarged left corners, the bra lines of both their legs renormalised by projector 1 --
    this move's P_1T / P_1B on the row cut, and on the column cut the up / down moves' projector 1:
    col_T = the up move's P_1T[k, xl, B_v] for the upper corner, col_B = the down move's
    P_1B[xl, B_v, k] for the lower one, each in its own move's frame (in the down move's frame ket
    and bra trade places, so there it acts on the ket line A.r).  In the D2-symmetric scheme
    both are this move's own pair (the defaults).  Leg orders:
        rho_T (k1, A.d, O.d | k2, A.r, O.r)    rho_B (k1, A.u, O.u | k2, B.r, O.r)
    the first three legs cut by projector 4, the last three remaining."""
    PBa, PTa, _ = left['alpha']                      # [xl, B_v, k], [k, xl, B_v]
    cT = PTa if col_T is None else col_T
    cB = PBa if col_B is None else col_B
    Ct1 = enlarged_c1(env, A, O, B)                   # [h, A.r, O.r, B.r, v, A.d, O.d, B.d]
    X = _c2('hpqrvabc,kvc->hpqrkab', Ct1, PTa)
    U = _c2('hpqrkab,jhr->kabjpq', X, cT)
    Ct4 = enlarged_c4(env, A, O, B)                   # [v, A.u, O.u, B.u, h, A.r, O.r, B.r]
    X = _c2('vabchpqr,vck->kabhpqr', Ct4, PBa)
    L = _c2('kabhpqr,hpj->kabjrq', X, cB)
    return U, L


def perpendicular_alpha_pairs(env, A, O, B, chi, cutoff=1e-12):
    """The up and down moves' stage-1 alpha pairs (P1) of this environment, each computed in its
    own frame (the half projector 4 of the directional scheme takes them from the same
    environment, as P^R is taken; see ``left_move``)."""
    out = []
    for w in ('U', 'D'):
        e, a, o, b = to_frame(w, env, A, O, B)
        Ct = top_block(e['C1'], e['T1'], e['C2'])
        Cb = bottom_block(e['C4'], e['T3'], e['C3'])
        Ua = upper_halves(Ct, e['T4'], e['T2'], a, o, b)[2]
        La = lower_halves(Cb, e['T4'], e['T2'], a, o, b)[2]
        out.append(projector_pair(Ua, La, T_AXES_LEFT['alpha'], chi, cutoff))
    return out


def composite_projectors(left, stage2):
    """Stage-1 then stage-2 projector of each cut, as one tensor on the cut's legs:
        P_alpha,B[xl, A_v, O_v, B_v, k],     P_alpha,T[k, xl, A_v, O_v, B_v]
        P_kappa,B[xl, A.d, s, O.u, B.u, k],  P_kappa,T[k, ...]
        P_iota,B [xl, A.d, O.d, s', B.u, k], P_iota,T [k, ...]"""
    PBa, PTa, _ = left['alpha']
    PBk, PTk, _ = left['kappa']
    PBi, PTi, _ = left['iota']
    P4B, P4T, _ = stage2['alpha']
    P5B, P5T, _ = stage2['kappa']
    P6B, P6T, _ = stage2['iota']
    return {
        'alpha': (_c2('xbK,Kaok->xaobk', PBa, P4B), _c2('kKao,Kxb->kxaob', P4T, PTa)),
        'kappa': (_c2('xsbK,Keok->xesobk', PBk, P5B), _c2('kKeo,Kxsb->kxesob', P5T, PTk)),
        'iota': (_c2('xtbK,Kefk->xeftbk', PBi, P6B), _c2('kKef,Kxtb->kxeftb', P6T, PTi)),
    }


def renormalise(env, A, O, B, P):
    """Fig. 5(c): C1' = C1~ P_alpha,T;  T4'^ket = P_alpha,B T4~^ket P_kappa,T;
    T4'^int = P_kappa,B T4~^int P_iota,T;  T4'^bra = P_iota,B T4~^bra P_alpha,T;
    C4' = C4~ P_alpha,B.  The lines that cross an edge tensor (e.g. O_v and B_v across T4~^ket)
    are summed between its two projectors; no identity tensor is formed."""
    Ct1, _, _, Ct4 = absorbed_corners(env)
    T4k, T4i, T4b = env['T4']
    PaB, PaT = P['alpha']
    PkB, PkT = P['kappa']
    PiB, PiT = P['iota']
    C1n = _c2('hvpob,kvpob->hk', Ct1, PaT)
    C4n = _c2('hvEfg,vEfgk->hk', Ct4, PaB)
    X = _c2('xpobK,xXl->pobKXl', PaB, T4k)
    X = _c2('pobKXl,splEr->obKXsEr', X, A)
    T4kn = _c2('obKXsEr,kXEsob->Kkr', X, PkT)
    X = _c2('xEsobK,xXL->EsobKXL', PkB, T4i)
    X = _c2('EsobKXL,tsoLfR->EbKXtfR', X, O)
    T4in = _c2('EbKXtfR,kXEftb->KkR', X, PiT)
    X = _c2('xEftbK,xXM->EftbKXM', PiB, T4b)
    X = _c2('EftbKXM,tbMgS->EfKXgS', X, B)
    T4bn = _c2('EfKXgS,kXEfg->KkS', X, PaT)
    return C1n, [T4kn, T4in, T4bn], C4n


# ----------------------------------------------------------------------------------------------
# the left move (Sec. III.B, Fig. 5): insertion, absorption, six-projector truncation
# ----------------------------------------------------------------------------------------------

def opposite_stage1(left):
    """The opposite boundary's stage-1 pairs as the images of this boundary's under the rotation
    by 180 degrees with ket <-> bra, the relabelling that turns the left move into the right move
    (``frame_rotate``; likewise the up move into the down move).  The Appendix's captions of
    projectors 4-6 take the right column's stage-1 pairs from the right move; in the D2-symmetric
    scheme that move is this one's image, so P^R_1T = P_1B, P^R_1B = P_1T, P^R_2T = P_3B,
    P^R_2B = P_3T, P^R_3T = P_2B, P^R_3B = P_2T.  The rotation puts the right column's alpha cut
    onto the left column's alpha cut, its kappa cut (ket | int) onto the left iota cut
    (int | bra) and its iota cut onto the left kappa cut, with the right environment bond onto
    the left one, the ket lines onto the bra lines and the physical line A-O onto O-A-bar.  Leg
    orders:
        right alpha (xr, A_v)      <- left alpha (xl, B_v)
        right kappa (xr, A.d, s)   <- left iota  (xl, s', B.u)
        right iota  (xr, A.d, s')  <- left kappa (xl, s, B.u)"""
    PBa, PTa, Sa = left['alpha']
    PBk, PTk, Sk = left['kappa']
    PBi, PTi, Si = left['iota']
    return {
        'alpha': (PTa.transpose(1, 2, 0), PBa.transpose(2, 0, 1), Sa),
        'kappa': (PTi.transpose(1, 3, 2, 0), PBi.transpose(3, 0, 2, 1), Si),
        'iota': (PTk.transpose(1, 3, 2, 0), PBk.transpose(3, 0, 2, 1), Sk),
    }


def stage1_left(env, A, O, B, chi, cutoff=1e-12):
    """This move's own stage-1 pairs (P1, P2, P3 on the bra-related legs of its column)."""
    halves = one_column_halves(env, A, O, B)
    return {cut: projector_pair(U, L, T_AXES_LEFT[cut], chi, cutoff) for cut, (U, L) in halves.items()}


def left_move(env, A, O, B, chi, cutoff=1e-12, info=None, normalise=True, right=None, p4='full'):
    """One left move.  Returns the renormalised, Frobenius-normalised (C1', [T4'^k, T4'^i, T4'^b],
    C4').

    Stage 1 (bra-related legs, P1 P2 P3) uses a one-column patch closed by the left and right
    environments: 2 rows for alpha (paper: 1x2 cells), 1 row for kappa / iota (paper: 1x1).
    Stage 2 (ket-related legs, P4 P5 P6) uses the two-column patch of the same height whose
    left column is already renormalised by the stage-1 pair and whose right column is
    renormalised by the mirror-image stage-1 pair of the opposite boundary (paper: "full"
    projector 4 and the 1x2 cells of projectors 5 and 6, with P^R computed in the same move).
    right: the opposite boundary's stage-1 pairs to use instead (``opposite_stage1`` of the
    opposite move's pairs: the paper's reading, P^R from the right move); None computes them here.
    p4: 'full' (the 2x2-cell patch) or 'half' (the 2x1-cell patch of the two enlarged corners,
    its column cuts renormalised by the up and down moves' P1 computed here from the same
    environment, ``perpendicular_alpha_pairs``).
    """
    halves = one_column_halves(env, A, O, B)
    if right is None:
        left, right = stage1_projectors(halves, chi, cutoff)
    else:
        left = {cut: projector_pair(U, L, T_AXES_LEFT[cut], chi, cutoff)
                for cut, (U, L) in halves.items()}
    halves2 = two_column_halves(env, A, O, B, left, right, alpha=(p4 != 'half'))
    if p4 == 'half':
        up, down = perpendicular_alpha_pairs(env, A, O, B, chi, cutoff)
        halves2['alpha'] = half_p4_halves(env, A, O, B, left, up[1], down[0])
    elif p4 != 'full':
        raise ValueError(p4)
    stage2 = {cut: projector_pair(U2, L2, (0, 1, 2), chi, cutoff) for cut, (U2, L2) in halves2.items()}
    P = composite_projectors(left, stage2)
    C1n, T4n, C4n = renormalise(env, A, O, B, P)
    if normalise:
        C1n = C1n / np.linalg.norm(C1n)
        C4n = C4n / np.linalg.norm(C4n)
        T4n = [t / np.linalg.norm(t) for t in T4n]
    if info is not None:
        info['spectra'] = {**{'1' + c: v[2] for c, v in left.items()},
                           **{'R' + c: v[2] for c, v in right.items()},
                           **{'2' + c: v[2] for c, v in stage2.items()}}
        info['projectors'] = P
        info['halves'] = halves
        info['halves2'] = halves2
        info['left'], info['right'] = left, right
    return C1n, T4n, C4n


def move(env, A, O, B, which, chi, cutoff=1e-12, right=None, info=None, p4='full'):
    """One directional move ('L', 'R', 'U' or 'D') on the stored environment (right, info, p4: as
    ``left_move``, in the move's own frame)."""
    e, a, o, b = to_frame(which, env, A, O, B)
    C1n, T4n, C4n = left_move(e, a, o, b, chi, cutoff, info=info, right=right, p4=p4)
    e = dict(e)
    e['C1'], e['T4'], e['C4'] = C1n, T4n, C4n
    return from_frame(which, e)


OPPOSITE_MOVE = {'L': 'R', 'R': 'L', 'U': 'D', 'D': 'U'}
UPDATED = {'L': ('C1', 'C4', 'T4'), 'R': ('C2', 'C3', 'T2'), 'U': ('C1', 'C2', 'T1'),
           'D': ('C3', 'C4', 'T3')}  # the stored tensors each move renormalises


def paired_move(env, A, O, B, pair, chi, cutoff=1e-12, svd_count=None, p4='full'):
    """Two opposite moves ('LR' or 'UD') on one environment: each move's stage-1 pairs are computed
    once and serve both as its own (P1-P3) and, mapped by ``opposite_stage1``, as the other move's
    P^R (the Appendix takes P^R from the right move); each move's stage-2 pairs and its
    renormalisation use the environment both started from.  The moves renormalise disjoint
    tensors (UPDATED), so the results are merged.  Twelve SVDs per pair, where two sequential
    moves with P^R in the move take eighteen."""
    w1, w2 = pair
    frames = {w: to_frame(w, env, A, O, B) for w in pair}
    left = {w: stage1_left(*frames[w], chi, cutoff) for w in pair}
    out = dict(env)
    for w, other in ((w1, w2), (w2, w1)):
        e, a, o, b = frames[w]
        inf = {}
        # left_move recomputes this move's stage-1 pairs from the same halves (same values)
        C1n, T4n, C4n = left_move(e, a, o, b, chi, cutoff, info=inf,
                                  right=opposite_stage1(left[other]), p4=p4)
        e2 = dict(e)
        e2['C1'], e2['T4'], e2['C4'] = C1n, T4n, C4n
        new = from_frame(w, e2)
        for key in UPDATED[w]:
            out[key] = new[key]
    if svd_count is not None:
        svd_count[0] += 12 + (4 if p4 == 'half' else 0)
    return out


def ctm_spectrum(env):
    """Singular values of rho_eff = C1 C2 C3 C4 / Tr(C1 C2 C3 C4) (Sec. III.D), the matrix product
    taken around the plaquette starting at the bond between C4 and C1."""
    rho = env['C1'].T @ env['C2'] @ env['C3'].T @ env['C4']
    rho = rho / np.trace(rho)
    return np.linalg.svd(rho, compute_uv=False)


def iterate(env, A, O, B, chi, max_iter, tol=None, cutoff=1e-12, S_prev=None, trace=None,
            pr='in-move', svd_count=None, p4='full'):
    """Power iteration of the environment: each iteration is the left, right, up and down moves in
    that order (Sec. III.B); stop once ||S[i+1] - S[i]||_2 < tol (Sec. III.D).  Spectra shorter
    than chi are padded with zeros.  Returns (env, iterations done, last dS, spectrum).
    pr: where each move's opposite-boundary stage-1 pairs (P^R) come from -- 'in-move' (their
    own SVDs in the move, nine SVDs per move) or 'opposite-move' (the Appendix's reading: the
    pairs of the latest opposite move, left <-> right and up <-> down, mapped by
    ``opposite_stage1``; six SVDs per move once the opposite move has run) or 'paired' (left and
    right, then up and down, as ``paired_move`` on one environment each: P^R is the opposite
    move's pair of the same environment, twelve SVDs per pair).  svd_count: a list whose first
    entry is increased by the number of SVDs made.  p4: projector 4's patch, as ``left_move``
    (with 'half' every move makes two more SVDs, the up and down moves' P1)."""
    S_old = np.zeros(chi) if S_prev is None else S_prev
    dS = np.inf
    it = 0
    last = {}
    for it in range(1, max_iter + 1):
        if pr == 'paired':
            for pair in ('LR', 'UD'):
                env = paired_move(env, A, O, B, pair, chi, cutoff, svd_count, p4)
        for w in ('LRUD' if pr != 'paired' else ''):
            right = None
            if pr == 'opposite-move' and OPPOSITE_MOVE[w] in last:
                right = opposite_stage1(last[OPPOSITE_MOVE[w]])
            elif pr not in ('in-move', 'opposite-move', 'paired'):
                raise ValueError(pr)
            inf = {}
            env = move(env, A, O, B, w, chi, cutoff, right=right, info=inf, p4=p4)
            last[w] = inf['left']
            if svd_count is not None:
                svd_count[0] += (6 if right is not None else 9) + (2 if p4 == 'half' else 0)
        S = np.zeros(chi)
        s = ctm_spectrum(env)
        S[:len(s)] = s[:chi]
        dS = float(np.linalg.norm(S - S_old))
        S_old = S
        if trace is not None:
            trace.append(dS)
        if tol is not None and dS < tol:
            break
    return env, it, dS, S_old


# ----------------------------------------------------------------------------------------------
# free energy and gradient (Sec. II, Fig. 4(b),(c))
# ----------------------------------------------------------------------------------------------

def local_contractions(env, A, O, B):
    """Z00 (four corners), Z10 (corners + one column of T1/T3), Z01 (corners + one row of T4/T2)
    and Z11 (the full 3x3 network around one site, Fig. 4(b))."""
    C1, C2, C3, C4 = env['C1'], env['C2'], env['C3'], env['C4']
    T2, T4 = env['T2'], env['T4']
    Ctop = top_block(C1, env['T1'], C2)
    Cbot = bottom_block(C4, env['T3'], C3)
    Z00 = float(np.sum((C1.T @ C2) * (C4.T @ C3)))
    Z10 = float(np.sum(Ctop * Cbot))
    Lrow = top_block(C1.T, T4, C4.T)        # [h1, la, lo, lb, h4]: C1 T4^k T4^i T4^b C4
    Rrow = top_block(C2.T, T2, C3.T)        # [h1, ra, ro, rb, h4]: C2 T2^k T2^i T2^b C3
    Z01 = float(np.sum(Lrow * Rrow))
    Uk, Ui, Ua = upper_halves(Ctop, T4, T2, A, O, B)
    Li, Lk, La = lower_halves(Cbot, T4, T2, A, O, B)
    Z11 = float(np.sum(Uk * Lk))
    return {'Z00': float(Z00), 'Z10': Z10, 'Z01': float(Z01), 'Z11': Z11,
            'Uk': Uk, 'Ui': Ui, 'Ua': Ua, 'Lk': Lk, 'Li': Li, 'La': La, 'Cbot': Cbot, 'Ctop': Ctop}


def ln_kappa(loc):
    """ln of the per-site value kappa = Z11 Z00 / (Z10 Z01)."""
    kappa = loc['Z11'] * loc['Z00'] / (loc['Z10'] * loc['Z01'])
    if not np.isfinite(kappa) or kappa <= 0:
        raise FloatingPointError('kappa = %r is not a positive finite number' % kappa)
    return float(np.log(kappa))


def bra_environment(env, loc):
    """E[s, u, l, d, r]: the network of Fig. 4(c) -- Z11 with the bra tensor B removed."""
    T4, T2 = env['T4'], env['T2']
    X = _c2('xeftby,xvl->eftbylv', loc['Ui'], T4[BRA])
    X = _c2('eftbylv,vefgw->tbylgw', X, loc['Cbot'])
    return _c2('tbylgw,ywr->tblgr', X, T2[BRA])


def ket_environment(env, loc):
    """The same network with the ket tensor A removed (diagnostic only)."""
    T4, T2 = env['T4'], env['T2']
    X = _c2('vaobw,vxl->aobwxl', loc['Ctop'], T4[KET])
    X = _c2('aobwxl,xesoby->awlesy', X, loc['Lk'])
    return _c2('awlesy,wyr->saler', X, T2[KET])


def evaluate(A, O_num, O_den, T, chi, max_iter, tol=None, cutoff=1e-12, env_num=None, env_den=None,
             pr='in-move', p4='full'):
    """f and g for PEPS A at temperature T (Eqs. "free energy expression" and "gradient
    expression"):
        f = -T (ln kappa_num - ln kappa_den),
        g = 2 d f / d A-bar = -2T (E_num / Z11_num - E_den / Z11_den).
    The numerator <psi|T|psi> uses the Ising PEPO, the denominator <psi|psi> the identity PEPO.
    Each network is iterated from the cold start (or from the given environment); pr and p4 as
    ``iterate``."""
    A = np.asarray(A, dtype=np.float64)
    B = A
    p, D = A.shape[0], A.shape[1]
    res = {}
    for name, O, e0 in (('num', O_num, env_num), ('den', O_den, env_den)):
        d = O.shape[2]
        env = init_env(chi, D, d) if e0 is None else copy_env(e0)
        svds = [0]
        env, it, dS, S = iterate(env, A, O, B, chi, max_iter, tol, cutoff, pr=pr, svd_count=svds,
                                 p4=p4)
        loc = local_contractions(env, A, O, B)
        E = bra_environment(env, loc)
        res[name] = {'env': env, 'iters': it, 'dS': dS, 'S': S, 'lnk': ln_kappa(loc),
                     'Z11': loc['Z11'], 'E': E, 'loc': loc, 'svds': svds[0]}
    beta_f = -(res['num']['lnk'] - res['den']['lnk'])
    f = T * beta_f if np.isfinite(T) else np.nan
    g = -2.0 * (res['num']['E'] / res['num']['Z11'] - res['den']['E'] / res['den']['Z11'])
    if np.isfinite(T):
        g = T * g
    res['beta_f'] = beta_f
    res['f'] = f
    res['g'] = g
    return res


def fd_directional_derivative(A, O_num, O_den, T, chi, v, h, tol, env_num, env_den, max_iter=400,
                              cutoff=1e-12):
    """Central finite difference of the converged free energy along v:
        (f(A + h v) - f(A - h v)) / (2 h),
    each f the split-CTMRG result iterated until ||S[i+1] - S[i]||_2 < tol (Sec. III.D) from the
    given environments (the converged ones of A: a warm start; the fixed point is the same).  This
    is the plain definition of the derivative of f_chi(A) that the fixed-point adjoint computes;
    the paper's environment gradient (Eq. "gradient expression") differs from it by the
    environment's dependence on A, which vanishes as chi grows."""
    fp = evaluate(A + h * v, O_num, O_den, T, chi, max_iter, tol, cutoff, env_num, env_den)['f']
    fm = evaluate(A - h * v, O_num, O_den, T, chi, max_iter, tol, cutoff, env_num, env_den)['f']
    return (fp - fm) / (2.0 * h)
