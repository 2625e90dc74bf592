"""The traditional reduced method, FP64 (oracle; test infrastructure only).

arXiv:2506.19339 Sec. II, Fig. 3: the physical legs of A, O and A-bar are contracted first into
a single-layer tensor a of bond D*d*D, which is then contracted with standard directional
CTMRG (corner tensors C, edge tensors T, projectors P).  This file is self-contained: it does not
use the split-CTMRG code, so that it can serve as an independent reference (the paper itself uses
the reduced method at large chi as its reference, Sec. IV.A).

Projectors: Corboz-style from the full 2x2 patch (the four quarters around the truncated bond),
rho_B rho_T contracted over the truncated legs, top-chi SVD, P_B = rho_T V S^-1/2,
P_T = S^-1/2 U^T rho_B.
"""
import numpy as np

from .bruteforce import reduced_site_tensor


def _c2(spec, X, Y):
    """Pairwise contraction written as an einsum spec and evaluated with a BLAS matrix product
    (numpy.tensordot): every label shared by X and Y and absent from the output is summed."""
    ins, out = spec.split('->')
    a, b = ins.split(',')
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


def _init(chi, m):
    C = np.zeros((chi, chi))
    C[0, 0] = 1.0
    T = np.zeros((chi, chi, m))
    T[0, 0, :] = 1.0
    return {'C1': C.copy(), 'C2': C.copy(), 'C3': C.copy(), 'C4': C.copy(),
            'T1': T.copy(), 'T2': T.copy(), 'T3': T.copy(), 'T4': T.copy()}


def _transpose(env, a):
    e = {'C1': env['C1'].T, 'C2': env['C4'].T, 'C3': env['C3'].T, 'C4': env['C2'].T,
         'T1': env['T4'], 'T2': env['T3'], 'T3': env['T2'], 'T4': env['T1']}
    return e, a.transpose(1, 0, 3, 2)


def _rotate(env, a):
    sw = lambda T: T.transpose(1, 0, 2)
    e = {'C1': env['C3'], 'C2': env['C4'], 'C3': env['C1'], 'C4': env['C2'],
         'T1': sw(env['T3']), 'T2': sw(env['T4']), 'T3': sw(env['T1']), 'T4': sw(env['T2'])}
    return e, a.transpose(2, 3, 0, 1)


def _pair(Rt, Rb, chi, cutoff):
    """Rt, Rb: matrices [t, r] (upper / lower half).  SVD of Rb^T Rt over the remaining legs."""
    M = Rb.T @ Rt
    U, S, Vh = np.linalg.svd(M)
    k = min(chi, len(S))
    U = U[:, :k]
    V = Vh[:k].T
    s = S[:k]
    inv = np.where(s > cutoff * S[0], 1.0 / np.sqrt(np.where(s > 0, s, 1.0)), 0.0)
    PB = np.zeros((Rt.shape[0], chi))
    PT = np.zeros((chi, Rt.shape[0]))
    PB[:, :k] = (Rt @ V) * inv
    PT[:k] = ((Rb @ U) * inv).T
    return PB, PT


def _left_move(env, a, chi, cutoff):
    C1, C2, C3, C4 = env['C1'], env['C2'], env['C3'], env['C4']
    T1, T2, T3, T4 = env['T1'], env['T2'], env['T3'], env['T4']
    m = a.shape[0]
    # quarters; t = (left bond, vertical site leg) at the cut between the two rows
    # [xl, a.d | h, a.r]
    Q1 = _c2('huxl,ulDr->xDhr', _c2('vhu,vxl->huxl', _c2('av,ahu->vhu', C1, T1), T4), a)
    # [h', a.l | a.d, xr]
    Q2 = _c2('Huyr,ulDr->HlDy', _c2('Hhu,hyr->Huyr', T1, _c2('hw,wyr->hyr', C2, T2)), a)
    # [xl, a.u | h, a.r]
    Q4 = _c2('hdxl,uldr->xuhr', _c2('vhd,xvl->hdxl', _c2('av,ahd->vhd', C4, T3), T4), a)
    # [h', a.l | a.u, xr]
    Q3 = _c2('Hdyr,uldr->Hluy', _c2('Hhd,hyr->Hdyr', T3, _c2('hw,ywr->hyr', C3, T2)), a)
    chi_l = T4.shape[1]
    Rt = _c2('xDhr,hrEy->xDEy', Q1, Q2).reshape(chi_l * m, -1)
    Rb = _c2('xuhr,hrEy->xuEy', Q4, Q3).reshape(chi_l * m, -1)
    PB, PT = _pair(Rt, Rb, chi, cutoff)
    PB = PB.reshape(chi_l, m, chi)
    PT = PT.reshape(chi, chi_l, m)
    C1n = _c2('vhu,kvu->hk', _c2('av,ahu->vhu', C1, T1), PT)
    C4n = _c2('vhd,vdk->hk', _c2('av,ahd->vhd', C4, T3), PB)
    T4n = _c2('KXDr,kXD->Kkr', _c2('uKXl,ulDr->KXDr', _c2('xuK,xXl->uKXl', PB, T4), a), PT)
    return [x / np.linalg.norm(x) for x in (C1n, T4n, C4n)]


def _move(env, a, w, chi, cutoff):
    if w == 'L':
        e, b = dict(env), a
    elif w == 'U':
        e, b = _transpose(env, a)
    elif w == 'R':
        e, b = _rotate(env, a)
    else:
        e, b = _transpose(*_rotate(env, a))
    C1n, T4n, C4n = _left_move(e, b, chi, cutoff)
    e = dict(e)
    e['C1'], e['T4'], e['C4'] = C1n, T4n, C4n
    if w == 'L':
        return e
    if w == 'U':
        return _transpose(e, a)[0]
    if w == 'R':
        return _rotate(e, a)[0]
    return _rotate(*_transpose(e, a))[0]


def _local(env, a):
    C1, C2, C3, C4 = env['C1'], env['C2'], env['C3'], env['C4']
    T1, T2, T3, T4 = env['T1'], env['T2'], env['T3'], env['T4']
    Z00 = float(np.sum((C1.T @ C2) * (C4.T @ C3)))
    top = _c2('vhu,hw->vuw', _c2('av,ahu->vhu', C1, T1), C2)
    bot = _c2('vhd,hw->vdw', _c2('av,ahd->vhd', C4, T3), C3)
    Z10 = float(np.sum(top * bot))
    lft = _c2('hxl,gx->hlg', _c2('hv,vxl->hxl', C1, T4), C4)
    rgt = _c2('hyl,gy->hlg', _c2('hw,wyl->hyl', C2, T2), C3)
    Z01 = float(np.sum(lft * rgt))
    X = _c2('vuw,vxl->uwxl', top, T4)
    X = _c2('uwxl,ulDr->wxDr', X, a)
    X = _c2('wxDr,wyr->xDy', X, T2)
    Z11 = float(np.sum(X * bot))
    return Z00, Z10, Z01, Z11, top, bot


def run(A, O, chi, max_iter, tol=None, cutoff=1e-12):
    """Reduced CTMRG of the network of a = A-bar O A.  Returns ln(kappa) and the bra environment E
    (Z11 with A-bar removed, in the layout of A) normalised by Z11."""
    a = reduced_site_tensor(A, O, A)
    m = a.shape[0]
    env = _init(chi, m)
    S_old = np.zeros(chi)
    dS = np.inf
    it = 0
    for it in range(1, max_iter + 1):
        for w in 'LRUD':
            env = _move(env, a, w, chi, cutoff)
        rho = env['C1'].T @ env['C2'] @ env['C3'].T @ env['C4']
        s = np.linalg.svd(rho / np.trace(rho), compute_uv=False)
        S = np.zeros(chi)
        S[:len(s)] = s[:chi]
        dS = float(np.linalg.norm(S - S_old))
        S_old = S
        if tol is not None and dS < tol:
            break
    loc = local_values(env, A, O)
    return {'lnk': float(np.log(loc['kappa'])), 'kappa': loc['kappa'], 'E': loc['E'] / loc['Z11'],
            'iters': it, 'dS': dS, 'env': env}


def local_values(env, A, O):
    """Z00, Z10, Z01, Z11, kappa = Z11 Z00 / (Z10 Z01) and the bra environment E (Z11 with A-bar
    removed, layout of A) for a reduced environment whose edge legs are grouped (A, O, A-bar)."""
    a = reduced_site_tensor(A, O, A)
    Z00, Z10, Z01, Z11, top, bot = _local(env, a)
    D, d = A.shape[1], O.shape[2]
    top6 = top.reshape(top.shape[0], D, d, D, top.shape[-1])
    bot6 = bot.reshape(bot.shape[0], D, d, D, bot.shape[-1])
    T4 = env['T4'].reshape(env['T4'].shape[0], env['T4'].shape[1], D, d, D)
    T2 = env['T2'].reshape(env['T2'].shape[0], env['T2'].shape[1], D, d, D)
    X = _c2('vpoqw,vxlLM->poqwxlLM', top6, T4)
    X = _c2('poqwxlLM,splEr->oqwxLMsEr', X, A)
    X = _c2('oqwxLMsEr,tsoLfR->qwxMErtfR', X, O)
    X = _c2('qwxMErtfR,wyrRS->qxMEtfyS', X, T2)
    E = _c2('qxMEtfyS,xEfgy->tqMgS', X, bot6)
    return {'Z00': float(Z00), 'Z10': Z10, 'Z01': Z01, 'Z11': Z11,
            'kappa': Z11 * Z00 / (Z10 * Z01), 'E': E}


def evaluate(A, O_num, O_den, T, chi, max_iter, tol=None, cutoff=1e-12):
    """f = -T (ln kappa_num - ln kappa_den) and g = -2T (E_num/Z11_num - E_den/Z11_den) with the
    reduced method (Sec. II)."""
    num = run(A, O_num, chi, max_iter, tol, cutoff)
    den = run(A, O_den, chi, max_iter, tol, cutoff)
    f = -T * (num['lnk'] - den['lnk'])
    g = -2.0 * T * (num['E'] - den['E'])
    return {'f': f, 'g': g, 'num': num, 'den': den}
