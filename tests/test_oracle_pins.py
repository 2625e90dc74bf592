"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test names the passage of arXiv:2506.19339 (or the external closed form) it checks.  They are
chosen so that a plausible mistake in the oracle -- a dropped term, a swapped leg, a wrong sign,
a transposed operand -- fails at least one of them.
"""
import os

import numpy as np
import pytest

from oracle import bruteforce, ising, onsager, reduced_ctmrg, split_ctmrg as sc
from paper_2506_19339_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), 'golden')


def _rand_env(rng, chi, D, d):
    env = {c: rng.standard_normal((chi, chi)) for c in ('C1', 'C2', 'C3', 'C4')}
    for t in ('T1', 'T2', 'T3', 'T4'):
        env[t] = [rng.standard_normal((chi, chi, m)) for m in (D, d, D)]
    return env


def _rand_problem(seed, chi=3, D=2, d=3, p=2):
    rng = np.random.default_rng(seed)
    O = rng.standard_normal((p, p, d, d, d, d))
    A = rng.standard_normal((p, D, D, D, D))
    B = rng.standard_normal((p, D, D, D, D))
    return _rand_env(rng, chi, D, d), A, O, B


# ---------------------------------------------------------------- V1: model tensors (Sec. II, IV)

def test_sqrt_boltzmann_closed_form():
    """sqrt(W)^2 = W, and the eigendecomposition gives the closed form: eigenvalues 2cosh(beta) on
    (1,1)/sqrt2 and 2sinh(beta) on (1,-1)/sqrt2."""
    for beta in (0.0, 0.1, 1 / 4.5115, 1.0):
        W = ising.boltzmann_matrix(beta)
        Q = ising.sqrt_boltzmann(beta)
        assert np.allclose(Q @ Q, W, rtol=1e-14, atol=1e-14)
        a = (np.sqrt(2 * np.cosh(beta)) + np.sqrt(2 * np.sinh(beta))) / 2
        b = (np.sqrt(2 * np.cosh(beta)) - np.sqrt(2 * np.sinh(beta))) / 2
        assert np.allclose(Q, [[a, b], [b, a]], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize('L', [(2, 2, 2), (2, 2, 3), (1, 3, 2)])
def test_pepo_trace_is_ising_partition_function(L):
    """Eq. "TN for partition function": tTr of the uniform O network equals the enumerated 3D Ising
    partition function on a periodic lattice."""
    beta = 1 / 4.6
    Z_tn = bruteforce.pepo_network_trace(ising.ising_pepo(beta), L)
    Z_bf = bruteforce.ising_Z_enumeration(beta, L)
    assert abs(Z_tn - Z_bf) <= 1e-13 * Z_bf


def test_pepo_symmetries():
    """O is invariant under the full cubic group (Sec. IV): any leg permutation, in particular
    s_up <-> s_dn, which the frames of the split-CTMRG rely on."""
    O = ising.ising_pepo(1 / 4.5)
    for perm in [(1, 0, 2, 3, 4, 5), (0, 1, 3, 2, 5, 4), (2, 3, 0, 1, 5, 4), (5, 4, 3, 2, 1, 0)]:
        assert np.allclose(O, O.transpose(perm), atol=1e-15)


# ---------------------------------------------------------------- V2: network conventions

@pytest.mark.parametrize('Lx,Ly', [(2, 2), (3, 2)])
def test_torus_overlap_equals_reduced_network(Lx, Ly):
    """Eq. "free energy expression": <psi|T|psi> with T built by enumeration from W and sqrt(W)
    equals the tensor trace of the reduced site tensor a = A-bar O A on the same torus; the norm
    <psi|psi> equals the trace of A-bar 1 A."""
    rng = np.random.default_rng(11)
    A = rng.standard_normal((2, 2, 2, 2, 2))
    beta = 1 / 4.5
    psi = bruteforce.peps_torus_amplitudes(A, Lx, Ly)
    Tm = bruteforce.transfer_matrix_torus(beta, Lx, Ly)
    num_bf = psi @ Tm @ psi
    den_bf = psi @ psi
    a = bruteforce.reduced_site_tensor(A, ising.ising_pepo(beta), A)
    a0 = bruteforce.reduced_site_tensor(A, ising.identity_pepo(), A)
    assert abs(bruteforce.torus_trace_site(a, Lx, Ly) - num_bf) <= 1e-12 * abs(num_bf)
    assert abs(bruteforce.torus_trace_site(a0, Lx, Ly) - den_bf) <= 1e-12 * abs(den_bf)


# ---------------------------------------------------------------- V3: split form == fused form

def _fuse(env):
    f = {k: env[k] for k in ('C1', 'C2', 'C3', 'C4')}
    for t in ('T1', 'T2', 'T3', 'T4'):
        k, i, b = env[t]
        F = np.einsum('acx,cey,ebz->abxyz', k, i, b)
        f[t] = F.reshape(F.shape[0], F.shape[1], -1)
    return f


def test_split_local_contractions_equal_fused():
    """Sec. III.A: Z00, Z10, Z01, Z11 and the bra environment E computed with the three split edge
    layers equal the same quantities with the layers fused into one edge tensor and A, O, A-bar
    fused into a (exact identity)."""
    env, A, O, _ = _rand_problem(1, chi=3, D=2, d=3)
    loc = sc.local_contractions(env, A, O, A)
    E = sc.bra_environment(env, loc)
    ref = reduced_ctmrg.local_values(_fuse(env), A, O)
    for k in ('Z00', 'Z10', 'Z01', 'Z11'):
        assert abs(loc[k] - ref[k]) <= 1e-12 * abs(ref[k]), k
    assert np.allclose(E, ref['E'], rtol=1e-11, atol=1e-11 * np.abs(ref['E']).max())


def test_z11_is_the_same_through_every_cut():
    """The full 3x3 network evaluated across the kappa, iota and alpha cuts and from the top."""
    env, A, O, B = _rand_problem(2, chi=5, D=4, d=3)
    loc = sc.local_contractions(env, A, O, B)
    vals = [np.sum(loc['Uk'] * loc['Lk']), np.sum(loc['Ui'] * loc['Li']),
            np.sum(loc['Ua'] * loc['Cbot']), np.sum(loc['Ctop'] * loc['La'])]
    assert np.allclose(vals, vals[0], rtol=1e-12)
    assert abs(np.sum(A * sc.ket_environment(env, loc)) - vals[0]) <= 1e-12 * abs(vals[0])
    assert abs(np.sum(B * sc.bra_environment(env, loc)) - vals[0]) <= 1e-12 * abs(vals[0])


# ---------------------------------------------------------------- frames (the four moves)

def test_frames_relabel_the_same_network():
    """The right / up / down moves are the left move in a relabelled network: Z00 and Z11 are
    unchanged, Z10 and Z01 trade places under the diagonal reflection, and every frame round-trips."""
    env, A, O, B = _rand_problem(3, chi=3, D=2, d=3)
    l0 = sc.local_contractions(env, A, O, B)
    for w in 'LRUD':
        e, a, o, b = sc.to_frame(w, env, A, O, B)
        l1 = sc.local_contractions(e, a, o, b)
        swap = w in 'UD'
        assert abs(l1['Z11'] - l0['Z11']) <= 1e-12 * abs(l0['Z11'])
        assert abs(l1['Z00'] - l0['Z00']) <= 1e-12 * abs(l0['Z00'])
        assert abs(l1['Z10'] - l0['Z01' if swap else 'Z10']) <= 1e-12 * abs(l1['Z10'])
        back = sc.from_frame(w, e)
        for k in ('C1', 'C2', 'C3', 'C4'):
            assert np.array_equal(back[k], env[k])
        for t in ('T1', 'T2', 'T3', 'T4'):
            for i in range(3):
                assert np.array_equal(back[t][i], env[t][i])


# ---------------------------------------------------------------- wiring: exact when nothing is cut

def _absorb_row(X, env, A, O, B):
    """X[v, a, o, b, A, O, B, w] (two columns, open at the bottom) -> one row further down."""
    T4k, T4i, T4b = env['T4']
    T2k, T2i, T2b = env['T2']
    X = sc._c2('vaobPQRw,vxl->xaobPQRwl', X, T4k)
    X = sc._c2('xaobPQRwl,salEr->xobPQRwsEr', X, A)
    X = sc._c2('xobPQRwsEr,SPrFG->xobQRwsESFG', X, A)
    X = sc._c2('xobQRwsESFG,wyG->xobQRsESFy', X, T2k)
    X = sc._c2('xobQRsESFy,xXl->XobQRsESFyl', X, T4i)
    X = sc._c2('XobQRsESFyl,tsolfq->XbQRESFytfq', X, O)
    X = sc._c2('XbQRESFytfq,TSQqgH->XbREFytfTgH', X, O)
    X = sc._c2('XbREFytfTgH,yYH->XbREFtfTgY', X, T2i)
    X = sc._c2('XbREFtfTgY,XZl->bREFtfTgYZl', X, T4b)
    X = sc._c2('bREFtfTgYZl,tblhm->REFfTgYZhm', X, B)
    X = sc._c2('REFfTgYZhm,TRmKn->EFfgYZhKn', X, B)
    X = sc._c2('EFfgYZhKn,YWn->EFfgZhKW', X, T2b)
    return X.transpose(4, 0, 2, 5, 1, 3, 6, 7)


def _two_column_Z(env, A, O, B, rows):
    Ct1, Ct2, Ct3, Ct4 = sc.absorbed_corners(env)
    X = np.einsum('hvpob,hwPQR->vpobPQRw', Ct1, Ct2)
    for _ in range(rows):
        X = _absorb_row(X, env, A, O, B)
    bot = np.einsum('hvpob,hwPQR->vpobPQRw', Ct4, Ct3)
    return float(np.sum(X * bot))


def test_untruncated_projectors_are_exact():
    """Sec. III.C: with every singular value kept, P_T P_B = I and inserting the projectors changes
    no network.  Pins the one-column patches, the two-column patches of every stage-2 projector
    (against a direct row-by-row contraction), and the renormalisation: after an untruncated left
    move the new corners / edges reproduce the old network one column wider
    (Z00' = Z10, Z01' = Z11)."""
    env, A, O, B = _rand_problem(4, chi=2, D=2, d=3)
    halves = sc.one_column_halves(env, A, O, B)
    left, right = sc.stage1_projectors(halves, None, 1e-10)
    for cut, (U, L) in halves.items():
        PB, PT, _ = left[cut]
        k = PT.shape[0]
        P = PT.reshape(k, -1) @ PB.reshape(-1, k)
        kept = np.diag(P) > 0.5
        assert np.allclose(P, np.diag(kept.astype(float)), atol=1e-8)
        assert kept.sum() == min(PB.reshape(-1, k).shape[0], k)
    h2 = sc.two_column_halves(env, A, O, B, left, right)
    z1 = _two_column_Z(env, A, O, B, 1)
    z2 = _two_column_Z(env, A, O, B, 2)
    assert abs(np.sum(h2['kappa'][0] * h2['kappa'][1]) - z1) <= 1e-8 * abs(z1)
    assert abs(np.sum(h2['iota'][0] * h2['iota'][1]) - z1) <= 1e-8 * abs(z1)
    assert abs(np.sum(h2['alpha'][0] * h2['alpha'][1]) - z2) <= 1e-8 * abs(z2)
    old = sc.local_contractions(env, A, O, B)
    C1n, T4n, C4n = sc.left_move(env, A, O, B, None, 1e-10, normalise=False)
    new_env = dict(env)
    new_env.update({'C1': C1n, 'T4': T4n, 'C4': C4n})
    new = sc.local_contractions(new_env, A, O, B)
    assert abs(new['Z00'] - old['Z10']) <= 1e-7 * abs(old['Z10'])
    assert abs(new['Z01'] - old['Z11']) <= 1e-7 * abs(old['Z11'])


# ---------------------------------------------------------------- V4: projector identities

def test_projector_pair_identities():
    """Eqs. "projector construction" and "projector construction 2": P_T P_B = I_chi;
    rho_B P_B = U~ S~^1/2 and P_T rho_T = S~^1/2 V~^T, so rho_B P_B P_T rho_T is the best rank-chi
    approximation of rho_B rho_T (Eckart-Young)."""
    rng = np.random.default_rng(5)
    U = rng.standard_normal((3, 4, 2, 5))
    L = rng.standard_normal((3, 4, 2, 5))
    chi = 6
    PB, PT, S = sc.projector_pair(U, L, (0, 2), chi, 1e-12)
    assert np.allclose(np.einsum('kab,abl->kl', PT, PB), np.eye(chi), atol=1e-10)
    Um = U.transpose(0, 2, 1, 3).reshape(6, 20)
    Lm = L.transpose(0, 2, 1, 3).reshape(6, 20)
    M = Lm.T @ Um
    approx = Lm.T @ PB.reshape(6, chi) @ PT.reshape(chi, 6) @ Um
    u, s, vh = np.linalg.svd(M)
    best = (u[:, :chi] * s[:chi]) @ vh[:chi]
    assert np.allclose(approx, best, atol=1e-10 * s[0])
    assert np.all(S[:-1] >= S[1:])
    # sign gauge: P_B[:, k] = rho_T v_k s_k^-1/2 fixes the sign the oracle gave the pair
    # (u_k, v_k); with that sign the largest-magnitude entry of u_k must be positive
    for k in range(chi):
        sign = np.sign(np.dot(PB.reshape(6, chi)[:, k], Um @ vh[k]))
        uk = sign * u[:, k]
        assert sign != 0 and uk[np.argmax(np.abs(uk))] > 0, k


# ---------------------------------------------------------------- V5 / V6: closed forms

def test_onsager_closed_forms():
    """Onsager: ln z(K_c) = ln(2)/2 + 2G/pi (G Catalan's constant), ln z(0) = ln 2."""
    G = 0.915965594177219015054603514932
    Kc = 0.5 * np.log(1 + np.sqrt(2))
    assert abs(onsager.ln_z_onsager(Kc) - (0.5 * np.log(2) + 2 * G / np.pi)) < 1e-12
    assert abs(onsager.ln_z_onsager(0.0) - np.log(2)) < 1e-15


def test_reduced_ctmrg_plus_state_is_onsager():
    """For the product PEPS |+> the numerator is cosh(beta) x the 2D Ising network (Sec. II with
    D=1), so f = -T[ln cosh(1/T) + ln z_Onsager(1/T)].  Reduced CTMRG, T = 4.6, chi = 16."""
    T = 4.6
    A = inputs.product_plus_peps()
    r = reduced_ctmrg.evaluate(A, ising.ising_pepo(1 / T), ising.identity_pepo(), T, 16, 100, 1e-13)
    assert abs(r['f'] - onsager.f_plus_state(T)) < 1e-10 * abs(r['f'])
    # an independent quadrature value of the same closed form at T = 4.6
    assert abs(onsager.f_plus_state(4.6) - (-3.5226689540075)) < 1e-12


def test_split_ctmrg_plus_state_is_onsager():
    """The same closed form through the split-CTMRG engine.  A product PEPS leaves the kappa / iota
    bonds at rank 2 in this scheme (their patches connect left and right only through the
    boundary and the trivial A / A-bar lines), an error of order the third corner singular value;
    at T = 10 it is far below the tolerance."""
    T = 10.0
    A = inputs.product_plus_peps()
    r = sc.evaluate(A, ising.ising_pepo(1 / T), ising.identity_pepo(), T, 8, 100, 1e-13)
    assert abs(r['f'] - onsager.f_plus_state(T)) < 1e-10 * abs(r['f'])


@pytest.mark.parametrize('D', [1, 2])
def test_infinite_temperature_product_state(D):
    """beta = 0: O has rank 1 in the plane, and for a product PEPS beta*f = -ln 2 exactly."""
    A = inputs.product_plus_peps(D)
    r = sc.evaluate(A, ising.ising_pepo(0.0), ising.identity_pepo(), np.inf, 4, 5, None)
    assert abs(r['beta_f'] + np.log(2)) < 1e-12


# ---------------------------------------------------------------- V7: invariances

def test_free_energy_invariances():
    """f(cA) = f(A) (so <A, g> = 0); f is invariant under an orthogonal gauge transformation of
    the virtual bonds (with the starting environment transformed alike, every step of the
    algorithm is covariant); kappa is invariant under rescaling of any environment tensor."""
    T = 4.6
    O, Oid = ising.ising_pepo(1 / T), ising.identity_pepo()
    A = inputs.perturbed_product_peps(2, 7)
    r0 = sc.evaluate(A, O, Oid, T, 6, 8)
    r1 = sc.evaluate(3.7 * A, O, Oid, T, 6, 8)
    assert abs(r0['f'] - r1['f']) < 1e-10 * abs(r0['f'])
    assert abs(np.sum(A * r0['g'])) < 1e-12 * np.linalg.norm(r0['g'])
    rng = np.random.default_rng(9)
    G = np.linalg.qr(rng.standard_normal((2, 2)))[0]
    H = np.linalg.qr(rng.standard_normal((2, 2)))[0]
    Ag = np.einsum('sulde,uU,lL,dD,eE->sULDE', A, H, G, H, G)
    envs = []
    for d in (2, 1):
        e = sc.init_env(6, 2, d)
        for t, M in (('T1', H), ('T3', H), ('T2', G), ('T4', G)):
            e[t] = [np.einsum('abm,mM->abM', e[t][0], M), e[t][1], np.einsum('abm,mM->abM', e[t][2], M)]
        envs.append(e)
    r2 = sc.evaluate(Ag, O, Oid, T, 6, 8, env_num=envs[0], env_den=envs[1])
    assert abs(r0['f'] - r2['f']) < 1e-10 * abs(r0['f'])
    env, A3, O3, B3 = _rand_problem(6)
    k0 = sc.local_contractions(env, A3, O3, B3)
    env['C2'] = 2.5 * env['C2']
    env['T3'][1] = -0.3 * env['T3'][1]
    k1 = sc.local_contractions(env, A3, O3, B3)
    kap = lambda l: l['Z11'] * l['Z00'] / (l['Z10'] * l['Z01'])
    assert abs(kap(k0) - kap(k1)) < 1e-12 * abs(kap(k0))


# ---------------------------------------------------------------- V8 / V9: reference algorithm, FD

@pytest.mark.slow
def test_split_converges_to_reduced_reference():
    """Sec. IV.A: the split result approaches the reduced method at large chi as chi grows (the
    paper's own accuracy check, with the reduced method as the reference)."""
    T = 4.6
    O, Oid = ising.ising_pepo(1 / T), ising.identity_pepo()
    A = inputs.perturbed_product_peps(2, 7)
    ref = reduced_ctmrg.evaluate(A, O, Oid, T, 48, 100, 1e-11)['f']
    gaps = [abs(sc.evaluate(A, O, Oid, T, chi, 100, 1e-10)['f'] - ref) for chi in (8, 16, 24)]
    assert gaps[0] > gaps[1] > gaps[2]
    assert gaps[2] < 1e-7


def _lnk_fixed_env(env, A, O, B):
    loc = sc.local_contractions(env, A, O, B)
    return loc['Z11'] * loc['Z00'] / (loc['Z10'] * loc['Z01'])


@pytest.mark.parametrize('D,chi,directions', [(2, 5, 'all'), (3, 4, 8), (4, 3, 8)])
def test_env_gradient_is_the_bra_derivative(D, chi, directions):
    """Eq. "gradient expression": g = -2T (E_num / Z11_num - E_den / Z11_den) is twice the
    derivative of f = -T (ln kappa_num - ln kappa_den) with respect to the bra tensor with the
    environments held fixed.  Central differences of f in the bra slot only (the environments
    and the ket A are not touched, so the difference quotient is exact up to O(h^2)) over all
    p D^4 = 32 components at D = 2 and random directions at D = 3, 4, on random environments."""
    T = 4.5
    rng = np.random.default_rng(40 + D)
    A = rng.standard_normal((2,) + (D,) * 4)
    O, Oid = ising.ising_pepo(1 / T), ising.identity_pepo()
    envs = [_rand_env(rng, chi, D, 2), _rand_env(rng, chi, D, 1)]
    for e in envs:  # positive environments keep every kappa positive
        for k in ('C1', 'C2', 'C3', 'C4'):
            e[k] = np.abs(e[k])
        for t in ('T1', 'T2', 'T3', 'T4'):
            e[t] = [np.abs(x) for x in e[t]]
    A = np.abs(A)

    def f_bra(B):
        return -T * (np.log(_lnk_fixed_env(envs[0], A, O, B)) - np.log(_lnk_fixed_env(envs[1], A, Oid, B)))

    Es = []
    Zs = []
    for e, Oo in zip(envs, (O, Oid)):
        loc = sc.local_contractions(e, A, Oo, A)
        Es.append(sc.bra_environment(e, loc))
        Zs.append(loc['Z11'])
    g = -2.0 * T * (Es[0] / Zs[0] - Es[1] / Zs[1])
    if directions == 'all':
        dirs = [np.eye(A.size)[i].reshape(A.shape) for i in range(A.size)]
    else:
        dirs = [rng.standard_normal(A.shape) for _ in range(directions)]
    h = 1e-5
    for v in dirs:
        fd = (f_bra(A + h * v) - f_bra(A - h * v)) / (2 * h)
        # g is twice the bra-slot derivative
        assert abs(2 * fd - np.sum(g * v)) <= 1e-7 * np.linalg.norm(g) * np.linalg.norm(v)


@pytest.mark.slow
def test_fd_reference_and_env_gradient_gap():
    """The finite-difference reference of d f_chi / dA (oracle.split_ctmrg.fd_directional_derivative:
    converged f at A +- h v) vanishes along A (f(cA) = f(A)), and the paper's environment gradient
    approaches it as chi grows (the environment's dependence on A drops out at the exact fixed
    point).  Measured on this input: a gap of ~1.4e-4 at chi = 6 and ~2.4e-6 at chi = 12 (relative
    to |g|)."""
    T = 4.6
    O, Oid = ising.ising_pepo(1 / T), ising.identity_pepo()
    A = inputs.perturbed_product_peps(2, 7)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(A.shape)
    v -= np.sum(v * A) * A / np.sum(A * A)
    v /= np.linalg.norm(v)
    gaps = []
    for chi in (6, 12):
        r = sc.evaluate(A, O, Oid, T, chi, 400, 1e-11)
        fd = sc.fd_directional_derivative(A, O, Oid, T, chi, v, 1e-5, 1e-11, r['num']['env'],
                                          r['den']['env'])
        gaps.append(abs(fd - np.sum(r['g'] * v)) / np.linalg.norm(r['g']))
        if chi == 12:
            along = sc.fd_directional_derivative(A, O, Oid, T, chi, A / np.linalg.norm(A), 1e-5,
                                                 1e-11, r['num']['env'], r['den']['env'])
            assert abs(along) <= 1e-8 * np.linalg.norm(r['g'])
    assert gaps[1] < gaps[0] / 10
    assert gaps[1] < 2e-5


def test_ctm_spectrum_is_a_gauge_invariant_plaquette_product():
    """Sec. III.D: the convergence measure is the spectrum of the product of the four corners
    around the plaquette, normalised by its trace.  Each of the four bonds that join neighbouring
    corners (top, right, bottom, and the left bond where the product is opened) carries an
    arbitrary orthogonal gauge; the spectrum must not depend on any of them, which fixes which leg
    of every corner meets which (a transposed corner or another product order breaks the
    invariance for generic corners).  The same check applied to wrong products (planted mistakes,
    on the CPU only) fails, so the pin has the power to detect them."""
    rng = np.random.default_rng(17)
    chi = 5
    env = {c: rng.standard_normal((chi, chi)) + 3 * np.eye(chi) for c in ('C1', 'C2', 'C3', 'C4')}

    def q():
        return np.linalg.qr(rng.standard_normal((chi, chi)))[0]

    def gauged(e, Gt, Gr, Gb, Gl):
        # C1[h,v]: h top, v left; C2[h,v]: h top, v right; C3[h,v]: h bottom, v right;
        # C4[h,v]: h bottom, v left
        return {'C1': Gt.T @ e['C1'] @ Gl, 'C2': Gt.T @ e['C2'] @ Gr,
                'C3': Gb.T @ e['C3'] @ Gr, 'C4': Gb.T @ e['C4'] @ Gl}

    S0 = sc.ctm_spectrum(env)
    assert np.all(S0[:-1] >= S0[1:]) and abs(np.sum(S0)) > 0
    for _ in range(3):
        S1 = sc.ctm_spectrum(gauged(env, q(), q(), q(), q()))
        assert np.allclose(S1, S0, rtol=1e-12, atol=1e-14)
    wrong = [lambda e: e['C1'] @ e['C2'] @ e['C3'].T @ e['C4'],        # C1 not transposed
             lambda e: e['C1'].T @ e['C2'] @ e['C3'] @ e['C4'],        # C3 not transposed
             lambda e: e['C1'].T @ e['C3'] @ e['C2'].T @ e['C4']]      # corners out of order
    for bad in wrong:
        def spec(e):
            r = bad(e)
            return np.linalg.svd(r / np.trace(r), compute_uv=False)
        moved = max(np.abs(spec(gauged(env, q(), q(), q(), q())) - spec(env)).max() for _ in range(3))
        assert moved > 1e-6


def _composite(pair):
    PB, PT = pair[0], pair[1]
    return np.tensordot(PB, PT, axes=([PB.ndim - 1], [0]))


def test_opposite_move_pairs_are_the_in_move_pairs():
    """Appendix, captions of projectors 4-6: the left move's P^R is the right move's stage-1 pair.
    On one environment of a PEPS without the D2 symmetry (D=2, chi=6, three iterations from the
    cold start) the right move's own stage-1 pairs, mapped by ``opposite_stage1`` (180-degree
    rotation with ket <-> bra: alpha -> alpha, kappa -> iota, iota -> kappa), equal the pairs the
    left move computes for the right column: singular values to 1e-13 of the largest, oblique
    projectors P_B P_T to 1e-10 (the pseudo-inverse square roots amplify rounding).  Mapping the
    kappa pair onto kappa instead fails."""
    T, D, chi = 4.5, 2, 6
    A = inputs.perturbed_product_peps(D, 3, eps=0.3)
    O = ising.ising_pepo(1.0 / T)
    env, *_ = sc.iterate(sc.init_env(chi, D, 2), A, O, A, chi, 3)
    inf_l, inf_r = {}, {}
    sc.move(env, A, O, A, 'L', chi, info=inf_l)
    sc.move(env, A, O, A, 'R', chi, info=inf_r)
    mapped = sc.opposite_stage1(inf_r['left'])
    for cut in ('alpha', 'kappa', 'iota'):
        want = inf_l['right'][cut]
        S, Sm = want[2], mapped[cut][2]
        assert np.max(np.abs(S - Sm)) <= 1e-13 * S[0], cut
        P, Pm = _composite(want), _composite(mapped[cut])
        assert np.linalg.norm(P - Pm) <= 1e-10 * np.linalg.norm(P), cut
    PBk, PTk, _ = inf_r['left']['kappa']
    planted = (PTk.transpose(1, 3, 2, 0), PBk.transpose(3, 0, 2, 1))
    P = _composite(inf_l['right']['kappa'])
    assert np.linalg.norm(P - _composite(planted)) > 1e-3 * np.linalg.norm(P)


def test_paired_moves_are_the_single_moves_of_one_environment():
    """``paired_move`` (left and right moves on one environment, each taking its P^R from the
    other's stage-1 pairs): the tensors each move renormalises are those of that move made alone
    on the same environment with P^R computed in the move, up to the sign gauge of the new bonds
    (the stage-2 SVDs fix their signs from vectors that P^R's own sign gauge enters): equal
    magnitudes (1e-10), and the same gauge-invariant values -- the convergence spectrum and
    ln kappa (1e-12) of the assembled environments; tensors neither move touches are the input's."""
    T, D, chi = 4.5, 2, 6
    A = inputs.perturbed_product_peps(D, 3, eps=0.3)
    O = ising.ising_pepo(1.0 / T)
    env, *_ = sc.iterate(sc.init_env(chi, D, 2), A, O, A, chi, 3)
    for pair in ('LR', 'UD'):
        out = sc.paired_move(env, A, O, A, pair, chi)
        assembled = dict(env)
        for w in pair:
            alone = sc.move(env, A, O, A, w, chi)
            for key in sc.UPDATED[w]:
                assembled[key] = alone[key]
                xs = [alone[key]] if key[0] == 'C' else alone[key]
                ys = [out[key]] if key[0] == 'C' else out[key]
                for x, y in zip(xs, ys):
                    assert np.linalg.norm(np.abs(x) - np.abs(y)) <= 1e-10 * np.linalg.norm(x), key
        S1, S2 = sc.ctm_spectrum(assembled), sc.ctm_spectrum(out)
        assert np.max(np.abs(S1 - S2)) <= 1e-12 * S1[0], pair
        l1 = sc.ln_kappa(sc.local_contractions(assembled, A, O, A))
        l2 = sc.ln_kappa(sc.local_contractions(out, A, O, A))
        assert abs(l1 - l2) <= 1e-12 * abs(l1), pair
        touched = set(sc.UPDATED[pair[0]]) | set(sc.UPDATED[pair[1]])
        for key in ('C1', 'C2', 'C3', 'C4', 'T1', 'T2', 'T3', 'T4'):
            if key not in touched:
                assert out[key] is env[key]


def test_half_p4_perpendicular_pairs_are_the_perpendicular_moves():
    """Appendix, projector 4(b): the half projector 4 renormalises the column cuts of the
    enlarged corners with the up and down moves' P1.  ``perpendicular_alpha_pairs`` computes them
    in the frame of whichever move calls it; on a non-symmetric environment (D=2, chi=6) the pairs
    it finds in the left, right, up and down moves' frames are the (up, down), (down, up),
    (left, right) and (right, left) moves' own stage-1 alpha pairs (oblique projectors 1e-9)."""
    T, D, chi = 4.5, 2, 6
    A = inputs.perturbed_product_peps(D, 3, eps=0.3)
    O = ising.ising_pepo(1.0 / T)
    env, *_ = sc.iterate(sc.init_env(chi, D, 2), A, O, A, chi, 3)
    own = {}
    for w in 'LRUD':
        inf = {}
        sc.move(env, A, O, A, w, chi, info=inf)
        own[w] = _composite(inf['left']['alpha'])
    expect = {'L': 'UD', 'R': 'DU', 'U': 'LR', 'D': 'RL'}
    for w in 'LRUD':
        up, down = sc.perpendicular_alpha_pairs(*sc.to_frame(w, env, A, O, A), chi)
        for got, m in zip((_composite(up), _composite(down)), expect[w]):
            assert np.linalg.norm(got - own[m]) <= 1e-9 * np.linalg.norm(got), (w, m)
            others = [x for x in 'LRUD' if x != m]
            assert all(np.linalg.norm(got - own[x]) > 1e-6 * np.linalg.norm(got) for x in others)


def test_directional_half_p4_is_the_symmetric_one_on_a_symmetric_environment():
    """On a D2-symmetric environment of a D4-symmetric PEPS (D=2, chi=6, four symmetric
    iterations), the directional half projector 4 -- the up and down moves' P1 computed from the
    environment -- is the symmetric scheme's, which takes them from the symmetry: the same
    singular values (1e-13 of the largest) and oblique projector (1e-11)."""
    from oracle import split_ctmrg_d2 as sd
    T, D, chi = 4.5, 2, 6
    A = sd.d4_project(inputs.perturbed_product_peps(D, 3, eps=0.3))
    O = ising.ising_pepo(1.0 / T)
    env = sd.sym_init_env(chi, D, 2)
    for _ in range(4):
        env = sd.sym_iteration(env, A, O, A, chi, p4='half')
    left = sc.stage1_left(env, A, O, A, chi)
    up, down = sc.perpendicular_alpha_pairs(env, A, O, A, chi)
    P_sym = sc.projector_pair(*sc.half_p4_halves(env, A, O, A, left), (0, 1, 2), chi, 1e-12)
    P_dir = sc.projector_pair(*sc.half_p4_halves(env, A, O, A, left, up[1], down[0]), (0, 1, 2),
                              chi, 1e-12)
    assert np.max(np.abs(P_sym[2] - P_dir[2])) <= 1e-13 * P_sym[2][0]
    a, b = _composite(P_sym), _composite(P_dir)
    assert np.linalg.norm(a - b) <= 1e-11 * np.linalg.norm(a)


def test_oracle_flop_counter():
    """The oracle's algorithmic FLOP count: 2 x the product of every distinct label's dimension
    for a pairwise contraction (2 M N K for a matrix product, batch labels included)."""
    rng = np.random.default_rng(1)
    X, Y = rng.standard_normal((3, 4, 5)), rng.standard_normal((5, 4, 6))
    sc.reset_flops()
    sc._c2('abk,kbn->abn', X, Y)      # batch b: 3*4*5*6 multiply-adds
    assert sc.FLOPS['contractions'] == 2 * 3 * 4 * 5 * 6
    sc.reset_flops()
    sc._c2('ak,kn->an', rng.standard_normal((7, 8)), rng.standard_normal((8, 9)))
    assert sc.FLOPS['contractions'] == 2 * 7 * 8 * 9


# ---------------------------------------------------------------- counter-based initialisation

def test_splitmix64_known_answers():
    lines = open(os.path.join(GOLDEN, 'splitmix64_seed0.txt')).read().splitlines()
    vals = [int(x) for x in lines if x.strip() and not x.startswith('#')]
    u = sc.splitmix64_uniform(0, [0, 1])
    assert u[0] == (vals[0] >> 11) * 2.0 ** -53
    assert u[1] == (vals[1] >> 11) * 2.0 ** -53
