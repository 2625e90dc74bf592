"""Onsager's exact free energy of the 2D Ising model on the square lattice (oracle; test
infrastructure only).  Used as a closed-form pin: for a D=1 product PEPS |+> the triple-layer
network of Sec. II reduces to cosh(beta) times the 2D Ising network at coupling beta.
"""
import numpy as np
from scipy import integrate


def ln_z_onsager(K):
    """ln Z / N of the zero-field 2D Ising model at coupling K (Onsager 1944):
        ln z = ln 2 + 1/(8 pi^2) int int ln[cosh^2 2K - sinh 2K (cos t1 + cos t2)] dt1 dt2,
    with the inner integral done in closed form,
        int_0^{2pi} ln(a - b cos t) dt = 2 pi ln((a + sqrt(a^2 - b^2)) / 2),
    and the outer one by adaptive quadrature."""
    c2 = np.cosh(2.0 * K) ** 2
    s2 = np.sinh(2.0 * K)

    def inner(t1):
        a = c2 - s2 * np.cos(t1)
        b = s2
        return np.log((a + np.sqrt(max(a * a - b * b, 0.0))) / 2.0)

    val, _ = integrate.quad(inner, 0.0, np.pi, epsabs=1e-15, epsrel=1e-15, limit=400)
    return np.log(2.0) + val / (2.0 * np.pi)


def f_plus_state(T):
    """Free-energy density of the D=1 PEPS |+> for the 3D Ising transfer matrix at temperature T:
    f = -T [ln cosh(1/T) + ln z_Onsager(1/T)] (the bra/ket layers contribute cosh(beta) per site
    through sum_s Q[k,s]/sqrt(2) = sqrt(2 cosh beta))."""
    beta = 1.0 / T
    return -T * (np.log(np.cosh(beta)) + ln_z_onsager(beta))
