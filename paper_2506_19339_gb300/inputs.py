"""Seeded synthetic inputs shared by the CUDA path's tests / bench and by the CPU oracle.

This module holds no arithmetic of the method: it only draws random numbers.  Every PEPS tensor
used by the tests and the benchmark comes from here, so that the oracle and the GPU path see the
same FP64 values (the GPU never regenerates them).
"""
import numpy as np


def random_peps(D, seed, p=2):
    """A[s,u,l,d,r] with i.i.d. N(0,1) entries (numpy PCG64 stream `seed`), divided by its
    Frobenius norm."""
    A = np.random.default_rng(seed).standard_normal((p, D, D, D, D))
    return A / np.linalg.norm(A)


def perturbed_product_peps(D, seed, eps=0.3, p=2):
    """A near the product state |+> (all virtual indices 0): (|+> delta + eps N(0,1)), normalised.
    For these states the numerator network has a unique dominant boundary and CTMRG converges,
    which a plain N(0,1) tensor does not guarantee."""
    A = eps * np.random.default_rng(seed).standard_normal((p, D, D, D, D))
    A[:, 0, 0, 0, 0] += 1.0 / np.sqrt(p)
    return A / np.linalg.norm(A)


def product_plus_peps(D=1, p=2):
    """The product state |+> embedded at virtual index 0."""
    A = np.zeros((p, D, D, D, D))
    A[:, 0, 0, 0, 0] = 1.0 / np.sqrt(p)
    return A


def temperature_sweep(n=32, lo=4.40, hi=4.62):
    """n temperatures uniform in [lo, hi] (linspace)."""
    return np.linspace(lo, hi, n)


def random_matrix(rows, cols, seed):
    """A (rows x cols) matrix with i.i.d. N(0,1) entries (numpy PCG64 stream `seed`), the operand
    recipe of the plain contraction tests."""
    return np.random.default_rng(seed).standard_normal((rows, cols))
