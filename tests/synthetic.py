"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

Holds no arithmetic of the method: it only draws random numbers.  Anything
the method computes (equilibria, weights, moments) is computed separately on
each side and passed in here as a plain array.
"""
import numpy as np

Q = 37


def random_populations(base, Lx, Ly, seed, rel_noise=0.05):
    """[37, Lx, Ly] float64: base[l] * (1 + rel_noise * (2U - 1)), U uniform.

    ``base`` is any per-population positive scale supplied by the caller."""
    rng = np.random.default_rng(seed)
    base = np.asarray(base, dtype=np.float64).reshape(Q, 1, 1)
    return base * (1.0 + rel_noise * (2.0 * rng.random((Q, Lx, Ly)) - 1.0))


def random_fields(Lx, Ly, seed, rho=(0.5, 2.0), u=0.05, T=(0.5, 1.5)):
    """Random macroscopic fields (rho, ux, uy, T), each [Lx, Ly]."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(rho[0], rho[1], (Lx, Ly))
    ux = rng.uniform(-u, u, (Lx, Ly))
    uy = rng.uniform(-u, u, (Lx, Ly))
    t = rng.uniform(T[0], T[1], (Lx, Ly))
    return r, ux, uy, t


def random_values(n, seed, lo, hi):
    return np.random.default_rng(seed).uniform(lo, hi, n)
