"""Seeded synthetic workloads: lattice sizes, seeds and parameters only.

Nothing here computes any part of the method; it draws the job mixes that
stand in for the paper's Rayleigh-Taylor production runs.
"""
import numpy as np


def batched_lattices(master_seed=1, n=64):
    """n independent Rayleigh-Taylor lattices: Lx uniform on {128, ..., 1024}
    (step 128), Ly uniform on {256, ..., 2048} (step 256), per-lattice seed and
    bottom temperature T_bot ~ U(1.2, 1.8).  Returns a list of dicts."""
    rng = np.random.default_rng(master_seed)
    Lx = rng.choice(np.arange(128, 1025, 128), n)
    Ly = rng.choice(np.arange(256, 2049, 256), n)
    seeds = rng.integers(1, 2 ** 31, n)
    T_bot = rng.uniform(1.2, 1.8, n)
    return [{"Lx": int(Lx[i]), "Ly": int(Ly[i]), "seed": int(seeds[i]), "T_bot": float(T_bot[i])}
            for i in range(n)]


def serving_trace(master_seed=1, rate=50.0, n_jobs=300, size_scale=1.0, steps=(100, 5000)):
    """Poisson arrivals at `rate` jobs/s: Lx log-uniform on [64, 2048], Ly
    log-uniform on [64, 4096] (both rounded to multiples of 8, then scaled by
    `size_scale` and re-rounded), steps uniform on `steps`, precision FP64 or
    FP32 storage with probability 1/2 each, per-job seed and T_bot ~ U(1.2, 1.8).
    Returns a list of dicts sorted by arrival time (seconds from 0)."""
    rng = np.random.default_rng(master_seed)
    gaps = rng.exponential(1.0 / rate, n_jobs)
    t = np.cumsum(gaps) - gaps[0]

    def logu(lo, hi):
        v = np.exp(rng.uniform(np.log(lo), np.log(hi), n_jobs)) * size_scale
        return np.maximum(8, np.round(v / 8) * 8).astype(int)

    Lx, Ly = logu(64, 2048), logu(64, 4096)
    st = rng.integers(steps[0], steps[1] + 1, n_jobs)
    prec = np.where(rng.random(n_jobs) < 0.5, "fp64", "fp32-df")
    seeds = rng.integers(1, 2 ** 31, n_jobs)
    T_bot = rng.uniform(1.2, 1.8, n_jobs)
    return [{"id": i, "arrival": float(t[i]), "Lx": int(Lx[i]), "Ly": int(Ly[i]), "steps": int(st[i]),
             "precision": str(prec[i]), "seed": int(seeds[i]), "T_bot": float(T_bot[i])} for i in range(n_jobs)]
