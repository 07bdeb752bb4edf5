"""Write the oracle's reference fields for the full-size Rayleigh-Taylor run.

The lattice is 2048 x 8192 (x periodic, walls at y = 0 and y = Ly - 1),
tau 0.8, g = (0, -1e-4), T_top 0.5, T_bot 1.5, seed 1: the benchmark lattice.
It is initialised and stepped by the FP64 CPU oracle (``oracle/``) alone;
nothing here touches the CUDA library.  At each requested step count the
script stores, per field (rho, ux, uy, T):

  * the values at a fixed sample of sites: three full columns (x = 0, Lx/2 - 1,
    Lx - 1: the wrapped edges and the middle, wall rows included), three full
    rows (y = 0, Ly/2, Ly - 1) and 8192 sites drawn uniformly (numpy
    ``default_rng(20170301)``);
  * the mean over x of every row and the mean over y of every column (these
    see every site of the lattice);
  * the lattice-wide maxima that the relative error metric divides by
    (max |rho|, max over both components of |u|, max |T|) and the totals of
    rho, rho ux, rho uy and rho T.

Usage (about 30 min per 100 steps on 8 cores; the runs are resumable through
``--cache``, which holds the full fields of each step count, ~0.5 GB each):

    python tests/golden/make_rt_golden.py --steps 100,1000 --cache DIR

writes ``tests/golden/rt_2048x8192_seed1.npz``.
"""
import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402

LX, LY, SEED = 2048, 8192, 1
PARAMS = dict(tau=0.8, g0=1e-4, T_top=0.5, T_bot=1.5)
SAMPLE_SEED = 20170301
N_RANDOM = 8192


def sample_sites(Lx, Ly):
    """(x, y) int32 arrays of the sampled sites, in a fixed order."""
    xs, ys = [], []
    for x in (0, Lx // 2 - 1, Lx - 1):
        xs.append(np.full(Ly, x))
        ys.append(np.arange(Ly))
    for y in (0, Ly // 2, Ly - 1):
        xs.append(np.arange(Lx))
        ys.append(np.full(Lx, y))
    rng = np.random.default_rng(SAMPLE_SEED)
    xs.append(rng.integers(0, Lx, N_RANDOM))
    ys.append(rng.integers(0, Ly, N_RANDOM))
    return np.concatenate(xs).astype(np.int32), np.concatenate(ys).astype(np.int32)


def summarise(rho, u, T, sx, sy):
    """The stored quantities of one step count (arrays [Lx, Ly], u [2, Lx, Ly])."""
    out = {}
    fields = {"rho": rho, "ux": u[0], "uy": u[1], "T": T}
    for k, v in fields.items():
        out[k + "_sample"] = v[sx, sy]
        out[k + "_rowmean"] = v.mean(axis=0)
        out[k + "_colmean"] = v.mean(axis=1)
    out["max_abs"] = np.array([np.abs(rho).max(), np.abs(u).max(), np.abs(T).max()])
    out["totals"] = np.array([rho.sum(), (rho * u[0]).sum(), (rho * u[1]).sum(), (rho * T).sum()])
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--steps", default="100,1000", help="comma-separated step counts")
    ap.add_argument("--cache", required=True, help="folder for the full fields (not committed)")
    ap.add_argument("--threads", type=int, default=0, help="oracle threads (0: all)")
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                  "rt_%dx%d_seed%d.npz" % (LX, LY, SEED)))
    a = ap.parse_args()
    counts = sorted(int(s) for s in a.steps.split(","))
    os.makedirs(a.cache, exist_ok=True)
    if a.threads:
        oracle.set_threads(a.threads)

    def cached(n):
        return os.path.join(a.cache, "rt_%dx%d_seed%d_step%d.npz" % (LX, LY, SEED, n))

    todo = [n for n in counts if not os.path.exists(cached(n))]
    if todo:
        lat = oracle.Lattice(LX, LY, **PARAMS)
        lat.init_rayleigh_taylor(SEED)
        done = 0
        for n in todo:
            t0 = time.time()
            while done < n:
                k = min(10, n - done)
                lat.run(k)
                done += k
                print("step %d  (%.0f s)" % (done, time.time() - t0), flush=True)
            rho, u, T = lat.fields()
            np.savez(cached(n) + ".tmp.npz", rho=rho, u=u, T=T)
            os.replace(cached(n) + ".tmp.npz", cached(n))
        lat.close()

    sx, sy = sample_sites(LX, LY)
    store = {"Lx": LX, "Ly": LY, "seed": SEED, "steps": np.array(counts), "sample_x": sx, "sample_y": sy,
             "params": np.array([PARAMS["tau"], PARAMS["g0"], PARAMS["T_top"], PARAMS["T_bot"]])}
    for n in counts:
        z = np.load(cached(n))
        for k, v in summarise(z["rho"], z["u"], z["T"], sx, sy).items():
            store["n%d_%s" % (n, k)] = v
    np.savez_compressed(a.out, **store)
    print("wrote", a.out, os.path.getsize(a.out), "bytes")


if __name__ == "__main__":
    main()
