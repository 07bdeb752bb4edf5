"""Full-size parity: the 2048 x 8192 benchmark lattice (seed 1, tau 0.8,
g0 1e-4, T_top 0.5, T_bot 1.5) against the FP64 CPU oracle, after 100 and
1000 steps, in the fused schedule bench.py times.

The oracle's side was computed once by ``tests/golden/make_rt_golden.py``,
which runs only ``oracle/``, and is stored in
``tests/golden/rt_2048x8192_seed1.npz``: the fields at three full columns
(the wrapped edges and the middle, wall rows included), three full rows and
8192 uniformly drawn sites, the mean of every row and of every column, the
lattice-wide maxima and the totals.

Metric (as everywhere in the FP64 tests): per field, max |a - b| / max |b|
over the lattice (u over both components jointly), evaluated on the stored
sites and on the row and column means.  Bars:
  * FP64, 100 and 1000 steps: 1e-12, the tolerance of the full FP64 step
    (measured after 1000 steps: rho 1.8e-13, u 2.3e-13, T 1.6e-13; the
    unstable Rayleigh-Taylor flow amplifies rounding differences in time, and
    the 1000-step run was only required to stay within 1e-10);
  * FP32 storage: relative L2 error over the stored sites, at the bars of the
    256 x 128 accuracy tests (measured errors times about 10).
"""
import os

import numpy as np
import pytest

import paper_1703_00185_gb300 as lbm

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rt_2048x8192_seed1.npz")
FP64_BARS = {100: 1e-12, 1000: 1e-12}
FP32_L2_BARS = {100: (2e-7, 5e-5, 2e-7), 1000: (1e-6, 1e-4, 1e-6)}


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_00185_gb300 import _build
    _build.build()
    lbm.load_library()


@pytest.fixture(scope="module")
def golden():
    return np.load(GOLDEN)


def field_errors(rho, u, T, z, n):
    """(rho, u, T) errors, max |a - b| / max |b|, over the stored sites and the
    row and column means of step count n."""
    sx, sy = z["sample_x"], z["sample_y"]
    vals = {"rho": rho, "ux": u[0], "uy": u[1], "T": T}
    mx = z["n%d_max_abs" % n]
    scale = {"rho": mx[0], "ux": mx[1], "uy": mx[1], "T": mx[2]}
    err = {}
    for k, v in vals.items():
        e = max(np.abs(v[sx, sy] - z["n%d_%s_sample" % (n, k)]).max(),
                np.abs(v.mean(axis=0) - z["n%d_%s_rowmean" % (n, k)]).max(),
                np.abs(v.mean(axis=1) - z["n%d_%s_colmean" % (n, k)]).max())
        err[k] = float(e / scale[k])
    return err["rho"], max(err["ux"], err["uy"]), err["T"]


def sample_rel_l2(rho, u, T, z, n):
    sx, sy = z["sample_x"], z["sample_y"]
    out = []
    for got, keys in ((rho[sx, sy], ["rho"]), (np.stack([u[0][sx, sy], u[1][sx, sy]]), ["ux", "uy"]),
                      (T[sx, sy], ["T"])):
        ref = np.stack([z["n%d_%s_sample" % (n, k)] for k in keys]).reshape(got.shape)
        out.append(float(np.sqrt(((got - ref) ** 2).sum() / (ref ** 2).sum())))
    return tuple(out)


def stored(bars, golden):
    """The step counts of `bars` that the stored oracle fields hold."""
    have = set(int(n) for n in golden["steps"])
    return {n: b for n, b in bars.items() if n in have}


def run(precision, steps):
    import torch
    lat = lbm.Lattice(2048, 8192, tau=0.8, g0=1e-4, T_top=0.5, T_bot=1.5, kernel="fused", precision=precision,
                      device="cuda:0", stream=torch.cuda.Stream(device="cuda:0"))
    lat.init_rayleigh_taylor(1)
    out, done = {}, 0
    for n in steps:
        lat.step(n - done)
        done = n
        out[n] = lat.fields()
    lat.close()
    return out


def test_golden_is_the_benchmark_lattice(golden):
    assert (int(golden["Lx"]), int(golden["Ly"]), int(golden["seed"])) == (2048, 8192, 1)
    assert np.array_equal(golden["params"], [0.8, 1e-4, 0.5, 1.5])
    assert sorted(golden["steps"].tolist()) == [100, 1000]


def test_fp64_full_size_against_oracle(golden):
    bars = stored(FP64_BARS, golden)
    fields = run("fp64", sorted(bars))
    for n, bar in bars.items():
        rho, u, T = fields[n]
        errs = field_errors(rho, u, T, golden, n)
        assert max(errs) <= bar, (n, errs)
        tot = golden["n%d_totals" % n]
        assert abs(rho.sum() - tot[0]) / tot[0] < 1e-12  # mass


@pytest.mark.parametrize("precision", ["fp32", "fp32-df"])
def test_fp32_full_size_against_oracle(precision, golden):
    todo = stored(FP32_L2_BARS, golden)
    fields = run(precision, sorted(todo))
    for n, bars in todo.items():
        errs = sample_rel_l2(*fields[n], golden, n)
        assert all(e <= b for e, b in zip(errs, bars)), (n, errs)
