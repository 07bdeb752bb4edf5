#!/usr/bin/env python3
"""Throughput of the thermal D2Q37 time step on GB300.

One step = pbc + fused propagate/bc/collide over the whole lattice (or the
four separate kernels with --kernel separate).  Default workload: one
2048 x 8192 Rayleigh-Taylor lattice in FP64, populations resident in HBM
(two copies, 2 x 5.0 GB, far larger than the 129 MB L2, so no flush is
needed between steps).  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank advances its own lattice (replicas; weak scaling,
no collective on the data path).  ``--impl reference`` times the CPU oracle
on the host cores instead (rank 0 only).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS per step"
UNIT = "MLUPS"
# algorithmic bytes per site update: 37 populations read + 37 written
BYTES_PER_SITE = {"fp64": 592, "fp32": 296, "fp32-df": 296}
# FP64-pipe instructions per site of the fused FP64 sites kernel (ncu on
# 2048 x 1024: 37 DFMA + 29 integer-to-FP64 conversions; the wall rows' FP64
# sums run in the wall-band kernel, 6 of the bench lattice's 8192 rows)
FP64_PIPE_INST_PER_SITE = 66.0
# FP64 pipe peak from unit counts and clocks: 2 FP64 instructions per SM per
# clock (ncu: ...dfma_pred_on.avg.peak_sustained = 2) x 152 SMs x 2.07 GHz
FP64_PEAK_GINST = 2 * 152 * 2.07
# FP64 flops of one site collision as the oracle writes the method out (its
# counting build, oracle/flop_count.cpp: every operation, and those without an
# operand of exactly 0 or +-1); tests/test_oracle_flops.py keeps these equal
ORACLE_FLOPS_PER_SITE = 42640
ORACLE_NONTRIVIAL_FLOPS_PER_SITE = 17477
# the same counting build applied to the collision with the equilibrium
# contracted by hand into its scalar polynomial, each population on its own
# (oracle/collide_contracted.c): the plain per-site FP64 work of the method,
# the flop term of the roofline min(HBM / bytes, FP64 peak / flops)
ORACLE_CONTRACTED_FLOPS_PER_SITE = 2354
# DRAM bytes per fused launch at 2048 x 8192, scaled by sites from the ncu
# capture of the same kernel on 2048 x 1024 (1223.0 MB per launch there)
FUSED_TRAFFIC_BYTES_2048x8192 = 1223.0e6 * 8
# the same for the FP32-storage double-float kernel, from its capture on
# 2048 x 2048 (1236.2 MB per launch there, with streaming stores)
FUSED32_DF_TRAFFIC_BYTES_2048x8192 = 1236.2e6 * 4


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--kernel", choices=["fused", "separate"], default="fused")
    ap.add_argument("--precision", choices=["fp64", "fp32", "fp32-df"], default="fp64")
    ap.add_argument("--no-precision-forms", dest="precision_forms", action="store_false",
                    help="skip timing the FP32-storage forms after the FP64 step")
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip timing the 64-lattice batched forms")
    ap.add_argument("--batched-steps", type=int, default=500, help="steps of the batched workload (500)")
    ap.add_argument("--batched-lattices", type=int, default=64,
                    help="lattices in the batched form (64 is the workload; fewer make a small profiling case)")
    ap.add_argument("--serving-jobs", type=int, default=40, help="0 skips the serving run")
    ap.add_argument("--serving-budget-gb", type=float, default=96.0)
    ap.add_argument("--serving-steps-per-tick", type=int, default=16)
    ap.add_argument("--serving-time-limit", type=float, default=90.0)
    ap.add_argument("--no-accuracy", dest="accuracy", action="store_false",
                    help="skip the comparison with the oracle's stored fields")
    ap.add_argument("--Lx", type=int, default=2048)
    ap.add_argument("--Ly", type=int, default=8192)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="CPU-baseline sample length")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def replica_seed(rank):
    """Each rank advances its own lattice (replicas): a different seed per rank."""
    return 1 + rank


def max_over_ranks(torch, dist, ms, device):
    """The slowest rank's timed region (ms); the value alone without ranks."""
    if not dist:
        return ms
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(sites_per_rank, world, steps, ms):
    """Site updates of all ranks over the slowest rank's time, in millions per second."""
    return sites_per_rank * world * steps / (ms * 1e-3) / 1e6


def workload_name(a):
    return "rayleigh_taylor_fp64_%dx%d" % (a.Lx, a.Ly)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


# --------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and parts[0] != self.uuid:
                continue
            rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


# ---------------------------------------------------------------- CPU oracle

def oracle_mlups(Lx, Ly, seconds, max_steps=None):
    """Time full oracle steps on an Lx x Ly Rayleigh-Taylor lattice."""
    import oracle
    lat = oracle.Lattice(Lx, Ly, tau=0.8, g0=1e-4, T_top=0.5, T_bot=1.5)
    lat.init_rayleigh_taylor(1)
    steps, t0 = 0, time.perf_counter()
    while True:
        lat.run(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds or (max_steps and steps >= max_steps):
            break
    lat.close()
    return Lx * Ly * steps / el / 1e6, steps, el, oracle.threads()


def cpu_baseline(a):
    import oracle
    Ly = max(6, a.Ly // 8)
    v, steps, el, cores = oracle_mlups(a.Lx, Ly, a.cpu_seconds)
    out = {"value": round(v, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "%d full oracle steps (pbc+propagate+bc+collide, FP64) of a %dx%d Rayleigh-Taylor lattice "
                     "(1/8 of the %dx%d workload's rows), %.1f s" % (steps, a.Lx, Ly, a.Lx, a.Ly, el)}
    # the same on one core, and the 256 x 128 parity case on all cores and on one,
    # each a bounded sample (a few seconds)
    c1 = {}
    for n in (cores, 1):
        oracle.set_threads(n)
        v1, s1, e1, _ = oracle_mlups(256, 128, min(a.cpu_seconds, 3.0), max_steps=100)
        c1["ms_per_step_%d_cores" % n] = round(e1 / s1 * 1e3, 3)
        if n == 1:
            vs, ss, es, _ = oracle_mlups(a.Lx, max(6, a.Ly // 512), min(a.cpu_seconds, 3.0))
            out["single_core"] = {"value": round(vs, 4), "unit": UNIT, "sample": "%d steps of a %dx%d strip, %.1f s"
                                  % (ss, a.Lx, max(6, a.Ly // 512), es)}
    oracle.set_threads(cores)
    out["c1_256x128"] = c1
    return out


def run_reference(a):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle
    Ly = 64  # a bounded sample of the workload per step: full width, 64 rows
    lat = oracle.Lattice(a.Lx, Ly, tau=0.8, g0=1e-4, T_top=0.5, T_bot=1.5)
    lat.init_rayleigh_taylor(1)
    lat.run(a.warmup)
    t0 = time.perf_counter()
    lat.run(a.steps)
    el = time.perf_counter() - t0
    v = a.Lx * Ly * a.steps / el / 1e6
    cores = oracle.threads()
    sample = "each step: one full oracle step (FP64, pbc+propagate+bc+collide) of a %dx%d strip of the %dx%d " \
             "Rayleigh-Taylor workload" % (a.Lx, Ly, a.Lx, a.Ly)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(el / a.steps * 1e3, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "Lx": a.Lx, "Ly": a.Ly, "sample_Ly": Ly},
            "cpu_baseline": {"value": round(v, 4), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": round(v, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------- GPU arm

DTYPES = {"fp64": "f64", "fp32": "f32 storage + f64 wide terms", "fp32-df": "f32 storage + double-float wide terms"}


def roofline_of(kind, avg_s, sites, precision, traffic=None):
    """Roofline entry of the dominant kernel: the HBM bound (algorithmic bytes
    per site over the measured copy bandwidth).  For the FP64 form the FP64
    pipe's share is given beside it (FP64-pipe instructions per site counted
    by ncu on the same kernel)."""
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    nbytes = (BYTES_PER_SITE[precision] if kind in ("fused", "propagate", "collide") else 0) * sites
    achieved = nbytes / avg_s / 1e9
    r = {"bound": "hbm", "kernel": kind, "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
         "frac": round(achieved / hbm_peak, 4) if hbm_peak else None, "traffic": traffic,
         "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
         "algorithmic_bytes_per_launch": nbytes}
    if precision == "fp64" and kind in ("fused", "collide"):
        # the roofline min(HBM / bytes, FP64 peak / flops), both terms: the
        # FP64 work of the method written plainly (hand-contracted equilibrium,
        # per population) bounds an FP64 evaluation far below the HBM term;
        # this step escapes it by doing its moment sums and equilibrium on the
        # integer pipes (66 FP64-pipe instructions per site: the relaxation's
        # FMAs and conversions), so the HBM term is the one that applies
        peak_flops = 2 * FP64_PEAK_GINST * 1e9
        hbm_bound = hbm_peak * 1e9 / BYTES_PER_SITE[precision] / 1e9 if hbm_peak else None
        flop_bound = peak_flops / ORACLE_CONTRACTED_FLOPS_PER_SITE / 1e9
        r["bounds"] = {
            "hbm_gsites_per_s": round(hbm_bound, 3) if hbm_bound else None,
            "hbm_derivation": "%s GB/s / %d B per site" % (hbm_peak, BYTES_PER_SITE[precision]),
            "fp64_flop_gsites_per_s": round(flop_bound, 4),
            "fp64_flop_derivation": "%.3f TFLOP/s FP64 peak / %d FP64 flops per site (oracle counting build, "
                                    "hand-contracted equilibrium)" % (peak_flops / 1e12,
                                                                       ORACLE_CONTRACTED_FLOPS_PER_SITE),
            "min_gsites_per_s": round(min(hbm_bound, flop_bound), 4) if hbm_bound else None,
            "achieved_gsites_per_s": round(sites / avg_s / 1e9, 4),
            "applies": "hbm: the kernel's equilibrium and moment sums run on the integer pipes, not as FP64 flops"}
        r["oracle_flops"] = {"contracted_flops_per_site": ORACLE_CONTRACTED_FLOPS_PER_SITE,
                             "tensor_form_flops_per_site": ORACLE_FLOPS_PER_SITE,
                             "tensor_form_nontrivial_flops_per_site": ORACLE_NONTRIVIAL_FLOPS_PER_SITE,
                             "fp64_peak_tflops": round(peak_flops / 1e12, 3)}
        ginst = FP64_PIPE_INST_PER_SITE * sites / avg_s / 1e9
        r["fp64_pipe"] = {"inst_per_site": FP64_PIPE_INST_PER_SITE, "achieved": round(ginst, 2),
                          "peak": round(FP64_PEAK_GINST, 2), "unit": "G FP64-pipe instructions/s",
                          "frac": round(ginst / FP64_PEAK_GINST, 4),
                          "peak_source": "derived: 2 FP64-pipe instructions/clk/SM x 152 SMs x 2.07 GHz"}
    r["avg_launch_ms"] = round(avg_s * 1e3, 4)  # per call of the step's launcher (one step)
    return r


def time_form(torch, lbm, a, dev, precision, kernel, steps, seed, dist=None, sampler=None):
    """Advance one lattice `steps` steps between CUDA events on its stream; per
    kernel event pairs from the library give the dominant kernel's launch time."""
    stream = torch.cuda.Stream(device=dev)  # a capturable stream of the lattice's own
    lat = lbm.Lattice(a.Lx, a.Ly, tau=0.8, g0=1e-4, T_top=0.5, T_bot=1.5, kernel=kernel, device=dev,
                      stream=stream, precision=precision)
    lat.init_rayleigh_taylor(seed)
    for _ in range(a.warmup):
        lat.step(1)
    lat.synchronize()
    lat.set_timing(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    if sampler:
        sampler.start()
        time.sleep(0.3)  # let nvidia-smi take its first samples
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = lat.launch_count
    e0.record(lat.stream)
    for _ in range(steps):
        lat.step(1)
    e1.record(lat.stream)
    e1.synchronize()
    torch.cuda.synchronize(dev)
    launches = lat.launch_count - n0
    ms = e0.elapsed_time(e1)
    if dist:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    kt = lat.kernel_times()
    lat.set_timing(False)
    return lat, ms, launches, kt, clocks


def separate_form(torch, lbm, a, dev):
    """The FP64 step as separate kernels (pbc, propagate, bc, collide) on the
    same workload: the propagate moves 592 B/site and the in-place collide
    another 592, so the schedule moves 1184 B/site; the HBM fraction is given
    against both 592 (the fused step's bytes) and 1184."""
    steps = max(1, min(a.steps, 100))
    lat, ms, launches, kt, _ = time_form(torch, lbm, a, dev, "fp64", "separate", steps, 1)
    lat.close()
    sites = a.Lx * a.Ly
    peak = measured_peaks().get("hbm_gbs")
    s_per_step = ms * 1e-3 / steps
    out = {"value": round(sites / s_per_step / 1e6, 3), "unit": UNIT, "ms_per_step": round(ms / steps, 4),
           "steps": steps, "gpu_launches": launches,
           "kernel_ms_per_launch": {k: round(v[0] / v[1], 4) for k, v in kt.items() if v[1]},
           "hbm": {"peak_gbs": peak, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}}
    for nbytes in (592, 1184):
        gbs = nbytes * sites / s_per_step / 1e9
        out["hbm"]["achieved_gbs_at_%d_B_per_site" % nbytes] = round(gbs, 1)
        out["hbm"]["frac_at_%d_B_per_site" % nbytes] = round(gbs / peak, 4) if peak else None
    if "propagate" in kt and kt["propagate"][1]:
        gbs = 592 * sites / (kt["propagate"][0] / kt["propagate"][1] * 1e-3) / 1e9
        out["propagate_kernel"] = {"achieved_gbs": round(gbs, 1), "frac": round(gbs / peak, 4) if peak else None}
    return out


def run_batched(torch, lbm, a, dev):
    """a.batched_lattices (64) uneven Rayleigh-Taylor lattices advanced together (graph-replayed),
    launch shape from the autotuner, and every shape beside it: one launch per step with
    block_y rows per tile, or one launch per lattice; FP64 and FP32 storage."""
    from paper_1703_00185_gb300 import workloads
    jobs = workloads.batched_lattices(1, a.batched_lattices)
    sites = sum(j["Lx"] * j["Ly"] for j in jobs)
    out = {"workload": "%d Rayleigh-Taylor lattices, Lx in {128..1024 step 128}, Ly in {256..2048 step 256}, "
                       "per-lattice seed and T_bot ~ U(1.2, 1.8) from master seed 1" % a.batched_lattices,
           "sites": sites}
    for prec in ("fp64", "fp32-df"):
        lats = []
        for j in jobs:
            lat = lbm.Lattice(j["Lx"], j["Ly"], tau=0.8, g0=1e-4, T_top=0.5, T_bot=j["T_bot"], device=dev,
                              precision=prec)
            lat.init_rayleigh_taylor(j["seed"])
            lats.append(lat)
        b = lbm.Batch(lats)
        tune = b.autotune(trial_steps=3, use_cache=False)

        def timed(steps):
            b.step(a.warmup)
            b.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            n0 = b.launch_count
            e0.record(b.stream)
            b.step(steps)
            e1.record(b.stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            return {"value": round(sites * steps / (ms * 1e-3) / 1e6, 3), "unit": UNIT,
                    "ms_per_step": round(ms / steps, 4), "steps": steps,
                    "gpu_launches": b.launch_count - n0,
                    "hbm_frac": round(BYTES_PER_SITE[prec] * sites * steps / (ms * 1e-3) / 1e9 /
                                      measured_peaks().get("hbm_gbs", float("nan")), 4)}

        out[prec] = dict(timed(a.batched_steps), launch_shape=tune)
        # every shape beside the autotuner's pick (100 steps each): one launch
        # per step (block_y rows per tile, one block per tile), and one launch
        # per lattice
        shapes = {}
        for by, bps in ((64, 0), (128, 0), (256, 0), (0, 0)):
            b.set_config(by, bps)
            shapes["block_y=%d" % by if by else "per_lattice"] = timed(min(100, a.batched_steps))
        b.set_config(tune["block_y"], tune["blocks_per_sm"])
        out[prec]["shapes"] = shapes
        b.close()
        for lat in lats:
            lat.close()
        torch.cuda.empty_cache()
    return out


def run_serving(a, dev):
    """The serving form: a finite Poisson trace at the configured rate (the
    first `serving_jobs` arrivals), plus lower rates on jobs of 1/4 the linear
    size, replayed in wall-clock time through the continuous-batching server."""
    from paper_1703_00185_gb300 import serving, workloads
    budget = int(a.serving_budget_gb * 2 ** 30)
    runs = {}
    trace = workloads.serving_trace(1, rate=50.0, n_jobs=a.serving_jobs)
    runs["rate50_full_size"] = serving.run_trace(trace, budget, a.serving_steps_per_tick, dev,
                                                 time_limit=a.serving_time_limit)
    # full-size jobs at a rate the GPU sustains (about 1.4e9 site updates per job)
    trace = workloads.serving_trace(3, rate=2.0, n_jobs=a.serving_jobs)
    runs["rate2_full_size"] = serving.run_trace(trace, budget, a.serving_steps_per_tick, dev,
                                                time_limit=a.serving_time_limit)
    for rate in (20.0, 5.0):
        trace = workloads.serving_trace(2, rate=rate, n_jobs=a.serving_jobs, size_scale=0.25)
        runs["rate%g_quarter_size" % rate] = serving.run_trace(trace, budget, a.serving_steps_per_tick, dev,
                                                               time_limit=a.serving_time_limit)
    return {"workload": "Poisson arrivals (seeded), Lx log-uniform [64, 2048], Ly log-uniform [64, 4096] "
                        "(multiples of 8; quarter-size runs divide both by 4), steps U(100, 5000), precision "
                        "50/50 FP64 or FP32 storage (double-float wide terms)",
            "budget_gb": a.serving_budget_gb, "max_steps_per_tick": a.serving_steps_per_tick, "runs": runs}


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "rt_2048x8192_seed1.npz")


def oracle_errors(rho, u, T, z, n):
    """Errors of one state against the oracle's stored fields after n steps:
    per field max |a - b| / max |b| (u over both components) on the stored
    sites and on the row and column means, and the relative L2 error over the
    stored sites."""
    sx, sy = z["sample_x"], z["sample_y"]
    mx = z["n%d_max_abs" % n]
    vals = {"rho": rho, "ux": u[0], "uy": u[1], "T": T}
    scale = {"rho": mx[0], "ux": mx[1], "uy": mx[1], "T": mx[2]}
    err, l2n, l2d = {}, {}, {}
    for k, v in vals.items():
        ref = z["n%d_%s_sample" % (n, k)]
        got = v[sx, sy]
        err[k] = max(np.abs(got - ref).max(), np.abs(v.mean(axis=0) - z["n%d_%s_rowmean" % (n, k)]).max(),
                     np.abs(v.mean(axis=1) - z["n%d_%s_colmean" % (n, k)]).max()) / scale[k]
        l2n[k], l2d[k] = ((got - ref) ** 2).sum(), (ref ** 2).sum()
    return {"max_rel": {"rho": float(err["rho"]), "u": float(max(err["ux"], err["uy"])), "T": float(err["T"])},
            "rel_l2_sample": {"rho": float(np.sqrt(l2n["rho"] / l2d["rho"])),
                              "u": float(np.sqrt((l2n["ux"] + l2n["uy"]) / (l2d["ux"] + l2d["uy"]))),
                              "T": float(np.sqrt(l2n["T"] / l2d["T"]))}}


def accuracy_vs_oracle(torch, lbm, a, dev):
    """Every precision form of the 2048 x 8192 workload (seed 1) stepped to the
    step counts of the oracle's stored fields (tests/golden, written by a
    script that runs only the oracle) and compared with them."""
    if (a.Lx, a.Ly) != (2048, 8192) or not os.path.exists(GOLDEN):
        return {}
    z = np.load(GOLDEN)
    counts = sorted(int(n) for n in z["steps"])
    out = {}
    for prec in ("fp64", "fp32", "fp32-df"):
        lat = lbm.Lattice(a.Lx, a.Ly, tau=0.8, g0=1e-4, T_top=0.5, T_bot=1.5, kernel="fused", precision=prec,
                          device=dev, stream=torch.cuda.Stream(device=dev))
        lat.init_rayleigh_taylor(1)
        done, res = 0, {}
        for n in counts:
            lat.step(n - done)
            done = n
            res["after_%d_steps" % n] = oracle_errors(*lat.fields(), z, n)
        lat.close()
        out[prec] = dict(res, oracle="FP64 CPU oracle, 2048x8192 seed 1: 8192 uniform sites, 3 full columns, "
                                     "3 full rows, all row and column means")
    return out


def run_ours(a):
    rank, local_rank, world = dist_env()
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline(a)  # before any CUDA work in this process
    import torch
    import paper_1703_00185_gb300 as lbm
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    sites = a.Lx * a.Ly
    uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    sampler = ClockSampler("GPU-" + str(uuid) if uuid is not None else None)
    lat, ms, launches, kt, clocks = time_form(torch, lbm, a, dev, a.precision, a.kernel, a.steps,
                                              replica_seed(rank), dist, sampler)
    ms = max_over_ranks(torch, dist, ms, dev)
    ms_per_step = ms / a.steps
    value = whole_job_mlups(sites, world, a.steps, ms)
    kind = max(kt, key=lambda k: kt[k][0])
    traffic = FUSED_TRAFFIC_BYTES_2048x8192 if (kind == "fused" and a.precision == "fp64" and
                                                 (a.Lx, a.Ly) == (2048, 8192)) else None
    # per step: the library times each launcher call, and the fused FP64 step is
    # two kernels (the sites, then the wall-band rows of walled lattices)
    roofline = roofline_of(kind, kt[kind][0] / a.steps * 1e-3, sites, a.precision, traffic)
    roofline["kernels_per_step"] = round(kt[kind][1] / a.steps, 3)

    # end to end through the C ABI with pinned host buffers: upload state, one step, read fields
    e2e = None
    if a.e2e_steps > 0:
        f_host = torch.empty((37, a.Lx, a.Ly), dtype=torch.float64, pin_memory=True)
        lat.populations(out=f_host.numpy())
        rho = torch.empty((a.Lx, a.Ly), dtype=torch.float64, pin_memory=True)
        u = torch.empty((2, a.Lx, a.Ly), dtype=torch.float64, pin_memory=True)
        T = torch.empty((a.Lx, a.Ly), dtype=torch.float64, pin_memory=True)
        lat.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.e2e_steps):
            lat.set_populations(f_host)
            lat.step(1)
            lat.fields(out=(rho, u, T))
        el = time.perf_counter() - t0
        e2e = {"value": round(sites * world * a.e2e_steps / el / 1e6, 3), "unit": UNIT,
               "h2d_bytes_per_step": f_host.numel() * 8,
               "d2h_bytes_per_step": (rho.numel() + u.numel() + T.numel()) * 8,
               "steps": a.e2e_steps}
    lat.close()

    # errors against the FP64 CPU oracle's stored fields of this workload (seed 1)
    accuracy = accuracy_vs_oracle(torch, lbm, a, dev) if (rank == 0 and world == 1 and a.accuracy) else {}
    # the FP32-storage forms on the same workload
    forms = {}
    if a.precision_forms and a.precision == "fp64":
        for prec in ("fp32", "fp32-df"):
            flat, fms, fl, fkt, _ = time_form(torch, lbm, a, dev, prec, "fused", a.steps, 1 + rank)
            flat.close()
            fkind = max(fkt, key=lambda k: fkt[k][0])
            forms[prec] = {"value": round(sites * a.steps / (fms * 1e-3) / 1e6, 3), "unit": UNIT,
                           "ms_per_step": round(fms / a.steps, 4), "dtype": DTYPES[prec],
                           "roofline": roofline_of(fkind, fkt[fkind][0] / a.steps * 1e-3, sites, prec,
                                                   FUSED32_DF_TRAFFIC_BYTES_2048x8192
                                                   if (fkind == "fused" and prec == "fp32-df" and
                                                       (a.Lx, a.Ly) == (2048, 8192)) else None),
                           "vs_oracle": accuracy.get(prec), "gpu_launches": fl}
    separate = separate_form(torch, lbm, a, dev) if (a.precision_forms and a.precision == "fp64" and
                                                     a.kernel == "fused") else None
    batched = run_batched(torch, lbm, a, dev) if (a.batched and a.precision == "fp64") else None
    serving_summary = run_serving(a, dev) if (a.serving_jobs > 0 and a.precision == "fp64") else None
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[a.precision], "data": "synthetic",
                "config": {"workload": workload_name(a), "Lx": a.Lx, "Ly": a.Ly, "kernel": a.kernel,
                           "precision": a.precision, "tau": 0.8, "g0": 1e-4, "T_top": 0.5, "T_bot": 1.5,
                           "seed": "1 + rank",
                           "l2": "no flush: inputs exceed L2 (2 x %.2f GB population copies vs 129 MB)" %
                                 (37 * (a.Lx + 6) * (a.Ly + 32) * (8 if a.precision == "fp64" else 4) / 1e9),
                           "parallelism": "replicas" if world > 1 else "single"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "vs_oracle": accuracy.get(a.precision),
                "kernel_ms": {k: round(v[0], 3) for k, v in kt.items() if v[1]}, "clocks": clocks,
                "precision_forms": forms or None, "separate_form": separate, "batched_forms": batched, "serving": serving_summary}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
