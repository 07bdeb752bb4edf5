"""Continuous-batching simulation service on top of the ``lbm_server_*`` C ABI.

:class:`Server` is a thin wrapper (argument marshalling only); admission,
memory pool, batched stepping and result copies are native.  :func:`run_trace`
replays a timed job trace (e.g. ``workloads.serving_trace``) in wall-clock
time: jobs are submitted when their arrival time has passed, the server ticks
continuously, and completion times give per-job latency.
"""
import collections
import ctypes
import time

import numpy as np

from . import (JOB_DONE, LBMError, PRECISIONS, _check, lbm_default_params, lbm_server_stats,
               load_library)


class Server:
    def __init__(self, budget_bytes, max_steps_per_tick=16, device=None):
        import torch
        self._torch = torch
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        lib = load_library()
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib.lbm_server_create(int(budget_bytes), int(max_steps_per_tick), ctypes.byref(h)),
                   "lbm_server_create")
        self._h = h
        self.sizes = {}

    def _dev(self):
        return self._torch.cuda.device(self.device)

    def submit(self, Lx, Ly, steps, precision="fp64", seed=1, tau=0.8, g0=1e-4, T_top=0.5, T_bot=1.5):
        p = lbm_default_params()
        p.tau, p.g0, p.T_top, p.T_bot = tau, g0, T_top, T_bot
        p.precision = PRECISIONS[precision]
        jid = ctypes.c_int64()
        _check(load_library().lbm_server_submit(self._h, Lx, Ly, steps, ctypes.byref(p), seed, ctypes.byref(jid)),
               "lbm_server_submit")
        self.sizes[jid.value] = (Lx, Ly)
        return jid.value

    def tick(self):
        k = ctypes.c_int()
        with self._dev():
            _check(load_library().lbm_server_tick(self._h, ctypes.byref(k)), "lbm_server_tick")
        return k.value

    def poll(self, max_ids=4096):
        ids = (ctypes.c_int64 * max_ids)()
        n = ctypes.c_int()
        _check(load_library().lbm_server_poll(self._h, ids, max_ids, ctypes.byref(n)), "lbm_server_poll")
        return list(ids[:n.value])

    def state(self, jid):
        st, left = ctypes.c_int(), ctypes.c_int()
        _check(load_library().lbm_server_job_state(self._h, jid, ctypes.byref(st), ctypes.byref(left)),
               "lbm_server_job_state")
        return st.value, left.value

    def fetch(self, jid):
        Lx, Ly = self.sizes.pop(jid)
        rho, u, T = np.empty((Lx, Ly)), np.empty((2, Lx, Ly)), np.empty((Lx, Ly))
        _check(load_library().lbm_server_fetch(self._h, jid, rho.ctypes.data, u.ctypes.data, T.ctypes.data),
               "lbm_server_fetch")
        return rho, u, T

    def stats(self):
        s = lbm_server_stats()
        _check(load_library().lbm_server_stats_get(self._h, ctypes.byref(s)), "lbm_server_stats_get")
        return {f: getattr(s, f) for f, _ in s._fields_}

    def close(self):
        if getattr(self, "_h", None):
            with self._dev():
                load_library().lbm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_trace(trace, budget_bytes, max_steps_per_tick=16, device=None, keep_results=False, time_limit=None):
    """Replay `trace` (dicts with arrival, Lx, Ly, steps, precision, seed,
    T_bot) in wall-clock time.  Returns a summary (jobs/s, latency
    percentiles) and, with keep_results, {trace id: (rho, u, T)}."""
    srv = Server(budget_bytes, max_steps_per_tick, device)
    pending = collections.deque(sorted(trace, key=lambda j: j["arrival"]))
    by_jid, arrival, done_at, rejected = {}, {}, {}, []
    results = {}
    t0 = time.perf_counter()
    busy = 0.0
    while pending or len(done_at) + len(rejected) < len(trace):
        now = time.perf_counter() - t0
        if time_limit is not None and now > time_limit:
            break
        while pending and pending[0]["arrival"] <= now:
            j = pending.popleft()
            try:
                jid = srv.submit(j["Lx"], j["Ly"], j["steps"], j["precision"], j["seed"], T_bot=j["T_bot"])
            except LBMError:
                rejected.append(j["id"])
                continue
            by_jid[jid] = j["id"]
            arrival[j["id"]] = j["arrival"]
        st = srv.stats()
        if st["active"] == 0 and st["queued"] == 0:
            if pending:
                time.sleep(max(0.0, pending[0]["arrival"] - (time.perf_counter() - t0)))
            continue
        tb = time.perf_counter()
        srv.tick()
        busy += time.perf_counter() - tb
        t_now = time.perf_counter() - t0
        for jid in srv.poll():
            tid = by_jid[jid]
            done_at[tid] = t_now
            r = srv.fetch(jid)
            if keep_results:
                results[tid] = r
    st = srv.stats()
    srv.close()
    lat = np.array([done_at[i] - arrival[i] for i in done_at]) if done_at else np.array([np.nan])
    first = min(arrival.values()) if arrival else 0.0
    last = max(done_at.values()) if done_at else 0.0
    summary = {"jobs": len(trace), "completed": len(done_at), "rejected": len(rejected),
               "makespan_s": round(last - first, 3),
               "jobs_per_s": round(len(done_at) / (last - first), 3) if last > first else None,
               "latency_p50_s": round(float(np.percentile(lat, 50)), 3),
               "latency_p99_s": round(float(np.percentile(lat, 99)), 3),
               "latency_mean_s": round(float(np.mean(lat)), 3),
               "site_updates": int(sum(j["Lx"] * j["Ly"] * j["steps"] for j in trace if j["id"] in done_at)),
               "ticks": st["ticks"], "launches": st["launches"], "busy_s": round(busy, 3)}
    if last > first:
        summary["mlups"] = round(summary["site_updates"] / (last - first) / 1e6, 3)
    return (summary, results) if keep_results else summary
