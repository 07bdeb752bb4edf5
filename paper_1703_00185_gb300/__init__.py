"""GB300 (sm_103a) thermal D2Q37 lattice Boltzmann step: Python binding.

A thin ``ctypes`` layer over the C ABI declared in ``include/d2q37.h`` and
built into ``libd2q37_gb300.so`` next to this file.  Functions named
``lbm_*`` marshal arguments and call the C entry point of the same name;
:class:`Lattice` bundles them with PyTorch-owned device memory and the
current PyTorch CUDA stream.  Every step of the method runs in the library's
CUDA kernels; this module computes nothing itself and raises if the library
is missing.
"""
import ctypes
import os

import numpy as np

Q = 37
LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ETIMEOUT, LBM_ESTATE, LBM_ETOOBIG = 0, -1, -2, -3, -4, -5, -6
LBM_STATIC_BATCH_MAX = 256
PHASE_PROPAGATE, PHASE_BC, PHASE_COLLIDE, PHASE_ALL = 1, 2, 4, 7
KERNEL_SEPARATE, KERNEL_FUSED, KERNEL_FUSED_SERIAL = 0, 1, 2
PRECISION_FP64, PRECISION_FP32_FP64, PRECISION_FP32_DF = 0, 1, 2
PRECISIONS = {"fp64": PRECISION_FP64, "fp32": PRECISION_FP32_FP64, "fp32-df": PRECISION_FP32_DF}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libd2q37_gb300.so")


class LBMError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (what, lbm_strerror(code) if _lib else "library error", code))


class lbm_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("active", ctypes.c_int64), ("ticks", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("budget_bytes", ctypes.c_size_t), ("bytes_in_use", ctypes.c_size_t),
                ("largest_free_bytes", ctypes.c_size_t)]


JOB_QUEUED, JOB_ACTIVE, JOB_DONE = 0, 1, 2


class lbm_params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("g0", ctypes.c_double), ("T_top", ctypes.c_double),
                ("T_bot", ctypes.c_double), ("precision", ctypes.c_int), ("kernel", ctypes.c_int),
                ("periodic_y", ctypes.c_int)]


_lib = None


def load_library():
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("D2Q37 CUDA library not built (%s missing): run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    pp = ctypes.POINTER(lbm_params)
    sig = {
        "lbm_default_params": (None, [pp]),
        "lbm_velocity_set": (ctypes.c_int, [ip, ip]),
        "lbm_quadrature": (ctypes.c_int, [dp, dp]),
        "lbm_required_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, pp]),
        "lbm_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, pp, ctypes.POINTER(vp)]),
        "lbm_create_ext": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, pp, vp, ctypes.c_size_t, vp,
                                          ctypes.POINTER(vp)]),
        "lbm_init_rayleigh_taylor": (ctypes.c_int, [vp, ctypes.c_uint64]),
        "lbm_set_populations": (ctypes.c_int, [vp, vp]),
        "lbm_get_populations": (ctypes.c_int, [vp, vp]),
        "lbm_step": (ctypes.c_int, [vp, ctypes.c_int]),
        "lbm_run_phases": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int]),
        "lbm_fields": (ctypes.c_int, [vp, vp, vp, vp]),
        "lbm_fields_device": (ctypes.c_int, [vp, vp, vp, vp]),
        "lbm_synchronize": (ctypes.c_int, [vp]),
        "lbm_launch_count": (ctypes.c_int64, [vp]),
        "lbm_set_timing": (ctypes.c_int, [vp, ctypes.c_int]),
        "lbm_kernel_times": (ctypes.c_int, [vp, dp, ctypes.POINTER(ctypes.c_int64)]),
        "lbm_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(vp), vp, ctypes.POINTER(vp)]),
        "lbm_batch_step": (ctypes.c_int, [vp, ctypes.c_int]),
        "lbm_batch_set_config": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int]),
        "lbm_batch_get_config": (ctypes.c_int, [vp, ip, ip]),
        "lbm_batch_autotune": (ctypes.c_int, [vp, ctypes.c_int, ip, ip, dp]),
        "lbm_batch_synchronize": (ctypes.c_int, [vp]),
        "lbm_batch_launch_count": (ctypes.c_int64, [vp]),
        "lbm_batch_destroy": (None, [vp]),
        "lbm_batch_step_static": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(vp), ctypes.c_int, vp]),
        "lbm_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(vp)]),
        "lbm_server_submit": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, pp, ctypes.c_uint64,
                                             ctypes.POINTER(ctypes.c_int64)]),
        "lbm_server_tick": (ctypes.c_int, [vp, ip]),
        "lbm_server_poll": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ip]),
        "lbm_server_job_state": (ctypes.c_int, [vp, ctypes.c_int64, ip, ip]),
        "lbm_server_fetch": (ctypes.c_int, [vp, ctypes.c_int64, vp, vp, vp]),
        "lbm_server_stats_get": (ctypes.c_int, [vp, ctypes.POINTER(lbm_server_stats)]),
        "lbm_server_destroy": (None, [vp]),
        "lbm_destroy": (None, [vp]),
        "lbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names of the C entry points this binding wraps."""
    return ["lbm_default_params", "lbm_velocity_set", "lbm_quadrature", "lbm_required_bytes", "lbm_create",
            "lbm_create_ext", "lbm_init_rayleigh_taylor", "lbm_set_populations", "lbm_get_populations",
            "lbm_step", "lbm_run_phases", "lbm_fields", "lbm_fields_device", "lbm_synchronize",
            "lbm_launch_count", "lbm_set_timing", "lbm_kernel_times", "lbm_destroy", "lbm_strerror",
            "lbm_batch_create", "lbm_batch_step", "lbm_batch_set_config", "lbm_batch_get_config",
            "lbm_batch_autotune", "lbm_batch_synchronize", "lbm_batch_launch_count", "lbm_batch_destroy",
            "lbm_batch_step_static",
            "lbm_server_create", "lbm_server_submit", "lbm_server_tick", "lbm_server_poll", "lbm_server_job_state",
            "lbm_server_fetch", "lbm_server_stats_get", "lbm_server_destroy"]


KERNEL_KINDS = ("wrap", "propagate", "bc", "collide", "fused", "fields", "init", "convert")


def _check(rc, what):
    if rc != LBM_OK:
        raise LBMError(rc, what)


def _ptr(a):
    """Address of a numpy array or torch tensor (host or device)."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


# ---------------------------------------------------------------- thin wrappers

def lbm_strerror(code):
    return load_library().lbm_strerror(code).decode()


def lbm_default_params():
    p = lbm_params()
    load_library().lbm_default_params(ctypes.byref(p))
    return p


def lbm_velocity_set():
    cx, cy = (ctypes.c_int * Q)(), (ctypes.c_int * Q)()
    _check(load_library().lbm_velocity_set(cx, cy), "lbm_velocity_set")
    return np.array(cx[:]), np.array(cy[:])


def lbm_quadrature():
    s, w = ctypes.c_double(), (ctypes.c_double * Q)()
    _check(load_library().lbm_quadrature(ctypes.byref(s), w), "lbm_quadrature")
    return s.value, np.array(w[:])


def lbm_required_bytes(Lx, Ly, params):
    return load_library().lbm_required_bytes(Lx, Ly, ctypes.byref(params))


def lbm_create(Lx, Ly, params):
    h = ctypes.c_void_p()
    _check(load_library().lbm_create(Lx, Ly, ctypes.byref(params), ctypes.byref(h)), "lbm_create")
    return h


def lbm_create_ext(Lx, Ly, params, dev_ptr, nbytes, cuda_stream):
    h = ctypes.c_void_p()
    _check(load_library().lbm_create_ext(Lx, Ly, ctypes.byref(params), dev_ptr, nbytes, cuda_stream,
                                         ctypes.byref(h)), "lbm_create_ext")
    return h


def lbm_init_rayleigh_taylor(h, seed):
    _check(load_library().lbm_init_rayleigh_taylor(h, seed), "lbm_init_rayleigh_taylor")


def lbm_set_populations(h, f):
    _check(load_library().lbm_set_populations(h, _ptr(f)), "lbm_set_populations")


def lbm_get_populations(h, f):
    _check(load_library().lbm_get_populations(h, _ptr(f)), "lbm_get_populations")


def lbm_step(h, n):
    _check(load_library().lbm_step(h, n), "lbm_step")


def lbm_run_phases(h, n, phases):
    _check(load_library().lbm_run_phases(h, n, phases), "lbm_run_phases")


def lbm_fields(h, rho, u, T):
    _check(load_library().lbm_fields(h, _ptr(rho), _ptr(u), _ptr(T)), "lbm_fields")


def lbm_fields_device(h, rho, u, T):
    _check(load_library().lbm_fields_device(h, _ptr(rho), _ptr(u), _ptr(T)), "lbm_fields_device")


def lbm_synchronize(h):
    _check(load_library().lbm_synchronize(h), "lbm_synchronize")


def lbm_launch_count(h):
    return load_library().lbm_launch_count(h)


def lbm_set_timing(h, enable):
    _check(load_library().lbm_set_timing(h, int(bool(enable))), "lbm_set_timing")


def lbm_kernel_times(h):
    """{kind: (total_ms, launches)} since timing was enabled."""
    n = len(KERNEL_KINDS)
    ms, cnt = (ctypes.c_double * n)(), (ctypes.c_int64 * n)()
    _check(load_library().lbm_kernel_times(h, ms, cnt), "lbm_kernel_times")
    return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_KINDS)}


def lbm_destroy(h):
    load_library().lbm_destroy(h)


def lbm_batch_step_static(handles, steps, cuda_stream):
    """Advance lattices (lbm_t handles) by `steps` steps without any device
    allocation; see include/d2q37.h.  cuda_stream is a cudaStream_t value."""
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    _check(load_library().lbm_batch_step_static(len(handles), arr, steps, cuda_stream), "lbm_batch_step_static")


# ------------------------------------------------------------------ Lattice

class Lattice:
    """One Lx x Ly lattice on a CUDA device, memory owned by PyTorch.

    ``kernel`` is "fused" (one propagate/bc/collide pass per step: the sites
    kernel and, with walls, the wall-band kernel started in its tail),
    "fused_serial" (the same two kernels one after the other) or "separate"
    (propagate, bc, collide).  ``precision`` is "fp64", "fp32"
    (FP32 deviation storage, FP64 wide terms) or "fp32-df" (FP32 deviation
    storage, double-float wide terms).  All work runs on ``stream`` (default:
    the current PyTorch stream of ``device``)."""

    def __init__(self, Lx, Ly, tau=0.8, g0=1e-4, T_top=0.5, T_bot=1.5, kernel="fused", periodic_y=False,
                 device=None, stream=None, precision="fp64"):
        import torch
        self._torch = torch
        load_library()
        self.Lx, self.Ly = int(Lx), int(Ly)
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        p = lbm_default_params()
        p.tau, p.g0, p.T_top, p.T_bot = tau, g0, T_top, T_bot
        p.kernel = {"fused": KERNEL_FUSED, "separate": KERNEL_SEPARATE, "fused_serial": KERNEL_FUSED_SERIAL}[kernel]
        p.precision = PRECISIONS[precision]
        self.precision = precision
        p.periodic_y = int(bool(periodic_y))
        self.params = p
        nbytes = lbm_required_bytes(self.Lx, self.Ly, p)
        if nbytes == 0:
            raise LBMError(LBM_EINVAL, "lbm_required_bytes")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self._mem = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self._h = lbm_create_ext(self.Lx, self.Ly, p, self._mem.data_ptr(), nbytes, self.stream.cuda_stream)

    # every call runs with this lattice's device current
    def _dev(self):
        return self._torch.cuda.device(self.device)

    def close(self):
        if getattr(self, "_h", None):
            with self._dev():
                lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_rayleigh_taylor(self, seed):
        with self._dev():
            lbm_init_rayleigh_taylor(self._h, seed)

    def step(self, n=1):
        with self._dev():
            lbm_step(self._h, n)

    def run_phases(self, n, phases):
        with self._dev():
            lbm_run_phases(self._h, n, phases)

    def set_populations(self, f):
        """f: [37, Lx, Ly] float64 host array (numpy or pinned torch) in library order."""
        if isinstance(f, np.ndarray):
            f = np.ascontiguousarray(f, dtype=np.float64)
        assert tuple(f.shape) == (Q, self.Lx, self.Ly)
        with self._dev():
            lbm_set_populations(self._h, f)
            if isinstance(f, np.ndarray):
                lbm_synchronize(self._h)

    def populations(self, out=None):
        f = out if out is not None else np.empty((Q, self.Lx, self.Ly))
        with self._dev():
            lbm_get_populations(self._h, f)
        return f

    def fields(self, out=None):
        """(rho[Lx, Ly], u[2, Lx, Ly], T[Lx, Ly]) as host float64 arrays."""
        if out is None:
            out = (np.empty((self.Lx, self.Ly)), np.empty((2, self.Lx, self.Ly)), np.empty((self.Lx, self.Ly)))
        with self._dev():
            lbm_fields(self._h, *out)
        return out

    def fields_device(self):
        """(rho, u, T) as float64 torch tensors on the device (asynchronous)."""
        t = self._torch
        rho = t.empty((self.Lx, self.Ly), dtype=t.float64, device=self.device)
        u = t.empty((2, self.Lx, self.Ly), dtype=t.float64, device=self.device)
        T = t.empty((self.Lx, self.Ly), dtype=t.float64, device=self.device)
        with self._dev():
            lbm_fields_device(self._h, rho, u, T)
        return rho, u, T

    def synchronize(self):
        with self._dev():
            lbm_synchronize(self._h)

    @property
    def launch_count(self):
        return lbm_launch_count(self._h)

    def set_timing(self, enable=True):
        with self._dev():
            lbm_set_timing(self._h, enable)

    def kernel_times(self):
        with self._dev():
            return lbm_kernel_times(self._h)


# ------------------------------------------------------------------ Batch

def _autotune_cache_path():
    return os.environ.get("D2Q37_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "d2q37_gb300", "autotune.json"))


class Batch:
    """Many lattices advanced together (``lbm_batch_*``): one launch per step
    over the tiles of every lattice, or one launch per lattice on parallel
    streams, as :meth:`set_config` or :meth:`autotune` choose.  All lattices
    must share the precision and have a state; while a batch is in use, step
    them only through it and call :meth:`synchronize` before reading their
    fields."""

    def __init__(self, lattices, stream=None):
        import torch
        self._torch = torch
        lib = load_library()
        if not lattices:
            raise ValueError("empty batch")
        self.lattices = list(lattices)
        self.device = self.lattices[0].device
        for lat in self.lattices:
            lat.synchronize()
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
            arr = (ctypes.c_void_p * len(self.lattices))(*[lat._h.value for lat in self.lattices])
            h = ctypes.c_void_p()
            _check(lib.lbm_batch_create(len(self.lattices), arr, self.stream.cuda_stream, ctypes.byref(h)),
                   "lbm_batch_create")
            self._h = h

    def _dev(self):
        return self._torch.cuda.device(self.device)

    def step(self, n=1):
        with self._dev():
            _check(load_library().lbm_batch_step(self._h, n), "lbm_batch_step")

    def set_config(self, block_y, blocks_per_sm):
        _check(load_library().lbm_batch_set_config(self._h, block_y, blocks_per_sm), "lbm_batch_set_config")

    def config(self):
        by, bps = ctypes.c_int(), ctypes.c_int()
        _check(load_library().lbm_batch_get_config(self._h, ctypes.byref(by), ctypes.byref(bps)),
               "lbm_batch_get_config")
        return by.value, bps.value

    def cache_key(self):
        name = self._torch.cuda.get_device_name(self.device)
        sites = sum(l.Lx * l.Ly for l in self.lattices)
        return "%s|%s|n=%d|sites~2^%d" % (name, self.lattices[0].precision, len(self.lattices),
                                           max(0, sites.bit_length() - 1))

    def autotune(self, trial_steps=3, use_cache=True):
        """Pick the fastest launch shape (does not advance the lattices).
        With ``use_cache`` the choice is kept in a JSON file keyed by GPU,
        precision, lattice count and total size, and reused."""
        import json
        path, key = _autotune_cache_path(), self.cache_key()
        cache = {}
        if use_cache and os.path.exists(path):
            try:
                with open(path) as fh:
                    cache = json.load(fh)
            except (OSError, ValueError):
                cache = {}
        if use_cache and key in cache:
            by, bps = cache[key]["block_y"], cache[key]["blocks_per_sm"]
            self.set_config(by, bps)
            return {"block_y": by, "blocks_per_sm": bps, "ms_per_step": cache[key].get("ms_per_step"),
                    "cached": True}
        by, bps, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        with self._dev():
            _check(load_library().lbm_batch_autotune(self._h, trial_steps, ctypes.byref(by), ctypes.byref(bps),
                                                     ctypes.byref(ms)), "lbm_batch_autotune")
        res = {"block_y": by.value, "blocks_per_sm": bps.value, "ms_per_step": ms.value, "cached": False}
        if use_cache:
            cache[key] = {k: res[k] for k in ("block_y", "blocks_per_sm", "ms_per_step")}
            try:
                os.makedirs(os.path.dirname(path), exist_ok=True)
                tmp = path + ".tmp%d" % os.getpid()
                with open(tmp, "w") as fh:
                    json.dump(cache, fh, indent=1)
                os.replace(tmp, path)
            except OSError:
                pass
        return res

    def synchronize(self):
        with self._dev():
            _check(load_library().lbm_batch_synchronize(self._h), "lbm_batch_synchronize")

    @property
    def launch_count(self):
        return load_library().lbm_batch_launch_count(self._h)

    def close(self):
        if getattr(self, "_h", None):
            with self._dev():
                load_library().lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
