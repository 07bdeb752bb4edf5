"""CPU oracle of the thermal D2Q37 lattice Boltzmann step (FP64).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import this package.  The product library
under ``paper_1703_00185_gb300/`` never imports, links or calls it.

Parts:
  * ``quadrature``  velocity set and weights (50-digit Newton solve);
  * ``d2q37_oracle.c``  the plain FP64 step (pbc, pull propagate, wall bc,
    BGK collide with the shifted 4th-order Hermite equilibrium), built with
    gcc ``-O2 -ffp-contract=off`` and driven through ``ctypes`` here;
  * ``naive``  a second, independent numpy formulation used to brute-force
    check the C oracle on tiny lattices.

All arrays crossing this interface are float64 numpy arrays.  Populations
are ``[37, Lx, Ly]`` in this oracle's own velocity order (``velocity_set()``);
fields are ``rho[Lx, Ly]``, ``u[2, Lx, Ly]``, ``T[Lx, Ly]``.
"""
import ctypes
import os
import subprocess

import numpy as np

from . import quadrature

Q = 37
PHASE_PROPAGATE, PHASE_BC, PHASE_COLLIDE = 1, 2, 4
PHASE_ALL = 7

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "d2q37_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle_d2q37.so")
_lib = None


def build(force=False):
    """Compile the C oracle with gcc (FP contraction off, OpenMP on)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_LIB_DIR, exist_ok=True)
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


_FLOP_SRC = os.path.join(_HERE, "flop_count.cpp")
_FLOP_LIB = os.path.join(_LIB_DIR, "liboracle_d2q37_flops.so")


def build_flop_counter(force=False):
    """Compile the counting build (g++); returns the library path."""
    srcs = (_FLOP_SRC, _SRC, os.path.join(_HERE, "collide_contracted.c"))
    if force or not os.path.exists(_FLOP_LIB) or \
            os.path.getmtime(_FLOP_LIB) < max(os.path.getmtime(p) for p in srcs):
        os.makedirs(_LIB_DIR, exist_ok=True)
        tmp = _FLOP_LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fpermissive",
                               "-w", "-fPIC", "-shared", "-D_DEFAULT_SOURCE", "-o", tmp, _FLOP_SRC, "-lm"])
        os.replace(tmp, _FLOP_LIB)
    return _FLOP_LIB


def collide_flops_per_site(nontrivial=False):
    """FP64 operations the oracle performs for one site collision (moments,
    shifted fields, the equilibrium as the full Hermite tensor contraction,
    relaxation), counted by compiling its source with a counting number type
    (oracle/flop_count.cpp, g++).  nontrivial=True leaves out operations with
    an operand of exactly 0 or +-1 (the Kronecker factors of the tensor form)."""
    lib = ctypes.CDLL(build_flop_counter())
    lib.orc_count_setup.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    lib.orc_count_setup.restype = ctypes.c_int
    lib.orc_count_collide_site.argtypes = [ctypes.c_int]
    lib.orc_count_collide_site.restype = ctypes.c_longlong
    s, w = scale_and_weights()
    cx, cy = velocity_set()
    c2 = (np.asarray(cx) ** 2 + np.asarray(cy) ** 2).tolist()
    w_shell = np.ascontiguousarray([float(np.asarray(w)[c2.index(k)]) for k in sorted(set(c2))])
    lib.orc_count_setup(float(s), w_shell.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return int(lib.orc_count_collide_site(1 if nontrivial else 0))


def _flop_lib():
    lib = ctypes.CDLL(build_flop_counter())
    lib.orc_count_setup.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    lib.orc_count_setup.restype = ctypes.c_int
    lib.orc_count_collide_form.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.orc_count_collide_form.restype = ctypes.c_longlong
    dp = ctypes.POINTER(ctypes.c_double)
    lib.orc_collide_form_values.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
    s, w = scale_and_weights()
    cx, cy = velocity_set()
    c2 = (np.asarray(cx) ** 2 + np.asarray(cy) ** 2).tolist()
    w_shell = np.ascontiguousarray([float(np.asarray(w)[c2.index(k)]) for k in sorted(set(c2))])
    lib.orc_count_setup(float(s), w_shell.ctypes.data_as(dp))
    return lib


def contracted_collide_flops_per_site(nontrivial=False):
    """FP64 operations of one site collision with the equilibrium contracted
    by hand into its scalar polynomial (oracle/collide_contracted.c), every
    population evaluated on its own: the plain per-site FP64 work of the
    method, counted by the same counting build."""
    return int(_flop_lib().orc_count_collide_form(1, 1 if nontrivial else 0))


def counted_collide_values(f, tau, gx, gy, contracted):
    """The relaxed populations of one site from the counting build, in the
    oracle's tensor form (contracted=False) or the hand-contracted one."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(Q)
    _flop_lib().orc_collide_form_values(1 if contracted else 0, _p(f), tau, gx, gy, _p(out))
    return out


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.orc_setup.argtypes = [ctypes.c_double, dp]
    lib.orc_setup.restype = ctypes.c_int
    lib.orc_velocity_set.argtypes = [ip, ip]
    lib.orc_weights.argtypes = [dp]
    lib.orc_threads.restype = ctypes.c_int
    lib.orc_set_threads.argtypes = [ctypes.c_int]
    lib.orc_equilibrium.argtypes = [ctypes.c_double] * 4 + [dp]
    lib.orc_site_moments.argtypes = [dp, dp, dp, dp, dp]
    lib.orc_collide_site.argtypes = [dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
    lib.orc_create.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 + [ctypes.c_int]
    lib.orc_create.restype = ctypes.c_void_p
    lib.orc_destroy.argtypes = [ctypes.c_void_p]
    lib.orc_set_populations.argtypes = [ctypes.c_void_p, dp]
    lib.orc_get_populations.argtypes = [ctypes.c_void_p, dp]
    lib.orc_run.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    lib.orc_run.restype = ctypes.c_int
    lib.orc_fields.argtypes = [ctypes.c_void_p, dp, dp, dp]
    lib.orc_splitmix64.argtypes = [ctypes.c_uint64]
    lib.orc_splitmix64.restype = ctypes.c_uint64
    lib.orc_rt_temperature.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_double,
                                       ctypes.c_double, dp]
    lib.orc_init_rayleigh_taylor.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    lib.orc_set_equilibrium.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
    s, w = quadrature.weights_fp64()
    wa = (ctypes.c_double * 8)(*w)
    if lib.orc_setup(s, wa) != Q:
        raise RuntimeError("oracle set-up failed")
    _lib = lib
    return lib


def _p(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def velocity_set():
    """(cx, cy) int arrays of the 37 hops in this oracle's order."""
    lib = _load()
    cx = (ctypes.c_int * Q)()
    cy = (ctypes.c_int * Q)()
    lib.orc_velocity_set(cx, cy)
    return np.array(cx[:]), np.array(cy[:])


def scale_and_weights():
    """(s, w[37]) as used by the oracle."""
    lib = _load()
    w = np.zeros(Q)
    lib.orc_weights(_p(w))
    return quadrature.weights_fp64()[0], w


def threads():
    return _load().orc_threads()


def set_threads(n):
    """OpenMP threads of the oracle's site loops (the results do not change)."""
    _load().orc_set_threads(int(n))


def equilibrium(rho, ux, uy, T):
    """f^eq_l(rho, u, T) for the 37 velocities (4th-order Hermite)."""
    out = np.zeros(Q)
    _load().orc_equilibrium(rho, ux, uy, T, _p(out))
    return out


def site_moments(f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    r = [ctypes.c_double() for _ in range(4)]
    _load().orc_site_moments(_p(f), *[ctypes.byref(x) for x in r])
    return tuple(x.value for x in r)


def collide_site(f, tau, gx, gy):
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(Q)
    _load().orc_collide_site(_p(f), tau, gx, gy, _p(out))
    return out


def splitmix64(v):
    return _load().orc_splitmix64(v)


def rt_temperature(Lx, Ly, seed, T_top=0.5, T_bot=1.5):
    T = np.zeros((Lx, Ly))
    _load().orc_rt_temperature(Lx, Ly, seed, T_top, T_bot, _p(T))
    return T


class Lattice:
    """An Lx x Ly lattice (x periodic; walls at y = 0 and y = Ly - 1 unless
    ``periodic_y``), gravity g = (0, -g0)."""

    def __init__(self, Lx, Ly, tau=0.8, g0=1e-4, T_top=0.5, T_bot=1.5, periodic_y=False):
        self._lib = _load()
        self.Lx, self.Ly = Lx, Ly
        self.tau, self.g0, self.T_top, self.T_bot = tau, g0, T_top, T_bot
        self.periodic_y = bool(periodic_y)
        self._h = self._lib.orc_create(Lx, Ly, tau, g0, T_top, T_bot, int(periodic_y))
        if not self._h:
            raise ValueError("invalid lattice parameters")

    def close(self):
        if self._h:
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (Q, self.Lx, self.Ly)
        self._lib.orc_set_populations(self._h, _p(f))

    def populations(self):
        f = np.zeros((Q, self.Lx, self.Ly))
        self._lib.orc_get_populations(self._h, _p(f))
        return f

    def set_equilibrium(self, rho, ux, uy, T):
        """Populations at equilibrium with the given [Lx, Ly] fields."""
        a = [np.ascontiguousarray(np.broadcast_to(v, (self.Lx, self.Ly)), dtype=np.float64) for v in (rho, ux, uy, T)]
        self._lib.orc_set_equilibrium(self._h, *[_p(v) for v in a])

    def init_rayleigh_taylor(self, seed):
        self._lib.orc_init_rayleigh_taylor(self._h, seed)

    def run(self, nsteps=1, phases=PHASE_ALL):
        if self._lib.orc_run(self._h, nsteps, phases) != 0:
            raise ValueError("bad phase mask %d" % phases)

    def fields(self):
        n = self.Lx * self.Ly
        rho, u, T = np.zeros(n), np.zeros(2 * n), np.zeros(n)
        self._lib.orc_fields(self._h, _p(rho), _p(u), _p(T))
        return rho.reshape(self.Lx, self.Ly), u.reshape(2, self.Lx, self.Ly), T.reshape(self.Lx, self.Ly)
