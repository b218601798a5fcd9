"""Reference oracle for the bump-function lattice Boltzmann scheme (arXiv 2501.00620).

TEST INFRASTRUCTURE ONLY.  A plain, slow FP64 CPU restatement of the method
(``bump_lbm_oracle.c``) and a ctypes wrapper around it.  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package; the CUDA library never calls it and shares no code with it.

Every function of the C file cites the passage of the paper it restates; the
readings taken where the paper is silent are listed in the C file's header.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bump_lbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

# -ffp-contract=off: no fused multiply-add, so the arithmetic is the plain
# IEEE double sequence written in the source on every host (x86 and Arm).
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp"]


def build(force=False):
    """Compile the oracle with gcc (plain C, no CUDA)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_set_threads.restype = ctypes.c_int
        L.orc_lattice_info.argtypes = [ctypes.c_int, ip, ip, ip, dp]
        L.orc_lattice_info.restype = ctypes.c_int
        L.orc_feq.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
        L.orc_beq.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp]
        L.orc_forcing.argtypes = [ctypes.c_int, dp, dp, dp]
        L.orc_create.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double, ctypes.c_double,
                                                      ctypes.c_int, ctypes.c_int]
        L.orc_create.restype = ctypes.c_void_p
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_init.argtypes = [ctypes.c_void_p, dp, dp, dp]
        L.orc_init.restype = ctypes.c_int
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
        L.orc_nstep.argtypes = [ctypes.c_void_p]
        L.orc_nstep.restype = ctypes.c_long
        L.orc_set_force.argtypes = [ctypes.c_void_p, dp]
        L.orc_set_model.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_set_wall_velocity.argtypes = [ctypes.c_void_p, dp, dp]
        L.orc_set_mrt.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]
        L.orc_set_mrt.restype = ctypes.c_int
        L.orc_moment_matrix.argtypes = [dp]
        L.orc_set_wall_velocity.restype = ctypes.c_int
        L.orc_set_model.restype = ctypes.c_int
        L.orc_std_feq.argtypes = [ctypes.c_int, ctypes.c_double, dp, ctypes.c_double, dp]
        L.orc_moments.argtypes = [ctypes.c_void_p, dp, dp, dp]
        L.orc_diagnostics.argtypes = [ctypes.c_void_p, dp]
        L.orc_get_emitted.argtypes = [ctypes.c_void_p, dp, dp]
        L.orc_get_state.argtypes = [ctypes.c_void_p, dp, dp]
        L.orc_set_emitted.argtypes = [ctypes.c_void_p, dp, dp]
        L.orc_gradient.argtypes = [ctypes.c_int] * 4 + [dp, dp]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(n):
    """Number of OpenMP threads the oracle's per-site loops use; returns it."""
    return lib().orc_set_threads(int(n))


def lattice(d):
    """(e [Q,3] int, w [Q] float) of the oracle's velocity set for dimension d."""
    Q = ctypes.c_int()
    nb = ctypes.c_int()
    lib().orc_lattice_info(d, ctypes.byref(Q), ctypes.byref(nb), None, None)
    e = np.zeros((Q.value, 3), dtype=np.int32)
    w = np.zeros(Q.value)
    lib().orc_lattice_info(d, ctypes.byref(Q), ctypes.byref(nb),
                           e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(w))
    return e, w


def n_b(d):
    return {1: 1, 2: 3, 3: 6}[d]


def n_q(d):
    return {1: 3, 2: 9, 3: 19}[d]


def feq(d, rho, u):
    out = np.zeros(n_q(d))
    uu = np.zeros(3)
    uu[:d] = np.asarray(u, dtype=np.float64)[:d]
    lib().orc_feq(d, float(rho), _p(uu), _p(out))
    return out


def beq(d, u, T):
    out = np.zeros(n_b(d))
    uu = np.zeros(3)
    uu[:d] = np.asarray(u, dtype=np.float64)[:d]
    lib().orc_beq(d, _p(uu), float(T), _p(out))
    return out


def moment_matrix():
    """Table M (Appendix B) with c = 1: the D3Q19 population-to-moment matrix."""
    out = np.zeros((19, 19))
    lib().orc_moment_matrix(_p(out))
    return out


def std_feq(d, rho, u, T):
    """Equilibrium of the standard-lattice comparator (Eq. 4, lattice units)."""
    out = np.zeros(n_q(d))
    uu = np.zeros(3)
    uu[:d] = np.asarray(u, dtype=np.float64)[:d]
    lib().orc_std_feq(d, float(rho), _p(uu), float(T), _p(out))
    return out


def forcing(d, F, G):
    out = np.zeros(n_q(d))
    FF = np.zeros(3)
    FF[:d] = np.asarray(F, dtype=np.float64)[:d]
    GG = np.ascontiguousarray(G, dtype=np.float64)
    lib().orc_forcing(d, _p(FF), _p(GG), _p(out))
    return out


def gradient(d, phi):
    """Isotropic gradient of a periodic scalar field phi with shape (nz, ny, nx)."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    nz, ny, nx = phi.shape
    out = np.zeros((d,) + phi.shape)
    lib().orc_gradient(d, nx, ny, nz, _p(phi), _p(out))
    return out


class Sim:
    """One oracle lattice.  Fields are numpy arrays of shape (nz, ny, nx);
    velocity is (d, nz, ny, nx)."""

    def __init__(self, d, nx, ny=1, nz=1, tau=0.8, T0=1.0 / 3.0, thermal=False,
                 bc="periodic", model="bump"):
        self.d, self.nx, self.ny, self.nz = d, nx, ny, nz
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.Q, self.nb = n_q(d), n_b(d)
        bcode = {"periodic": 0, "fixed": 1, "walls": 2}[bc]
        self._h = lib().orc_create(d, nx, ny, nz, float(tau), float(T0),
                                   int(bool(thermal)), bcode)
        if not self._h:
            raise ValueError("oracle: invalid lattice parameters")
        if lib().orc_set_model(self._h, {"bump": 0, "standard": 1}[model]) != 0:
            raise ValueError("oracle: the standard comparator runs on periodic or walled lattices")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def init(self, rho, u, T):
        rho = np.ascontiguousarray(np.broadcast_to(rho, self.shape), dtype=np.float64)
        T = np.ascontiguousarray(np.broadcast_to(T, self.shape), dtype=np.float64)
        u = np.ascontiguousarray(np.broadcast_to(u, (self.d,) + self.shape), dtype=np.float64)
        if lib().orc_init(self._h, _p(rho), _p(u), _p(T)) != 0:
            raise ValueError("oracle: rho and T must be positive")

    def step(self, n=1):
        lib().orc_step(self._h, int(n))

    def set_mrt(self, s3, s4):
        """MRT collision in the basis of Table M (D3Q19): rates of the third-
        and fourth-order moments; the others relax at omega."""
        if lib().orc_set_mrt(self._h, float(s3), float(s4)) != 0:
            raise ValueError("oracle: MRT needs the D3Q19 bump scheme and rates in (0, 2)")

    def set_wall_velocity(self, lo, hi):
        """Tangential velocities of the lower and upper walls (d components)."""
        ll, hh = np.zeros(3), np.zeros(3)
        ll[:self.d] = np.asarray(lo, dtype=np.float64)[:self.d]
        hh[:self.d] = np.asarray(hi, dtype=np.float64)[:self.d]
        if lib().orc_set_wall_velocity(self._h, _p(ll), _p(hh)) != 0:
            raise ValueError("oracle: wall velocities need walls and must be tangential")

    def set_force(self, a):
        """Uniform body-force acceleration (d components)."""
        aa = np.zeros(3)
        aa[:self.d] = np.asarray(a, dtype=np.float64)[:self.d]
        lib().orc_set_force(self._h, _p(aa))

    @property
    def nstep(self):
        return lib().orc_nstep(self._h)

    def moments(self):
        rho = np.zeros(self.shape)
        u = np.zeros((self.d,) + self.shape)
        T = np.zeros(self.shape)
        lib().orc_moments(self._h, _p(rho), _p(u), _p(T))
        return rho, u, T

    def diagnostics(self):
        out = np.zeros(self.d + 2)
        lib().orc_diagnostics(self._h, _p(out))
        return out

    def emitted(self):
        """Post-collision (emitted) populations and bbar: (Q, nz, ny, nx), (nb, ...)."""
        f = np.zeros((self.Q,) + self.shape)
        b = np.zeros((self.nb,) + self.shape)
        lib().orc_get_emitted(self._h, _p(f), _p(b))
        return f, b

    def set_emitted(self, f, b):
        """Restart from an emitted state (Q, nz, ny, nx), (nb, nz, ny, nx)."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        lib().orc_set_emitted(self._h, _p(f), _p(b))

    def state(self):
        """Pre-collision fbar and bbar at the current time."""
        f = np.zeros((self.Q,) + self.shape)
        b = np.zeros((self.nb,) + self.shape)
        lib().orc_get_state(self._h, _p(f), _p(b))
        return f, b
