"""Thin ctypes binding of the C ABI in include/lbm.h (liblbm.so).

Argument marshalling only: every step of the method runs in the CUDA
library.  Functions keep the C names (lbm_create, lbm_init, lbm_step, ...);
``Simulation`` is a small convenience wrapper that owns a handle and moves
numpy arrays in and out.  Importing this module fails loudly if liblbm.so
has not been built -- there is no CPU fallback.

Field shapes follow the library's layout: rho and T are (nz, ny, nx), u is
(d, nz, ny, nx); populations are (Q, nz, ny, nx) and the variance tensor
(nb, nz, ny, nx).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_EBUSY, LBM_EIO = range(8)
LBM_BC_PERIODIC, LBM_BC_FIXED_STATE, LBM_BC_WALLS = 0, 1, 2
LBM_F64, LBM_F32, LBM_F16_SHIFTED, LBM_BF16_SHIFTED = 0, 1, 2, 3
DTYPES = {"f64": LBM_F64, "f32": LBM_F32, "f16": LBM_F16_SHIFTED, "bf16": LBM_BF16_SHIFTED}
BCS = {"periodic": LBM_BC_PERIODIC, "fixed": LBM_BC_FIXED_STATE, "walls": LBM_BC_WALLS}
LBM_MODEL_BUMP, LBM_MODEL_STANDARD = 0, 1
MODELS = {"bump": LBM_MODEL_BUMP, "standard": LBM_MODEL_STANDARD}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class lbm_opts(ctypes.Structure):
    _fields_ = [
        ("dtype", ctypes.c_int),
        ("thermal", ctypes.c_int),
        ("device", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("alloc", ALLOC_FN),
        ("free", FREE_FN),
        ("alloc_ctx", ctypes.c_void_p),
        ("tile", ctypes.c_int),
        ("chunk", ctypes.c_int),
        ("steps_per_launch", ctypes.c_int),
        ("diagnostics", ctypes.c_int),
        ("use_graphs", ctypes.c_int),
        ("model", ctypes.c_int),
        ("halo", ctypes.c_int),
        ("inplace", ctypes.c_int),
        ("cluster", ctypes.c_int),
    ]


class lbm_fields_in(ctypes.Structure):
    _fields_ = [("rho", ctypes.POINTER(ctypes.c_double)),
                ("u", ctypes.POINTER(ctypes.c_double)),
                ("T", ctypes.POINTER(ctypes.c_double))]


class lbm_fields_out(ctypes.Structure):
    _fields_ = [("rho", ctypes.POINTER(ctypes.c_double)),
                ("u", ctypes.POINTER(ctypes.c_double)),
                ("T", ctypes.POINTER(ctypes.c_double))]


class LBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("lbm status %d: %s" % (status, msg))
        self.status = status


class lbm_server_opts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t),
                ("max_active", ctypes.c_int),
                ("device", ctypes.c_int),
                ("round_ms", ctypes.c_double),
                ("idle_ms", ctypes.c_double)]


class lbm_request(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int),
                ("nx", ctypes.c_int),
                ("ny", ctypes.c_int),
                ("tau", ctypes.c_double),
                ("T0", ctypes.c_double),
                ("thermal", ctypes.c_int),
                ("bc", ctypes.c_int),
                ("steps", ctypes.c_long),
                ("rho", ctypes.POINTER(ctypes.c_double)),
                ("u", ctypes.POINTER(ctypes.c_double)),
                ("T", ctypes.POINTER(ctypes.c_double))]


class lbm_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64),
                ("completed", ctypes.c_uint64),
                ("active", ctypes.c_int),
                ("queued", ctypes.c_int),
                ("site_updates", ctypes.c_double),
                ("busy_s", ctypes.c_double),
                ("rounds", ctypes.c_uint64),
                ("first_submit_s", ctypes.c_double),
                ("last_done_s", ctypes.c_double),
                ("pool_bytes", ctypes.c_size_t),
                ("pool_in_use", ctypes.c_size_t),
                ("kernel_launches", ctypes.c_uint64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("liblbm.so is not built (run __graft_entry__.build() or "
                          "python -m paper_2501_00620_gb300.build); the CUDA library is required")
    L = ctypes.CDLL(LIB_PATH)
    dp = ctypes.POINTER(ctypes.c_double)
    vp = ctypes.c_void_p
    L.lbm_default_opts.argtypes = [ctypes.POINTER(lbm_opts)]
    L.lbm_default_opts.restype = None
    L.lbm_create.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                  ctypes.POINTER(vp)]
    L.lbm_create_ex.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                     ctypes.POINTER(lbm_opts), ctypes.POINTER(vp)]
    L.lbm_init.argtypes = [vp, ctypes.POINTER(lbm_fields_in)]
    L.lbm_step.argtypes = [vp, ctypes.c_long]
    L.lbm_set_force.argtypes = [vp, dp]
    L.lbm_set_wall_velocity.argtypes = [vp, dp, dp]
    L.lbm_set_mrt.argtypes = [vp, ctypes.c_double, ctypes.c_double]
    L.lbm_set_debug.argtypes = [vp, ctypes.c_int]
    L.lbm_set_small_t.argtypes = [vp, ctypes.c_double]
    L.lbm_halo_bytes.argtypes = [vp]
    L.lbm_halo_bytes.restype = ctypes.c_size_t
    L.lbm_halo_pack.argtypes = [vp, ctypes.c_int, vp]
    L.lbm_halo_unpack.argtypes = [vp, ctypes.c_int, vp]
    L.lbm_halo_exchange.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
    L.lbm_sync.argtypes = [vp]
    L.lbm_moments.argtypes = [vp, ctypes.POINTER(lbm_fields_out)]
    L.lbm_diagnostics.argtypes = [vp, dp]
    L.lbm_diagnostics_history.argtypes = [vp, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.lbm_last_diagnostics.argtypes = [vp, dp]
    L.lbm_get_state.argtypes = [vp, dp, dp]
    L.lbm_set_state.argtypes = [vp, dp, dp]
    L.lbm_flags.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.lbm_flags.restype = ctypes.c_int
    L.lbm_step_count.argtypes = [vp]
    L.lbm_step_count.restype = ctypes.c_long
    L.lbm_launch_config.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_char_p)]
    L.lbm_save.argtypes = [vp, ctypes.c_char_p]
    L.lbm_load.argtypes = [vp, ctypes.c_char_p]
    L.lbm_step_noalloc.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double, ctypes.c_double, ctypes.c_int] + [vp] * 6
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    L.lbm_server_default_opts.argtypes = [ctypes.POINTER(lbm_server_opts)]
    L.lbm_server_default_opts.restype = None
    L.lbm_server_create.argtypes = [ctypes.POINTER(lbm_server_opts), ctypes.POINTER(vp)]
    L.lbm_server_submit.argtypes = [vp, ctypes.POINTER(lbm_request), ctypes.POINTER(ctypes.c_uint64)]
    L.lbm_server_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(lbm_fields_out), dp]
    L.lbm_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(lbm_fields_out), dp]
    L.lbm_server_stats_get.argtypes = [vp, ctypes.POINTER(lbm_server_stats)]
    L.lbm_server_destroy.argtypes = [vp]
    L.lbm_server_destroy.restype = None
    L.lbm_last_error.restype = ctypes.c_char_p
    L.lbm_version.restype = ctypes.c_char_p
    for name in ("lbm_create", "lbm_create_ex", "lbm_init", "lbm_step", "lbm_set_force", "lbm_set_wall_velocity", "lbm_set_mrt", "lbm_set_debug", "lbm_set_small_t", "lbm_halo_pack", "lbm_halo_unpack",
                 "lbm_halo_exchange", "lbm_sync", "lbm_moments",
                 "lbm_diagnostics", "lbm_diagnostics_history", "lbm_last_diagnostics", "lbm_get_state", "lbm_set_state",
                 "lbm_save", "lbm_load", "lbm_step_noalloc", "lbm_launch_config", "lbm_server_create",
                 "lbm_server_submit", "lbm_server_poll", "lbm_server_wait", "lbm_server_stats_get"):
        getattr(L, name).restype = ctypes.c_int
    return L


_lib = _load()


def lib():
    return _lib


def _check(status):
    if status != LBM_OK:
        raise LBMError(status, _lib.lbm_last_error().decode())


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


# --- C names -----------------------------------------------------------------

def lbm_version():
    return _lib.lbm_version().decode()


def lbm_default_opts():
    o = lbm_opts()
    _lib.lbm_default_opts(ctypes.byref(o))
    return o


def lbm_create(dim, nx, ny, nz, tau, T0, bc=LBM_BC_PERIODIC, opts=None):
    h = ctypes.c_void_p()
    if opts is None:
        _check(_lib.lbm_create(dim, nx, ny, nz, tau, T0, bc, ctypes.byref(h)))
    else:
        _check(_lib.lbm_create_ex(dim, nx, ny, nz, tau, T0, bc, ctypes.byref(opts), ctypes.byref(h)))
    return h


def lbm_init(sim, rho, u, T):
    fi = lbm_fields_in(_dp(rho), _dp(u), _dp(T))
    _check(_lib.lbm_init(sim, ctypes.byref(fi)))


def lbm_step(sim, n):
    _check(_lib.lbm_step(sim, int(n)))


def lbm_set_mrt(sim, s3, s4):
    _check(_lib.lbm_set_mrt(sim, float(s3), float(s4)))


LBM_DEBUG_MISSING_COPY = 1


def lbm_set_small_t(sim, kappa):
    _check(_lib.lbm_set_small_t(sim, float(kappa)))


def lbm_set_debug(sim, flags):
    _check(_lib.lbm_set_debug(sim, int(flags)))


def lbm_halo_bytes(sim):
    return int(_lib.lbm_halo_bytes(sim))


def lbm_halo_pack(sim, side, dst_ptr):
    _check(_lib.lbm_halo_pack(sim, int(side), ctypes.c_void_p(dst_ptr)))


def lbm_halo_unpack(sim, side, src_ptr):
    _check(_lib.lbm_halo_unpack(sim, int(side), ctypes.c_void_p(src_ptr)))


def lbm_halo_exchange(sims):
    arr = (ctypes.c_void_p * len(sims))(*[s.h if isinstance(s, Simulation) else s for s in sims])
    _check(_lib.lbm_halo_exchange(arr, len(sims)))


def lbm_set_wall_velocity(sim, lo, hi):
    ll = None if lo is None else np.ascontiguousarray(lo, dtype=np.float64)
    hh = None if hi is None else np.ascontiguousarray(hi, dtype=np.float64)
    _check(_lib.lbm_set_wall_velocity(sim, _dp(ll), _dp(hh)))


def lbm_set_force(sim, a):
    if a is None:
        _check(_lib.lbm_set_force(sim, None))
        return
    aa = np.ascontiguousarray(a, dtype=np.float64)
    _check(_lib.lbm_set_force(sim, _dp(aa)))


def lbm_sync(sim):
    _check(_lib.lbm_sync(sim))


def lbm_moments(sim, rho, u, T):
    fo = lbm_fields_out(_dp(rho), _dp(u), _dp(T))
    _check(_lib.lbm_moments(sim, ctypes.byref(fo)))


def lbm_diagnostics(sim, out):
    _check(_lib.lbm_diagnostics(sim, _dp(out)))


def lbm_diagnostics_history(sim, out, cap):
    n = ctypes.c_int()
    _check(_lib.lbm_diagnostics_history(sim, _dp(out), int(cap), ctypes.byref(n)))
    return n.value


def lbm_last_diagnostics(sim, out):
    _check(_lib.lbm_last_diagnostics(sim, _dp(out)))


def lbm_get_state(sim, f, b):
    _check(_lib.lbm_get_state(sim, _dp(f), _dp(b)))


def lbm_set_state(sim, f, b):
    _check(_lib.lbm_set_state(sim, _dp(f), _dp(b)))


def lbm_flags(sim):
    v = ctypes.c_int()
    _check(_lib.lbm_flags(sim, ctypes.byref(v)))
    return v.value


def lbm_step_count(sim):
    return _lib.lbm_step_count(sim)


def lbm_launch_config(sim):
    """(tile, chunk, kernel name) of the step launches; (-1, -1, '') before the first step."""
    t, c, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_char_p()
    _check(_lib.lbm_launch_config(sim, ctypes.byref(t), ctypes.byref(c), ctypes.byref(k)))
    return t.value, c.value, (k.value or b"").decode()


def lbm_save(sim, path):
    _check(_lib.lbm_save(sim, os.fsencode(path)))


def lbm_load(sim, path):
    _check(_lib.lbm_load(sim, os.fsencode(path)))


def lbm_step_noalloc(dim, nx, ny, nz, tau, T0, thermal, f_in, b_in, f_out, b_out, diag_out=None, stream=None):
    """One step on caller-owned FP64 device buffers without any device
    allocation (the library's fixed scratch array); pointers are integers
    (e.g. ``tensor.data_ptr()``), ``diag_out`` and ``stream`` may be None."""
    _check(_lib.lbm_step_noalloc(dim, nx, ny, nz, float(tau), float(T0), int(bool(thermal)),
                                 f_in, b_in, f_out, b_out, diag_out, stream))


def lbm_destroy(sim):
    _lib.lbm_destroy(sim)


# --- convenience wrapper -------------------------------------------------------

def n_q(d):
    return {1: 3, 2: 9, 3: 19}[d]


def n_b(d):
    return {1: 1, 2: 3, 3: 6}[d]


class TorchAllocator:
    """Device allocator callbacks backed by PyTorch's caching allocator."""

    def __init__(self, device=0):
        import torch
        self.torch = torch
        self.device = device
        self._alloc = ALLOC_FN(self._a)
        self._free = FREE_FN(self._f)

    def _a(self, nbytes, ctx):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device)
        except Exception:
            return None

    def _f(self, ptr, nbytes, ctx):
        self.torch.cuda.caching_allocator_delete(ptr)


class Simulation:
    """One lattice on the GPU.  dims = (nx, ny, nz); unused extents are 1."""

    def __init__(self, dim, nx, ny=1, nz=1, tau=0.8, T0=1.0 / 3.0, bc="periodic", dtype="f64",
                 thermal=False, device=0, stream=None, tile=-1, chunk=0, diagnostics=True,
                 use_graphs=True, torch_allocator=False, steps_per_launch=0, model="bump", halo=0,
                 inplace=False, cluster=0):
        self.dim, self.nx, self.ny, self.nz = dim, nx, ny, nz
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.Q, self.nb = n_q(dim), n_b(dim)
        o = lbm_default_opts()
        o.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        o.thermal = int(bool(thermal))
        o.device = device
        o.stream = stream
        o.tile = tile
        o.chunk = chunk
        o.diagnostics = int(bool(diagnostics))
        o.use_graphs = int(bool(use_graphs))
        o.steps_per_launch = int(steps_per_launch)
        o.model = MODELS[model] if isinstance(model, str) else int(model)
        o.halo = int(halo)
        o.inplace = int(bool(inplace))
        o.cluster = int(cluster)
        self.halo = int(halo)
        self._allocator = None
        if torch_allocator:
            self._allocator = TorchAllocator(device)
            o.alloc = self._allocator._alloc
            o.free = self._allocator._free
        self._opts = o
        self.h = lbm_create(dim, nx, ny, nz, tau, T0, BCS[bc] if isinstance(bc, str) else bc, o)

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, rho, u, T):
        rho = np.ascontiguousarray(np.broadcast_to(rho, self.shape), dtype=np.float64)
        T = np.ascontiguousarray(np.broadcast_to(T, self.shape), dtype=np.float64)
        u = np.ascontiguousarray(np.broadcast_to(u, (self.dim,) + self.shape), dtype=np.float64)
        lbm_init(self.h, rho, u, T)

    def step(self, n=1):
        lbm_step(self.h, n)

    def set_mrt(self, s3, s4):
        """MRT collision (D3Q19): rates of the third- and fourth-order moments."""
        lbm_set_mrt(self.h, s3, s4)

    def halo_bytes(self):
        """Bytes of one halo message (lbm_opts.halo slabs)."""
        return lbm_halo_bytes(self.h)

    def halo_pack(self, side, dst_ptr):
        """Outermost owned planes on `side` (0 low, 1 high) into device memory."""
        lbm_halo_pack(self.h, side, dst_ptr)

    def halo_unpack(self, side, src_ptr):
        """A neighbour's message into the halo planes on `side`."""
        lbm_halo_unpack(self.h, side, src_ptr)

    def set_small_t(self, kappa):
        """FP64 temperature recovery where T < kappa |u|^2 (thermal, 32/16-bit storage)."""
        lbm_set_small_t(self.h, kappa)

    def set_debug(self, flags):
        """Test switches of the staged kernels (LBM_DEBUG_MISSING_COPY)."""
        lbm_set_debug(self.h, flags)

    def set_wall_velocity(self, lo, hi):
        """Velocities of the lower and upper walls (dim components each)."""
        cut = lambda v: None if v is None else np.asarray(v, dtype=np.float64)[: self.dim]
        lbm_set_wall_velocity(self.h, cut(lo), cut(hi))

    def set_force(self, a):
        """Uniform body-force acceleration (dim components; None removes it)."""
        lbm_set_force(self.h, None if a is None else np.asarray(a, dtype=np.float64)[: self.dim])

    def sync(self):
        lbm_sync(self.h)

    def flags(self):
        return lbm_flags(self.h)

    @property
    def nstep(self):
        return lbm_step_count(self.h)

    def moments(self):
        rho = np.empty(self.shape)
        u = np.empty((self.dim,) + self.shape)
        T = np.empty(self.shape)
        lbm_moments(self.h, rho, u, T)
        return rho, u, T

    def diagnostics(self):
        out = np.empty(self.dim + 2)
        lbm_diagnostics(self.h, out)
        return out

    def diagnostics_history(self, cap=4096):
        out = np.empty((cap, self.dim + 3))
        n = lbm_diagnostics_history(self.h, out, cap)
        return out[:n]

    def last_diagnostics(self):
        out = np.empty(self.dim + 3)
        lbm_last_diagnostics(self.h, out)
        return out

    def emitted(self):
        f = np.empty((self.Q,) + self.shape)
        b = np.empty((self.nb,) + self.shape)
        lbm_get_state(self.h, f, b)
        return f, b

    def set_emitted(self, f, b):
        f = np.ascontiguousarray(f, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        lbm_set_state(self.h, f, b)

    def launch_config(self):
        return lbm_launch_config(self.h)

    def save(self, path):
        lbm_save(self.h, path)

    def load(self, path):
        lbm_load(self.h, path)


# ---------------------------------------------------------------------------
# Serving (include/lbm_serve.h)

def lbm_server_default_opts():
    o = lbm_server_opts()
    _lib.lbm_server_default_opts(ctypes.byref(o))
    return o


class ServeResult(tuple):
    """(rho, u, T, latency_s) of a finished request; ``unstable`` is True when
    the simulation became non-physical (the fields are those it reached)."""
    unstable = False


class Server:
    """Continuous-batching service for D1Q3 / D2Q9 requests (FP32)."""

    def __init__(self, hbm_budget=0, max_active=0, device=0, round_ms=0.0, idle_ms=0.0):
        o = lbm_server_default_opts()
        o.hbm_budget = int(hbm_budget)
        if max_active:
            o.max_active = int(max_active)
        o.device = device
        if round_ms:
            o.round_ms = float(round_ms)
        if idle_ms:
            o.idle_ms = float(idle_ms)
        h = ctypes.c_void_p()
        _check(_lib.lbm_server_create(ctypes.byref(o), ctypes.byref(h)))
        self.h = h
        self._shapes = {}

    def submit(self, dim, nx, ny, tau, T0, thermal, bc, steps, rho, u, T):
        """Queue one request; rho, T of N values and u of dim x N (any shape). Returns the ticket."""
        N = nx * ny
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(N)
        T = np.ascontiguousarray(T, dtype=np.float64).reshape(N)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(dim * N)
        q = lbm_request(dim, nx, ny, float(tau), float(T0), int(bool(thermal)),
                        BCS[bc] if isinstance(bc, str) else int(bc), int(steps), _dp(rho), _dp(u), _dp(T))
        t = ctypes.c_uint64()
        _check(_lib.lbm_server_submit(self.h, ctypes.byref(q), ctypes.byref(t)))
        self._shapes[t.value] = (dim, ny, nx)
        return t.value

    def _result(self, fn, ticket, *extra):
        dim, ny, nx = self._shapes[ticket]
        rho = np.empty((ny, nx))
        u = np.empty((dim, ny, nx))
        T = np.empty((ny, nx))
        lat = ctypes.c_double()
        out = lbm_fields_out(_dp(rho), _dp(u), _dp(T))
        st = fn(self.h, ctypes.c_uint64(ticket), *extra, ctypes.byref(out), ctypes.byref(lat))
        if st == LBM_EBUSY:
            return None
        if st not in (LBM_OK, LBM_EUNSTABLE):
            _check(st)
        del self._shapes[ticket]
        r = ServeResult((rho, u, T, lat.value))
        r.unstable = st == LBM_EUNSTABLE
        return r

    def poll(self, ticket):
        """ServeResult (rho, u, T, latency_s) once done, else None."""
        return self._result(_lib.lbm_server_poll, ticket)

    def wait(self, ticket, timeout=600.0):
        r = self._result(_lib.lbm_server_wait, ticket, ctypes.c_double(timeout))
        if r is None:
            raise LBMError(LBM_EBUSY, "request %d not finished after %.0f s" % (ticket, timeout))
        return r

    def stats(self):
        st = lbm_server_stats()
        _check(_lib.lbm_server_stats_get(self.h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in lbm_server_stats._fields_}

    def close(self):
        if getattr(self, "h", None):
            _lib.lbm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
