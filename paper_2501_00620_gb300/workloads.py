"""Seeded synthetic inputs: the initial macroscopic fields (rho, u, T) of the
benchmark and test workloads, and the serving request mix.

This module holds none of the lattice Boltzmann arithmetic.  It only builds
initial conditions on the host as numpy arrays, so the CUDA path and the
CPU reference oracle start from byte-identical inputs.

Field shapes: rho and T are (nz, ny, nx); u is (d, nz, ny, nx).  Lattice
units throughout (dx = dt = c = 1).

Temperature scales (lattice units, c^2 = 1):
* 1D sound wave: T0 = 1/3, where the equilibrium bump width b^eq vanishes at
  rest (the standard-lattice limit).
* 1D two-state Riemann problem: the stated temperatures 1.0 and 0.8 are in
  units of T_UNIT_RIEMANN = 0.15 c^2.  With the pressure ratio of 10 the
  scheme is usable only in a narrow window of the temperature scale at
  tau = 0.55: below about 0.1 c^2 the finite-difference correction at the jump
  drives T negative within tens of steps; from 0.1 to 0.14 c^2 the run
  survives but, once the waves reach the frozen reservoirs, perturbations
  grow (a 1e-13 change in the start grows to ~1e-9 by step 4600 at 0.12);
  above 0.15 the shock approaches the lattice speed and the run fails.  At
  0.15 a 1e-6 perturbation stays at 1e-6 over 5000 steps.  The shock moves
  about 0.88 cells per step and reaches the right reservoir of a 4096-cell
  line after about 2300 steps.
* 2D Taylor-Green + pulse: T0 = 0.1 c^2.
* 3D solenoidal field: T0 = 0.05 c^2 (the paper's lowest temperature).
"""
import math

import numpy as np

T_UNIT_RIEMANN = 0.15


def _shape(d, nx, ny, nz):
    return (nz if d == 3 else 1, ny if d >= 2 else 1, nx)


def sound_wave_1d(nx=256, T0=1.0 / 3.0, amp=1e-3):
    """rho = 1 + amp sin(2 pi x / nx), u = 0, T = T0 (1D periodic sound wave)."""
    x = np.arange(nx, dtype=np.float64)
    rho = (1.0 + amp * np.sin(2.0 * np.pi * x / nx)).reshape(1, 1, nx)
    u = np.zeros((1, 1, 1, nx))
    T = np.full((1, 1, nx), T0)
    return rho, u, T


def riemann_1d(nx=4096, T_unit=T_UNIT_RIEMANN, rho_l=1.0, rho_r=0.125, t_l=1.0, t_r=0.8):
    """Two-state Riemann data: x < nx/2 left state, x >= nx/2 right state, u = 0."""
    x = np.arange(nx)
    left = x < nx // 2
    rho = np.where(left, rho_l, rho_r).astype(np.float64).reshape(1, 1, nx)
    T = (T_unit * np.where(left, t_l, t_r)).astype(np.float64).reshape(1, 1, nx)
    u = np.zeros((1, 1, 1, nx))
    return rho, u, T


def taylor_green_pulse_2d(n=2048, T0=0.1, u0=0.1, amp=0.2, sigma=None):
    """Taylor-Green vortex u = u0 sin(kx)cos(ky), v = -u0 cos(kx)sin(ky),
    k = 2 pi / n, plus a Gaussian pulse g = exp(-r^2/(2 sigma^2)) about the
    centre in density (rho = 1 + amp g) and temperature (T = T0 (1 + amp g)).
    sigma defaults to 64 cells at n = 2048 and scales with n."""
    if sigma is None:
        sigma = 64.0 * n / 2048.0
    k = 2.0 * np.pi / n
    y, x = np.meshgrid(np.arange(n, dtype=np.float64), np.arange(n, dtype=np.float64), indexing="ij")
    c = (n - 1) / 2.0
    g = np.exp(-((x - c) ** 2 + (y - c) ** 2) / (2.0 * sigma ** 2))
    rho = (1.0 + amp * g)[None]
    T = (T0 * (1.0 + amp * g))[None]
    u = np.zeros((2, 1, n, n))
    u[0, 0] = u0 * np.sin(k * x) * np.cos(k * y)
    u[1, 0] = -u0 * np.cos(k * x) * np.sin(k * y)
    return rho, u, T


def solenoidal_3d(n=256, k0=8.0, mach=0.3, T0=0.05, thermal=False, seed=0):
    """Random solenoidal velocity with energy spectrum E(k) ~ k^4 exp(-2k^2/k0^2)
    (k = integer mode number), Helmholtz-projected in Fourier space and scaled
    to rms Mach number `mach`: sqrt(<|u|^2>) = mach * c_s with
    c_s = sqrt(T0) (isothermal) or sqrt((d+2) T0 / d) = sqrt(5 T0 / 3) (thermal).
    rho = 1, T = T0.  Seeded white noise filtered in Fourier space."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((3, n, n, n))
    uh = np.fft.fftn(noise, axes=(1, 2, 3))
    kk = np.fft.fftfreq(n, d=1.0 / n)
    kz, ky, kx = np.meshgrid(kk, kk, kk, indexing="ij")
    kvec = np.stack([kx, ky, kz])           # component order (x, y, z)
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    kmag = np.sqrt(k2)
    with np.errstate(divide="ignore", invalid="ignore"):
        amp = np.where(k2 > 0, np.sqrt(kmag ** 4 * np.exp(-2.0 * k2 / k0 ** 2) / (4 * np.pi * k2)), 0.0)
        uh = uh * amp[None]
        div = (kvec * uh).sum(0)
        uh = uh - np.where(k2 > 0, kvec * div[None] / k2[None], 0.0)
    u = np.real(np.fft.ifftn(uh, axes=(1, 2, 3)))
    cs = math.sqrt(5.0 * T0 / 3.0) if thermal else math.sqrt(T0)
    urms = math.sqrt(float((u ** 2).sum(0).mean()))
    u *= mach * cs / urms
    rho = np.ones((n, n, n))
    T = np.full((n, n, n), T0)
    return rho, np.ascontiguousarray(u), T


# ---------------------------------------------------------------------------
# The five configurations (name -> parameters).  Step counts are the stated
# run lengths; tests use shorter runs where they say so.
CONFIGS = {
    "sound1d": dict(d=1, nx=256, ny=1, nz=1, tau=0.8, T0=1.0 / 3.0, thermal=False,
                    bc="periodic", steps=2000, dtype="f64"),
    "riemann1d": dict(d=1, nx=4096, ny=1, nz=1, tau=0.55, T0=T_UNIT_RIEMANN, thermal=True,
                      bc="fixed", steps=5000, dtype="f64"),
    "tgv2d": dict(d=2, nx=2048, ny=2048, nz=1, tau=0.6, T0=0.1, thermal=True,
                  bc="periodic", steps=10000, dtype="f32"),
    "turb3d": dict(d=3, nx=256, ny=256, nz=256, tau=0.52, T0=0.05, thermal=False,
                   bc="periodic", steps=2000, dtype="f32"),
    # the standard-lattice comparator on the turb3d velocity field, at its
    # native temperature cs2 = 1/3 (at T0 = 0.05 its diagonal equilibria
    # would be negative)
    "std3d": dict(d=3, nx=256, ny=256, nz=256, tau=0.52, T0=1.0 / 3.0, thermal=False,
                  bc="periodic", steps=2000, dtype="f32", model="standard"),
    # plane Poiseuille flow: half-way bounce-back walls normal to z, a
    # uniform acceleration along x (u_max = a H^2 / (8 T tau) ~ 0.02 c at
    # H = 256 once developed), from rest
    "channel3d": dict(d=3, nx=256, ny=256, nz=256, tau=0.6, T0=0.1, thermal=False,
                      bc="walls", steps=2000, dtype="f32", force=(1.0e-7, 0.0, 0.0)),
    # the turb3d lattice and fields with the MRT collision of Appendix B:
    # third- and fourth-order moments relaxed at their own rates
    "mrt3d": dict(d=3, nx=256, ny=256, nz=256, tau=0.52, T0=0.05, thermal=False,
                  bc="periodic", steps=2000, dtype="f32", mrt=(1.2, 1.4)),
}


def fields_for(name, scale=None, seed=0):
    """Initial fields of a named configuration.  `scale` replaces the grid edge
    (nx for 1D, n for 2D/3D) to build a smaller instance of the same workload."""
    c = CONFIGS[name]
    if name == "sound1d":
        return sound_wave_1d(scale or c["nx"], c["T0"])
    if name == "riemann1d":
        return riemann_1d(scale or c["nx"], c["T0"])
    if name == "tgv2d":
        return taylor_green_pulse_2d(scale or c["nx"], c["T0"])
    if name == "turb3d":
        n = scale or c["nx"]
        return solenoidal_3d(n, k0=8.0 * n / 256.0, T0=c["T0"], thermal=c["thermal"], seed=seed)
    if name == "channel3d":
        n = scale or c["nx"]
        return np.ones((n, n, n)), np.zeros((3, n, n, n)), np.full((n, n, n), c["T0"])
    if name == "mrt3d":
        n = scale or c["nx"]
        return solenoidal_3d(n, k0=8.0 * n / 256.0, T0=c["T0"], thermal=c["thermal"], seed=seed)
    if name == "std3d":
        n = scale or c["nx"]
        t = CONFIGS["turb3d"]
        rho, u, _ = solenoidal_3d(n, k0=8.0 * n / 256.0, T0=t["T0"], thermal=False, seed=seed)
        return rho, u, np.full_like(rho, c["T0"])
    raise KeyError(name)


# ---------------------------------------------------------------------------
# Serving mix: Poisson arrivals of 1D / 2D sound-wave and Riemann requests.

def serving_requests(n_requests=1000, rate=200.0, seed=0, steps_range=(100, 5000),
                     nx1d_range=(64, 65536), n2d_range=(64, 1024)):
    """Seeded request list.  Each request: arrival time (s), dim, grid, kind
    ('sound' | 'riemann'), steps.  Half 1D, half 2D; half sound waves, half
    Riemann; 1D nx and 2D edge log-uniform; steps uniform integers.  Riemann
    requests are planar in x (periodic in y for 2D)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n_requests)
    t = np.cumsum(gaps) - gaps[0]
    reqs = []
    for i in range(n_requests):
        dim = 1 if rng.random() < 0.5 else 2
        kind = "sound" if rng.random() < 0.5 else "riemann"
        if dim == 1:
            nx = int(round(math.exp(rng.uniform(math.log(nx1d_range[0]), math.log(nx1d_range[1])))))
            ny = 1
        else:
            nx = int(round(math.exp(rng.uniform(math.log(n2d_range[0]), math.log(n2d_range[1])))))
            ny = nx
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        reqs.append(dict(id=i, t_arrival=float(t[i]), dim=dim, nx=nx, ny=ny, kind=kind, steps=steps))
    return reqs


def request_fields(req):
    """Initial fields of a serving request (sound wave or planar Riemann)."""
    d, nx, ny = req["dim"], req["nx"], req["ny"]
    if req["kind"] == "sound":
        T0 = 1.0 / 3.0
        x = np.arange(nx, dtype=np.float64)
        line = 1.0 + 1e-3 * np.sin(2.0 * np.pi * x / nx)
        rho = np.broadcast_to(line, (1, ny, nx)).copy()
        T = np.full((1, ny, nx), T0)
    else:
        T0 = T_UNIT_RIEMANN
        x = np.arange(nx)
        left = x < nx // 2
        rho = np.broadcast_to(np.where(left, 1.0, 0.125), (1, ny, nx)).astype(np.float64).copy()
        T = np.broadcast_to(T0 * np.where(left, 1.0, 0.8), (1, ny, nx)).astype(np.float64).copy()
    u = np.zeros((d, 1, ny, nx))
    return rho, u, T


def request_params(req):
    """(tau, T0, thermal, bc) of a serving request, as for configs 1 and 2."""
    if req["kind"] == "sound":
        return (0.8, 1.0 / 3.0, False, "periodic")
    return (0.55, T_UNIT_RIEMANN, True, "fixed")
