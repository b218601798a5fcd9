"""Closed forms and independent solvers used to pin the oracle.

Nothing here calls the oracle or the CUDA library: these are textbook results
the bump-function scheme must reproduce.

* ``exact_riemann`` -- exact solution of the Riemann problem for the 1D Euler
  equations of an ideal gas (the two-shock/two-rarefaction pressure function
  solved by root finding, then sampled along x/t), following the exact
  Riemann solver of E. F. Toro, "Riemann Solvers and Numerical Methods for
  Fluid Dynamics", ch. 4.
* ``fit_damped_mode`` -- least-squares fit of a(t) = exp(-g t)(A cos w t +
  B sin w t), the free response of a damped linear sound mode.
* ``standard_d1q3_bgk`` -- the textbook D1Q3 BGK scheme (second-order Hermite
  equilibrium, relaxation time tau_LB), for the standard-lattice limit.
"""
import numpy as np
from scipy.optimize import brentq, curve_fit


def _f_K(p, rhoK, pK, aK, g):
    """Velocity jump across the K wave as a function of the star pressure."""
    if p > pK:  # shock
        A = 2.0 / ((g + 1.0) * rhoK)
        B = (g - 1.0) / (g + 1.0) * pK
        return (p - pK) * np.sqrt(A / (p + B))
    # rarefaction
    return 2.0 * aK / (g - 1.0) * ((p / pK) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def star_state(L, R, g):
    rL, uL, pL = L
    rR, uR, pR = R
    aL, aR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    fun = lambda p: _f_K(p, rL, pL, aL, g) + _f_K(p, rR, pR, aR, g) + (uR - uL)
    hi = max(pL, pR)
    while fun(hi) < 0:
        hi *= 2.0
    ps = brentq(fun, 1e-14 * min(pL, pR), hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    us = 0.5 * (uL + uR) + 0.5 * (_f_K(ps, rR, pR, aR, g) - _f_K(ps, rL, pL, aL, g))
    return ps, us


def exact_riemann(L, R, g, s):
    """Density, velocity, pressure of the exact solution at similarity
    coordinates s = x/t (array).  L, R = (rho, u, p)."""
    rL, uL, pL = L
    rR, uR, pR = R
    aL, aR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    ps, us = star_state(L, R, g)
    s = np.asarray(s, dtype=np.float64)
    rho = np.empty_like(s)
    u = np.empty_like(s)
    p = np.empty_like(s)
    gm = (g - 1.0) / (g + 1.0)
    for k, S in enumerate(s):
        if S <= us:  # left of the contact
            if ps > pL:  # left shock
                SL = uL - aL * np.sqrt((g + 1) / (2 * g) * ps / pL + (g - 1) / (2 * g))
                if S <= SL:
                    rho[k], u[k], p[k] = rL, uL, pL
                else:
                    rho[k] = rL * ((ps / pL + gm) / (gm * ps / pL + 1.0))
                    u[k], p[k] = us, ps
            else:  # left rarefaction
                aSL = aL * (ps / pL) ** ((g - 1) / (2 * g))
                SHL, STL = uL - aL, us - aSL
                if S <= SHL:
                    rho[k], u[k], p[k] = rL, uL, pL
                elif S >= STL:
                    rho[k] = rL * (ps / pL) ** (1.0 / g)
                    u[k], p[k] = us, ps
                else:
                    c = 2.0 / (g + 1) + gm / aL * (uL - S)
                    rho[k] = rL * c ** (2.0 / (g - 1))
                    u[k] = 2.0 / (g + 1) * (aL + (g - 1) / 2 * uL + S)
                    p[k] = pL * c ** (2 * g / (g - 1))
        else:  # right of the contact
            if ps > pR:  # right shock
                SR = uR + aR * np.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))
                if S >= SR:
                    rho[k], u[k], p[k] = rR, uR, pR
                else:
                    rho[k] = rR * ((ps / pR + gm) / (gm * ps / pR + 1.0))
                    u[k], p[k] = us, ps
            else:  # right rarefaction
                aSR = aR * (ps / pR) ** ((g - 1) / (2 * g))
                SHR, STR = uR + aR, us + aSR
                if S >= SHR:
                    rho[k], u[k], p[k] = rR, uR, pR
                elif S <= STR:
                    rho[k] = rR * (ps / pR) ** (1.0 / g)
                    u[k], p[k] = us, ps
                else:
                    c = 2.0 / (g + 1) - gm / aR * (uR - S)
                    rho[k] = rR * c ** (2.0 / (g - 1))
                    u[k] = 2.0 / (g + 1) * (-aR + (g - 1) / 2 * uR + S)
                    p[k] = pR * c ** (2 * g / (g - 1))
    return rho, u, p


def damped(t, A, B, g, w):
    return np.exp(-g * t) * (A * np.cos(w * t) + B * np.sin(w * t))


def fit_damped_mode(t, a, g0, w0):
    """Fit a(t) = exp(-g t)(A cos wt + B sin wt); returns (g, w)."""
    p0 = [a[0], 0.0, g0, w0]
    popt, _ = curve_fit(damped, t, a, p0=p0, maxfev=20000)
    return abs(popt[2]), abs(popt[3])


def fit_exponential(t, a):
    """Fit a(t) = A exp(-g t) by least squares on log|a|; returns g."""
    c = np.polyfit(t, np.log(np.abs(a)), 1)
    return -c[0]


def mode_amplitude(field, k, axis_coord):
    """Projection of a periodic field onto sin(k x): (2/N) sum f sin(kx)."""
    return 2.0 * np.mean(field * np.sin(k * axis_coord))


def standard_d1q3_bgk(rho0, u0, tau_lb, nsteps, sample):
    """Textbook D1Q3 BGK with the second-order Hermite equilibrium
    f_i = w_i rho (1 + 3 e u + 9/2 (e u)^2 - 3/2 u^2), w = (2/3, 1/6, 1/6),
    e = (0, +1, -1), periodic streaming.  The populations start by streaming
    the local equilibrium of (rho0, u0).  Returns rho at the sample steps."""
    e = np.array([0, 1, -1])
    w = np.array([2 / 3, 1 / 6, 1 / 6])

    def eq(rho, u):
        eu = e[:, None] * u[None, :]
        return w[:, None] * rho[None, :] * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * u[None, :] ** 2)

    def stream(fs):
        return np.stack([np.roll(fs[i], e[i]) for i in range(3)])

    f = stream(eq(rho0, u0))
    out = {}
    if 0 in sample:
        out[0] = f.sum(0)
    for t in range(1, nsteps + 1):
        rho = f.sum(0)
        u = (f * e[:, None]).sum(0) / rho
        fs = f - (f - eq(rho, u)) / tau_lb
        f = stream(fs)
        if t in sample:
            out[t] = f.sum(0)
    return out
