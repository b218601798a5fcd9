"""Pins of the oracle's standard-lattice comparator (no GPU).

The comparator is the textbook BGK scheme with the Hermite equilibrium of
Eq. 4 (lattice units, cs2 = 1/3, temperature T0).  Sec. I explains why it
cannot match the bump scheme: on nearest-neighbour lattices its third moment
is fixed at rho cs2 (u delta + ...), so the shear viscosity is rho cs2 tau
whatever T0 is (the first line of the standard momentum equation), while the
bump scheme's is rho T tau (Eq. 84).

* equilibrium moments: rho, rho u and rho (T I + u u), exactly;
* the 1D scheme equals an independent numpy D1Q3 BGK to round-off;
* shear waves decay at cs2 tau k^2 for T0 = 0.2 (the bump scheme at the same
  T0: T0 tau k^2) -- the paper's central contrast;
* sound travels at sqrt(T0) (pressure rho T0);
* mass and momentum are conserved to round-off;
* at T0 = cs2 the bump scheme reduces to the comparator to O(A^2) on D2Q9;
* between moving walls the comparator's plane Couette profile is exactly linear.
"""
import numpy as np
import pytest

import oracle
from _physics import fit_damped_mode, fit_exponential, mode_amplitude, standard_d1q3_bgk


@pytest.mark.parametrize("d", [1, 2, 3])
def test_std_equilibrium_moments(d):
    e, _ = oracle.lattice(d)
    e = e[:, :d].astype(float)
    rng = np.random.default_rng(20 + d)
    for _ in range(5):
        rho = 0.5 + rng.random()
        u = 0.3 * rng.standard_normal(d)
        T = 0.05 + 0.4 * rng.random()
        f = oracle.std_feq(d, rho, u, T)
        assert abs(f.sum() - rho) < 1e-14
        assert np.abs(f @ e - rho * u).max() < 1e-14
        P = np.einsum("i,ia,ib->ab", f, e, e)
        assert np.abs(P - rho * (T * np.eye(d) + np.outer(u, u))).max() < 1e-14


def test_std_1d_equals_textbook_bgk():
    """T0 = cs2: the comparator is the textbook D1Q3 BGK with relaxation time
    tau + 1/2 (same omega convention as the bump scheme)."""
    N, tau = 128, 0.7
    rng = np.random.default_rng(3)
    rho0 = 1 + 0.01 * rng.standard_normal(N)
    u0 = 0.02 * rng.standard_normal(N)
    ref = standard_d1q3_bgk(rho0, u0, tau + 0.5, 300, {300})
    s = oracle.Sim(1, N, tau=tau, T0=1 / 3, model="standard")
    s.init(rho0[None, None, :], u0[None, None, None, :], 1 / 3)
    s.step(300)
    r, _, _ = s.moments()
    assert np.abs(r[0, 0] - ref[300]).max() < 1e-13


@pytest.mark.parametrize("d,shape", [(2, (1, 4, 64)), (3, (2, 2, 64))])
def test_std_shear_viscosity_ignores_T(d, shape):
    """T0 = 0.2: the comparator's shear wave decays at tau k^2 / 3, the bump
    scheme's at T0 tau k^2 (Sec. I vs Eq. 84)."""
    T, tau = 0.2, 0.8
    nz, ny, nx = shape
    k = 2 * np.pi / nx
    x = np.arange(nx)[None, None, :] * np.ones(shape)
    u = np.zeros((d,) + shape)
    u[1] = 1e-3 * np.sin(k * x)
    rates = {}
    for model in ("standard", "bump"):
        s = oracle.Sim(d, nx, ny, nz, tau=tau, T0=T, model=model)
        s.init(1.0, u, T)
        ts, a = [], []
        for t in range(301):
            _, uu, _ = s.moments()
            ts.append(t)
            a.append(mode_amplitude(uu[1], k, x))
            s.step(1)
        rates[model] = fit_exponential(np.array(ts, float), np.array(a))
    assert abs(rates["standard"] / (tau * k * k / 3) - 1) < 5e-3
    assert abs(rates["bump"] / (T * tau * k * k) - 1) < 5e-3


def test_std_sound_speed():
    """Isothermal sound at T0 = 0.1 travels at sqrt(T0)."""
    N, T, tau = 128, 0.1, 0.6
    s = oracle.Sim(1, N, tau=tau, T0=T, model="standard")
    k = 2 * np.pi / N
    x = np.arange(N)[None, None, :]
    s.init(1 + 1e-4 * np.sin(k * x), np.zeros((1, 1, 1, N)), T)
    ts, a = [], []
    for t in range(1201):
        r, _, _ = s.moments()
        ts.append(t)
        a.append(mode_amplitude(r - 1, k, x))
        s.step(1)
    _, w = fit_damped_mode(np.array(ts, float), np.array(a), k * k * tau / 3, k * np.sqrt(T))
    assert abs(w / (k * np.sqrt(T)) - 1) < 1e-2


@pytest.mark.parametrize("d,shape", [(1, (1, 1, 50)), (2, (1, 9, 14)), (3, (5, 4, 6))])
def test_std_conservation(d, shape):
    rng = np.random.default_rng(30 + d)
    s = oracle.Sim(d, shape[2], shape[1], shape[0], tau=0.6, T0=0.15, model="standard")
    s.init(1 + 0.05 * rng.standard_normal(shape), 0.05 * rng.standard_normal((d,) + shape), 0.15)
    d0 = s.diagnostics()
    s.step(100)
    d1 = s.diagnostics()
    assert np.abs(d1[: d + 1] - d0[: d + 1]).max() / d0[0] < 1e-13


def test_bump_reduces_to_standard_at_cs2():
    """T0 = 1/3 and amplitude A = 1e-3: b^eq = O(A^2), so the bump scheme and
    the comparator agree to O(A^2) on D2Q9 (a 2D check of the standard-lattice
    limit); at T0 = 0.2 their shear viscosities differ and so do their
    velocities, at O(A)."""
    n, A = 32, 1e-3
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    k = 2 * np.pi / n
    rho = 1 + A * np.sin(k * x) * np.cos(2 * k * y)
    u = np.stack([A * np.sin(k * y), A * np.cos(k * x)])[:, None]
    out = {}
    for T in (1 / 3, 0.2):
        r = {}
        for model in ("bump", "standard"):
            s = oracle.Sim(2, n, n, tau=0.7, T0=T, model=model)
            s.init(rho[None], u, T)
            s.step(200)
            r[model] = s.moments()
        out[T] = (np.abs(r["bump"][0] - r["standard"][0]).max(), np.abs(r["bump"][1] - r["standard"][1]).max())
    assert max(out[1 / 3]) < 10 * A * A
    assert out[0.2][1] > 0.1 * A


def test_std_couette_linear_exact():
    """The comparator between moving half-way bounce-back walls: the plane
    Couette profile is exactly linear (the textbook property of this wall
    rule), as for the bump scheme."""
    H, U = 24, 0.02
    s = oracle.Sim(2, 1, H, tau=0.6, T0=1 / 3, bc="walls", model="standard")
    s.set_wall_velocity([0.0, 0.0], [U, 0.0])
    s.init(1.0, np.zeros((2, 1, H, 1)), 1 / 3)
    s.step(int(8 * H * H / (0.6 / 3)))
    _, u, _ = s.moments()
    z = np.arange(H) + 0.5
    assert np.abs(u[0].ravel() - U * z / H).max() < 1e-10 * U
