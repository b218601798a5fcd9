"""Pins of the oracle's half-way bounce-back walls and body force (no GPU).

Sec. III.A measures the shear viscosity in Poiseuille flow: a uniform
acceleration a drives the fluid between two stationary half-step bounce-back
walls, the steady profile is the parabola u(z) = rho a z (H - z) / (2 eta),
and the viscosity read off its maximum, eta = rho a H^2 / (8 u_max), follows
eta = rho T tau (Eq. 84) -- a line in T of slope rho tau.  The walls sit half a
site outside the lattice, so z is measured from -1/2.

* uniform force on a periodic lattice: total momentum grows by exactly M a per
  step and the fluid velocity is a (t + 1/2) (the corrected velocity of
  Eq. 57 carries half a step of force); in thermal mode the work of the force
  appears as kinetic energy alone, so T stays at its start value;
* walls conserve mass to round-off;
* Poiseuille: eta / (rho T tau) within 1% at H = 32 over several (T, tau),
  the slope of eta(T) equal to rho tau, and the error falling as 1/H^2;
* D2Q9 (walls normal to y) and D3Q19 (walls normal to z, uniform in x, y)
  give the same profile, which ties the two wall paths together;
* hydrostatics with the force normal to the walls: T d(rho)/dz = rho a_z
  (the z-equation of the Couette problem of Sec. III.D), rho ~ exp(a z / T);
* moving walls (Sec. III.D): plane Couette flow is the exact linear profile;
  with gravity normal to the walls the profile follows the closed form
  u = u_b + (u_t - u_b) (1 - exp(-a z / T)) / (1 - exp(-a H / T)), and the
  frame shift (0, U) -> (-U/2, U/2) moves the profile by -U/2 only;
* the standard-lattice comparator in the same channel has eta = rho tau / 3
  whatever T is (Sec. I) -- the contrast to eta = rho T tau above.

A planted mistake in the wall image of the gradient stencil (u0 not reversed)
moves eta / (rho T tau) at T = 0.1 by about 9%, far outside these bounds.
"""
import numpy as np
import pytest

import oracle


def poiseuille(d, H, tau, T, a=1e-6, steps=None, model="bump"):
    if d == 2:
        s = oracle.Sim(2, 1, H, tau=tau, T0=T, bc="walls", model=model)
        shape = (1, H, 1)
    else:
        s = oracle.Sim(3, 1, 1, H, tau=tau, T0=T, bc="walls")
        shape = (H, 1, 1)
    s.init(1.0, np.zeros((d,) + shape), T)
    s.set_force([a] + [0.0] * (d - 1))
    nu = T * tau
    s.step(steps if steps is not None else int(6 * H * H / nu))  # ~ 6 diffusion times
    rho, u, _ = s.moments()
    return rho.ravel(), u[0].ravel(), u


def test_uniform_force_momentum_growth():
    """Periodic, uniform state, uniform a: P(t) - P(0) = t M a exactly and
    u(t) = a (t + 1/2) at every site."""
    s = oracle.Sim(2, 8, 6, tau=0.6, T0=0.2)
    s.init(1.0, np.zeros((2, 1, 6, 8)), 0.2)
    a = np.array([1e-5, -2e-5])
    s.set_force(a)
    d0 = s.diagnostics()
    s.step(10)
    d1 = s.diagnostics()
    assert np.allclose((d1[1:3] - d0[1:3]) / (10 * d0[0]), a, rtol=1e-10, atol=0)
    _, u, _ = s.moments()
    assert np.allclose(u, a[:, None, None, None] * 10.5, rtol=1e-10, atol=0)


def test_uniform_force_thermal_temperature_constant():
    """Thermal mode: the force's second-moment source rho (u a + a u) with the
    corrected u makes the energy grow by the kinetic energy alone, so the
    moment temperature stays at its start value T0 + |a|^2 / (4 d) (the
    offset: the start emits u = 0 while the reported u carries a/2)."""
    d = 2
    s = oracle.Sim(d, 8, 8, tau=0.6, T0=0.2, thermal=True)
    s.init(1.0, np.zeros((2, 1, 8, 8)), 0.2)
    a = np.array([3e-4, -2e-4])
    s.set_force(a)
    _, _, T0 = s.moments()
    s.step(50)
    _, u, T = s.moments()
    assert np.allclose(u, a[:, None, None, None] * 50.5, rtol=1e-10, atol=0)
    assert np.abs(T0 - (0.2 + a @ a / (4 * d))).max() < 1e-15
    assert np.abs(T - T0).max() < 1e-14


@pytest.mark.parametrize("d,shape", [(2, (1, 12, 10)), (3, (7, 5, 6))])
def test_walls_conserve_mass(d, shape):
    rng = np.random.default_rng(10 + d)
    nz, ny, nx = shape
    s = oracle.Sim(d, nx, ny, nz, tau=0.6, T0=0.1, thermal=True, bc="walls")
    s.init(1 + 0.1 * rng.normal(size=shape), 0.05 * rng.normal(size=(d,) + shape),
           0.1 * (1 + 0.1 * rng.normal(size=shape)))
    s.set_force(1e-4 * rng.normal(size=d))
    m0 = s.diagnostics()[0]
    s.step(200)
    assert abs(s.diagnostics()[0] / m0 - 1) < 1e-13


@pytest.mark.parametrize("tau,T", [(0.5, 0.1), (1.0, 0.1), (0.5, 0.2), (0.5, 0.3), (1.0, 0.2)])
def test_poiseuille_viscosity(tau, T):
    """eta = rho a H^2 / (8 u_max) against eta = rho T tau, H = 32; the whole
    profile against the parabola."""
    H, a = 32, 1e-6
    rho, ux, _ = poiseuille(2, H, tau, T, a)
    eta = rho.mean() * a * H * H / (8 * ux.max())
    assert abs(eta / (rho.mean() * T * tau) - 1) < 1e-2
    z = np.arange(H) + 0.5
    exact = a * z * (H - z) / (2 * T * tau)
    assert np.abs(ux - exact).max() / exact.max() < 1.5e-2


def test_poiseuille_viscosity_slope():
    """eta(T) is a line of slope rho tau (Sec. III.A, Fig. 4c), tau = 0.5, 1."""
    H, a = 32, 1e-6
    Ts = np.array([0.1, 0.2, 0.3])
    for tau in (0.5, 1.0):
        eta = []
        for T in Ts:
            rho, ux, _ = poiseuille(2, H, tau, T, a)
            eta.append(rho.mean() * a * H * H / (8 * ux.max()))
        slope = np.polyfit(Ts, eta, 1)[0]
        assert abs(slope / tau - 1) < 1e-2


def test_poiseuille_second_order_in_H():
    """Half-way bounce-back is second order: the viscosity error at H = 16 is
    about four times the one at H = 32."""
    err = []
    for H in (16, 32):
        rho, ux, _ = poiseuille(2, H, 0.5, 0.1)
        err.append(rho.mean() * 1e-6 * H * H / (8 * ux.max()) / (0.1 * 0.5) - 1)
    assert 3.0 < err[0] / err[1] < 5.0


def test_walls_collapse_2d_3d():
    """The D3Q19 channel (walls normal to z, uniform in x, y) equals the D2Q9
    channel (walls normal to y, uniform in x): same rho and velocity profile."""
    H = 12
    r2, u2, _ = poiseuille(2, H, 0.6, 0.15, a=1e-4, steps=800)
    r3, u3, _ = poiseuille(3, H, 0.6, 0.15, a=1e-4, steps=800)
    assert np.abs(r2 - r3).max() < 1e-13
    assert np.abs(u2 - u3).max() / np.abs(u2).max() < 1e-11


def test_hydrostatic_profile():
    """Force normal to the walls, isothermal: at rest T d(rho)/dz = rho a_z,
    so log rho is a line of slope a_z / T (interior sites, 2% tolerance: the
    wall image holds rho b, i.e. the pressure, constant across the wall)."""
    H, T, a = 32, 0.2, -2e-3
    s = oracle.Sim(2, 1, H, tau=0.6, T0=T, bc="walls")
    s.init(1.0, np.zeros((2, 1, H, 1)), T)
    s.set_force([0.0, a])
    s.step(20000)
    rho, u, _ = s.moments()
    rho = rho.ravel()
    z = np.arange(H) + 0.5
    slope = np.polyfit(z[2:-2], np.log(rho[2:-2]), 1)[0]
    assert abs(slope / (a / T) - 1) < 2e-2
    assert np.abs(u).max() < 1e-3 * abs(a) * H


def couette(d, H, tau, T, ub, ut, g, steps=None):
    """Walls moving along x (2D) / y (3D) at ub (lower) and ut (upper),
    gravity g along the wall normal; returns rho and the wall-parallel u."""
    if d == 2:
        s = oracle.Sim(2, 1, H, tau=tau, T0=T, bc="walls")
        s.init(1.0, np.zeros((2, 1, H, 1)), T)
        s.set_wall_velocity([ub, 0.0], [ut, 0.0])
        s.set_force([0.0, g])
    else:
        s = oracle.Sim(3, 1, 1, H, tau=tau, T0=T, bc="walls")
        s.init(1.0, np.zeros((3, H, 1, 1)), T)
        s.set_wall_velocity([0.0, ub, 0.0], [0.0, ut, 0.0])
        s.set_force([0.0, 0.0, g])
    s.step(steps if steps is not None else int(8 * H * H / (T * tau)))
    rho, u, _ = s.moments()
    return rho.ravel(), (u[0] if d == 2 else u[1]).ravel()


def test_couette_linear_exact():
    H, U = 32, 0.02
    _, u = couette(2, H, 0.6, 0.1, 0.0, U, 0.0)
    z = np.arange(H) + 0.5
    assert np.abs(u - U * z / H).max() < 1e-10 * U


def test_couette_gravity_closed_form_and_frame_shift():
    """Sec. III.D: T = 0.1, a_z = -1e-3 (density ratio 1.35 across the
    channel).  Profile within 1.5% of U of the closed form; the shifted frame
    within 1% of U of the shifted profile."""
    H, U, T, g = 32, 0.02, 0.1, -1e-3
    z = np.arange(H) + 0.5
    _, ua = couette(2, H, 0.6, T, 0.0, U, g)
    _, ub = couette(2, H, 0.6, T, -U / 2, U / 2, g)
    k = g / T
    exact = U * (1 - np.exp(-k * z)) / (1 - np.exp(-k * H))
    assert np.abs(ua - exact).max() < 1.5e-2 * U
    assert np.abs(ub + U / 2 - ua).max() < 1e-2 * U


def test_couette_3d_equals_2d():
    r2, u2 = couette(2, 12, 0.6, 0.15, -0.01, 0.02, -1e-3, steps=600)
    r3, u3 = couette(3, 12, 0.6, 0.15, -0.01, 0.02, -1e-3, steps=600)
    assert np.abs(r2 - r3).max() < 1e-13
    assert np.abs(u2 - u3).max() < 1e-13


@pytest.mark.parametrize("T", [0.2, 1 / 3])
def test_standard_poiseuille_viscosity_ignores_T(T):
    """The comparator (textbook BGK, Eq. 4) in the same channel: eta = rho tau / 3
    at T0 = 0.2 and 1/3, against the bump scheme's rho T tau."""
    H, a, tau = 32, 1e-6, 0.5
    rho, ux, _ = poiseuille(2, H, tau, T, a, steps=int(6 * H * H / (tau / 3)), model="standard")
    eta = rho.mean() * a * H * H / (8 * ux.max())
    assert abs(eta / (rho.mean() * tau / 3) - 1) < 1.5e-2
