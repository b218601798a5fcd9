"""Pins of the oracle's local building blocks against what the paper and the
mathematics fix (no GPU).

* velocity order: Appendix B (rows 2-4 of the transformation matrix);
* equilibria: the moment-matching conditions Eqs. 28-31 against the
  Maxwell-Boltzmann moments of Eq. 2 computed by Gauss-Hermite quadrature
  (independent of any closed form);
* discrete moments of f^eq, Eqs. 32-35, and the b^eq/P relation, Eq. 36;
* forcing projection: its moments must be 0, F, G (Eqs. 58-61);
* isotropic gradient: closed form of the stencil on plane waves, and exact
  antisymmetry (zero global sum).
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden_d3q19():
    rows = [list(map(int, l.split())) for l in open(os.path.join(GOLDEN, "d3q19_velocity_rows_table_m.txt"))
            if l.strip() and not l.startswith("#")]
    return np.array(rows).T  # (19, 3)


def expected_velocities(d):
    if d == 3:
        return golden_d3q19()
    if d == 2:  # rest, +x, +y, -x, -y, ++, +-, -+, --
        return np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0],
                         [1, 1, 0], [1, -1, 0], [-1, 1, 0], [-1, -1, 0]])
    return np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0]])


def sym(d, bvec):
    """nb-vector -> full symmetric d x d tensor (component order of the oracle)."""
    B = np.zeros((d, d))
    if d == 1:
        B[0, 0] = bvec[0]
    elif d == 2:
        B[0, 0], B[1, 1], B[0, 1] = bvec[0], bvec[1], bvec[2]
        B[1, 0] = B[0, 1]
    else:
        B[0, 0], B[1, 1], B[2, 2] = bvec[0], bvec[1], bvec[2]
        B[0, 1] = B[1, 0] = bvec[3]
        B[0, 2] = B[2, 0] = bvec[4]
        B[1, 2] = B[2, 1] = bvec[5]
    return B


def mb_moments_quadrature(d, rho, u, T, order=3):
    """Moments 0..3 of the Maxwell-Boltzmann distribution of Eq. 2 by
    tensor-product Gauss-Hermite quadrature (exact for these polynomials)."""
    x, wq = np.polynomial.hermite_e.hermegauss(8)  # weight exp(-x^2/2)
    wq = wq / np.sqrt(2 * np.pi)
    grids = np.meshgrid(*([x] * d), indexing="ij")
    W = np.ones_like(grids[0])
    for a in range(d):
        W = W * np.meshgrid(*([wq] * d), indexing="ij")[a]
    v = [u[a] + np.sqrt(T) * grids[a] for a in range(d)]
    M0 = rho * W.sum()
    M1 = np.array([rho * (W * v[a]).sum() for a in range(d)])
    M2 = np.array([[rho * (W * v[a] * v[b]).sum() for b in range(d)] for a in range(d)])
    M3 = np.array([[[rho * (W * v[a] * v[b] * v[c]).sum() for c in range(d)]
                    for b in range(d)] for a in range(d)])
    return M0, M1, M2, M3


def bump_moments(d, f, e, B):
    """Moments of the bump expansion, Eqs. 24-27."""
    E = e[:, :d].astype(np.float64)
    M0 = f.sum()
    M1 = (f[:, None] * E).sum(0)
    M2 = np.einsum("i,ia,ib->ab", f, E, E) + f.sum() * B
    M3 = (np.einsum("i,ia,ib,ic->abc", f, E, E, E)
          + np.einsum("i,ia,bc->abc", f, E, B)
          + np.einsum("i,ic,ab->abc", f, E, B)
          + np.einsum("i,ib,ca->abc", f, E, B))
    return M0, M1, M2, M3


@pytest.mark.parametrize("d", [1, 2, 3])
def test_velocity_order(d):
    e, w = oracle.lattice(d)
    np.testing.assert_array_equal(e, expected_velocities(d))
    assert abs(w.sum() - 1.0) < 1e-15


def test_d3q19_is_table_m():
    e, _ = oracle.lattice(3)
    np.testing.assert_array_equal(e, golden_d3q19())
    # 18 moving velocities, |e|^2 in {1, 2}, closed under inversion
    s = {tuple(v) for v in e}
    assert all(tuple(-np.array(v)) in s for v in s)
    assert sorted((e ** 2).sum(1).tolist()) == [0] + [1] * 6 + [2] * 12


@pytest.mark.parametrize("d", [1, 2, 3])
def test_weights_isotropy(d):
    """sum w = 1, sum w e e = delta/3, sum w e e e e = (dd+dd+dd)/9: the
    properties the gradient and the forcing projection rely on."""
    e, w = oracle.lattice(d)
    E = e[:, :d].astype(float)
    I = np.eye(d)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, E, E), I / 3, atol=1e-15)
    np.testing.assert_allclose(np.einsum("i,ia->a", w, E), 0, atol=1e-15)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, E, E, E, E)
    iso = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
           + np.einsum("ad,bc->abcd", I, I)) / 9
    np.testing.assert_allclose(m4, iso, atol=1e-15)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_equilibrium_matches_maxwell_boltzmann(d):
    """Eqs. 28-31: the bump expansion of (f^eq, b^eq) reproduces the MB
    moments of Eq. 2 through third order, for random (rho, u, T)."""
    rng = np.random.default_rng(100 + d)
    e = expected_velocities(d)
    for _ in range(40):
        rho = rng.uniform(0.3, 3.0)
        u = rng.uniform(-0.4, 0.4, size=d)
        T = rng.uniform(0.02, 1.2)
        f = oracle.feq(d, rho, u)
        B = sym(d, oracle.beq(d, u, T))
        got = bump_moments(d, f, e, B)
        ref = mb_moments_quadrature(d, rho, u, T)
        for g_, r_ in zip(got, ref):
            scale = rho * (1 + T) ** 1.5
            np.testing.assert_allclose(g_, r_, rtol=0, atol=1e-13 * scale)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_discrete_moments_of_feq(d):
    """Eqs. 32-35: sum f e e = rho(2uu + c^2 I)/3, sum f eee = rho c^2 (sym u I)/3."""
    rng = np.random.default_rng(7 + d)
    E = expected_velocities(d)[:, :d].astype(float)
    I = np.eye(d)
    for _ in range(20):
        rho = rng.uniform(0.5, 2.0)
        u = rng.uniform(-0.3, 0.3, size=d)
        f = oracle.feq(d, rho, u)
        np.testing.assert_allclose(f.sum(), rho, rtol=1e-14)
        np.testing.assert_allclose(f @ E, rho * u, atol=1e-14)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", f, E, E),
                                   rho * (2 * np.outer(u, u) + I) / 3, atol=1e-14)
        m3 = np.einsum("i,ia,ib,ic->abc", f, E, E, E)
        ref = rho * (np.einsum("bc,a->abc", I, u) + np.einsum("ab,c->abc", I, u)
                     + np.einsum("ca,b->abc", I, u)) / 3
        np.testing.assert_allclose(m3, ref, atol=1e-14)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_beq_pressure_relation(d):
    """Eq. 36 with P = rho T I (Appendix A componentwise): b^eq = T I + (uu - I)/3;
    at T = c^2/3 and u = 0 the bump has zero width (the delta-function limit)."""
    rng = np.random.default_rng(3)
    I = np.eye(d)
    for _ in range(10):
        u = rng.uniform(-0.3, 0.3, size=d)
        T = rng.uniform(0.05, 0.5)
        B = sym(d, oracle.beq(d, u, T))
        np.testing.assert_allclose(B, T * I + (np.outer(u, u) - I) / 3, atol=1e-15)
    np.testing.assert_allclose(oracle.beq(d, np.zeros(d), 1.0 / 3.0), 0.0, atol=1e-16)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_feq_collapse(d):
    """Reading R1: summing the D3Q19 equilibrium over e_z (u_z = 0) gives the
    D2Q9 one; summing D2Q9 over e_y (u_y = 0) gives D1Q3."""
    if d == 3:
        pytest.skip("3D is the source of the collapse")
    rng = np.random.default_rng(11)
    e_hi = expected_velocities(d + 1)
    e_lo = expected_velocities(d)
    for _ in range(20):
        rho = rng.uniform(0.5, 2.0)
        u = np.zeros(d + 1)
        u[:d] = rng.uniform(-0.3, 0.3, size=d)
        f_hi = oracle.feq(d + 1, rho, u)
        f_lo = oracle.feq(d, rho, u[:d])
        summed = np.zeros(len(e_lo))
        for i, v in enumerate(e_hi):
            j = [k for k, w in enumerate(e_lo) if tuple(w[:d]) == tuple(v[:d])][0]
            summed[j] += f_hi[i]
        np.testing.assert_allclose(summed, f_lo, atol=1e-15)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_forcing_moments(d):
    """Eqs. 58-61: sum Phi = 0, sum Phi e = F, sum Phi e e = G."""
    rng = np.random.default_rng(5)
    E = expected_velocities(d)[:, :d].astype(float)
    nb = oracle.n_b(d)
    for _ in range(20):
        F = rng.normal(size=d)
        G = rng.normal(size=nb)
        phi = oracle.forcing(d, F, G)
        np.testing.assert_allclose(phi.sum(), 0, atol=1e-14)
        np.testing.assert_allclose(phi @ E, F, atol=1e-14)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", phi, E, E), sym(d, G), atol=1e-14)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_gradient_plane_wave(d):
    """Reading R6 on phi = sin(kx + ly + mz): the lattice-weight central
    difference along x equals cos(theta) sin(k) [1/3 + (cos l + cos m)/3] in
    D3Q19, cos(theta) sin(k) [2/3 + cos(l)/3] in D2Q9 and cos(theta) sin(k)
    in D1Q3; in the long-wave limit it is the exact derivative."""
    nx, ny, nz = 16, (8 if d >= 2 else 1), (4 if d == 3 else 1)
    k, l, m = 2 * np.pi * 3 / nx, (2 * np.pi / ny if d >= 2 else 0), (2 * np.pi / nz if d == 3 else 0)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    th = k * x + l * y + m * z
    g = oracle.gradient(d, np.sin(th))
    if d == 3:
        ref = np.cos(th) * np.sin(k) * (1 / 3 + (np.cos(l) + np.cos(m)) / 3)
    elif d == 2:
        ref = np.cos(th) * np.sin(k) * (2 / 3 + np.cos(l) / 3)
    else:
        ref = np.cos(th) * np.sin(k)
    np.testing.assert_allclose(g[0], ref, atol=1e-14)
    # antisymmetric stencil: the gradient of any periodic field sums to zero
    rnd = np.random.default_rng(0).normal(size=(nz, ny, nx))
    assert abs(oracle.gradient(d, rnd).sum(axis=(1, 2, 3))).max() < 1e-12
