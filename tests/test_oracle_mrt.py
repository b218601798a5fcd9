"""Pins of the oracle's MRT collision in the moment basis of Table M
(Appendix B), D3Q19 (no GPU).

* the matrix is the printed table (golden transcription), its rows 1-3 are
  the velocity components and rows 4-9 the second-order Hermite moments
  e_a e_b - delta_ab / 3; the rows are orthogonal under the weighted sum
  sum_i w_i m^a_i m^b_i (what makes f_i = w_i sum_a m^a_i N^a M^a with
  N^a = 1 / sum_i w_i (m^a_i)^2 the inverse) and the matrix has rank 19;
* with the third- and fourth-order rates equal to omega the MRT step is the
  SRT step (Eq. 55) to round-off;
* with other rates it still conserves mass, momentum and (thermal mode)
  energy, and the long-wave shear viscosity is still rho T tau (Eq. 84):
  only the second-order rows carry it.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "d3q19_moment_matrix_table_m.txt")


def golden_table_m():
    rows = []
    with open(GOLDEN) as fh:
        for ln in fh:
            if ln.strip() and not ln.startswith("#"):
                rows.append([float(Fraction(t)) for t in ln.split()])
    return np.array(rows)


def test_table_m_structure():
    m = oracle.moment_matrix()
    np.testing.assert_array_equal(m, golden_table_m())
    e, w = oracle.lattice(3)
    np.testing.assert_array_equal(m[0], np.ones(19))
    np.testing.assert_array_equal(m[1:4], e.T)
    E = e.astype(float)
    second = [E[:, 0] ** 2 - 1 / 3, E[:, 1] ** 2 - 1 / 3, E[:, 2] ** 2 - 1 / 3,
              E[:, 0] * E[:, 1], E[:, 0] * E[:, 2], E[:, 1] * E[:, 2]]
    np.testing.assert_allclose(m[4:10], np.array(second), atol=1e-15)
    G = m @ np.diag(w) @ m.T
    assert np.abs(G - np.diag(np.diag(G))).max() < 1e-15
    assert np.linalg.matrix_rank(m) == 19


def random_3d(shape, seed, T0):
    rng = np.random.default_rng(seed)
    return (1 + 0.05 * rng.random(shape), 0.05 * rng.standard_normal((3,) + shape),
            T0 * (1 + 0.05 * rng.random(shape)))


@pytest.mark.parametrize("thermal", [False, True])
def test_mrt_with_equal_rates_is_srt(thermal):
    shape = (5, 6, 7)
    fields = random_3d(shape, 1, 0.1)
    out = []
    for mrt in (False, True):
        s = oracle.Sim(3, 7, 6, 5, tau=0.6, T0=0.1, thermal=thermal)
        if mrt:
            s.set_mrt(1 / 1.1, 1 / 1.1)   # omega = 1 / (tau + 1/2)
        s.init(*fields)
        s.set_force([1e-4, 0.0, -1e-4])
        s.step(40)
        out.append(s.emitted()[0])
    assert np.abs(out[0] - out[1]).max() < 1e-13


def test_mrt_conserves():
    shape = (5, 6, 7)
    s = oracle.Sim(3, 7, 6, 5, tau=0.6, T0=0.1, thermal=True)
    s.set_mrt(1.3, 1.6)
    s.init(*random_3d(shape, 2, 0.1))
    d0 = s.diagnostics()
    s.step(100)
    d1 = s.diagnostics()
    assert np.abs(d1[:4] - d0[:4]).max() / d0[0] < 1e-13
    assert abs(d1[4] / d0[4] - 1) < 1e-12


def test_mrt_shear_viscosity_unchanged():
    """Shear wave u_y = A sin(kx) at T = 0.2, tau = 0.8: decay rate T tau k^2
    with the higher-order rates far from omega."""
    from _physics import fit_exponential, mode_amplitude
    T, tau, nx = 0.2, 0.8, 64
    shape = (2, 2, nx)
    s = oracle.Sim(3, nx, 2, 2, tau=tau, T0=T)
    s.set_mrt(1.5, 1.2)
    k = 2 * np.pi / nx
    x = np.arange(nx)[None, None, :] * np.ones(shape)
    u = np.zeros((3,) + shape)
    u[1] = 1e-3 * np.sin(k * x)
    s.init(1.0, u, T)
    ts, a = [], []
    for t in range(301):
        _, uu, _ = s.moments()
        ts.append(t)
        a.append(mode_amplitude(uu[1], k, x))
        s.step(1)
    g = fit_exponential(np.array(ts, float), np.array(a))
    assert abs(g / (T * tau * k * k) - 1) < 5e-3


def test_mrt_rejects_other_lattices():
    with pytest.raises(ValueError):
        oracle.Sim(2, 8, 8).set_mrt(1.2, 1.2)
    with pytest.raises(ValueError):
        oracle.Sim(3, 4, 4, 4, model="standard").set_mrt(1.2, 1.2)
