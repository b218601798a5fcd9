"""Half-way bounce-back walls (at rest or moving) and the uniform body force
on the GPU, against the FP64 oracle, through the C ABI (needs a GB300).

FP64 storage: 1e-12 norm-wise on rho, T and the emitted populations and
1e-12 absolute on u (units of c), as for the periodic lattices -- the wall
and force terms add a handful of operations per site, in the same order on
both sides up to fused multiply-adds.  FP32 storage: the Poiseuille viscosity
read off the profile agrees with the FP64 oracle's to 1e-3 relative.
"""
import numpy as np
import pytest

import oracle
from _parity import normwise

try:
    from paper_2501_00620_gb300 import lbm
except ImportError as _e:
    lbm = None
    _IMPORT_ERROR = _e

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(autouse=True)
def _library_loaded():
    if lbm is None:
        raise _IMPORT_ERROR


def pair(d, shape, fields, tau, T0, thermal, bc, acc, dtype="f64", uw=None, **kw):
    """GPU and oracle lattices from the same fields.  Wall velocities are set
    before the start: the oracle streams the start emission at init, the GPU
    in its first step, and both then see the same walls."""
    nz, ny, nx = shape
    g = lbm.Simulation(d, nx, ny, nz, tau=tau, T0=T0, bc=bc, dtype=dtype, thermal=thermal, **kw)
    o = oracle.Sim(d, nx, ny, nz, tau=tau, T0=T0, thermal=thermal, bc=bc)
    if uw is not None:
        g.set_wall_velocity(*uw)
        o.set_wall_velocity(*uw)
    g.init(*fields)
    o.init(*fields)
    if acc is not None:
        g.set_force(acc)
        o.set_force(acc)
    return g, o


def assert_parity(g, o):
    gr, gu, gT = g.moments()
    orr, ou, oT = o.moments()
    assert normwise(gr, orr) < TOL
    assert np.abs(gu - ou).max() < TOL
    assert normwise(gT, oT) < TOL
    gf, gb = g.emitted()
    of, ob = o.emitted()
    assert normwise(gf, of) < TOL
    assert np.abs(gb - ob).max() < TOL


def random_fields(d, shape, seed, T0):
    rng = np.random.default_rng(seed)
    rho = 1 + 0.05 * rng.random(shape)
    u = 0.03 * rng.standard_normal((d,) + shape)
    T = T0 * (1 + 0.05 * rng.random(shape))
    return rho, u, T


@pytest.mark.parametrize("thermal", [False, True])
@pytest.mark.parametrize("acc", [None, (2e-4, -1e-4)])
def test_walls_2d_fp64(thermal, acc):
    """D2Q9 channel 300 x 70 (walls normal to y; x tiles with a ragged tail,
    several chunks along y, so chunk edges meet the walls and the interior)."""
    shape = (1, 70, 300)
    g, o = pair(2, shape, random_fields(2, shape, 1, 0.1), 0.6, 0.1, thermal, "walls", acc)
    g.step(60)
    o.step(60)
    assert_parity(g, o)


@pytest.mark.parametrize("thermal", [False, True])
def test_walls_3d_fp64(thermal):
    """D3Q19 channel 40 x 20 x 24 (walls normal to z), forced along y."""
    shape = (24, 20, 40)
    g, o = pair(3, shape, random_fields(3, shape, 2, 0.05), 0.52, 0.05, thermal, "walls",
                (0.0, 1e-4, -5e-5))
    g.step(20)
    o.step(20)
    assert_parity(g, o)


@pytest.mark.parametrize("d,shape", [(1, (1, 1, 200)), (2, (1, 17, 40)), (3, (9, 7, 12))])
def test_force_periodic_fp64(d, shape):
    acc = np.array([3e-4, -2e-4, 1e-4])[:d]
    g, o = pair(d, shape, random_fields(d, shape, 3, 0.1), 0.7, 0.1, True, "periodic", acc)
    d0 = g.diagnostics()
    g.step(30)
    o.step(30)
    assert_parity(g, o)
    # total momentum grows by exactly M a per step
    d1 = g.diagnostics()
    assert np.allclose((d1[1:1 + d] - d0[1:1 + d]) / (30 * d0[0]), acc, rtol=1e-9, atol=0)


@pytest.mark.parametrize("d,shape", [(2, (1, 16, 24)), (3, (10, 6, 8))])
def test_walls_conserve_mass_fp64(d, shape):
    g, _ = pair(d, shape, random_fields(d, shape, 4, 0.1), 0.6, 0.1, True, "walls", [1e-4] * d)
    m0 = g.diagnostics()[0]
    g.step(300)
    assert abs(g.diagnostics()[0] / m0 - 1) < 1e-13


def test_poiseuille_fp32_matches_oracle_viscosity():
    """FP32 storage, D2Q9 channel 64 x 32, tau = 0.5, T = 0.1: the viscosity
    eta = rho a H^2 / (8 u_max) equals the FP64 oracle's (one column) to
    1e-3 and eta = rho T tau to 1%."""
    H, a, tau, T = 32, 1e-5, 0.5, 0.1
    steps = int(6 * H * H / (T * tau))
    g = lbm.Simulation(2, 64, H, tau=tau, T0=T, bc="walls", dtype="f32")
    g.init(1.0, np.zeros((2, 1, H, 64)), T)
    g.set_force([a, 0.0])
    g.step(steps)
    r, u, _ = g.moments()
    eta_g = r.mean() * a * H * H / (8 * u[0].max())
    o = oracle.Sim(2, 1, H, tau=tau, T0=T, bc="walls")
    o.init(1.0, np.zeros((2, 1, H, 1)), T)
    o.set_force([a, 0.0])
    o.step(steps)
    ro, uo, _ = o.moments()
    eta_o = ro.mean() * a * H * H / (8 * uo[0].max())
    assert abs(eta_g / eta_o - 1) < 1e-3
    assert abs(eta_g / (r.mean() * T * tau) - 1) < 1e-2
    # uniform in x
    assert np.abs(u[0] - u[0][:, :, :1]).max() < 1e-6 * np.abs(u[0]).max() + 1e-9


def test_force_switches_to_kernels_with_the_force():
    """A forced lattice runs on a kernel that implements the force: setting a
    force on a tuned periodic FP32 lattice re-tunes among the generic kernel
    and the staged kernel's force/MRT tile, and the momentum then grows by
    M a per step; a walled lattice whose extents the walls tile does not
    divide runs on the generic kernel."""
    n = 64
    g = lbm.Simulation(3, n, n, n, tau=0.6, T0=0.1, dtype="f32")
    g.init(1.0, np.zeros((3, n, n, n)), 0.1)
    g.step(2)
    assert g.launch_config()[0] != EXT_TILE
    acc = np.array([1e-4, 0.0, -2e-4])
    g.set_force(acc)
    d0 = g.diagnostics()
    g.step(10)
    tile, _, kernel = g.launch_config()
    assert kernel == "step_kernel" or tile == EXT_TILE
    d1 = g.diagnostics()
    assert np.allclose((d1[1:4] - d0[1:4]) / (10 * d0[0]), acc, rtol=1e-4, atol=1e-9)
    w = lbm.Simulation(2, 250, 64, tau=0.6, T0=0.1, bc="walls", dtype="f32")
    w.init(1.0, np.zeros((2, 1, 64, 250)), 0.1)
    w.step(1)
    assert w.launch_config()[2] == "step_kernel"  # 250 is no multiple of the walls tile's 128


EXT_TILE = 150  # the staged kernel's force/MRT tile


@pytest.mark.parametrize("d,shape", [(3, (20, 32, 64)), (3, (9, 16, 96)), (2, (1, 40, 256)), (2, (1, 17, 384))])
def test_staged_force_tile_matches_generic_and_oracle(d, shape):
    """The staged kernel's force/MRT tile with a body force: equal to the
    generic kernel up to FP32 rounding after several steps (chunk lengths
    that do and do not divide the march), and one step from an identical
    state equal to the FP64 oracle to the FP32 storage precision."""
    nz, ny, nx = shape
    rho, u, T = random_fields(d, shape, 31, 0.1)
    acc = [2e-4, -1e-4, 5e-5][:d]
    ref = lbm.Simulation(d, nx, ny, nz, tau=0.6, T0=0.1, thermal=True, dtype="f32", tile=0, chunk=4)
    ref.set_force(acc)
    ref.init(rho, u, T)
    ref.step(7)
    fr, br = ref.emitted()
    for chunk in (3, 8):
        g = lbm.Simulation(d, nx, ny, nz, tau=0.6, T0=0.1, thermal=True, dtype="f32", tile=EXT_TILE, chunk=chunk)
        g.set_force(acc)
        g.init(rho, u, T)
        g.step(6)
        assert g.launch_config()[0] == EXT_TILE
        f0, b0 = g.emitted()
        g.step(1)
        f1, b1 = g.emitted()
        assert normwise(f1, fr) < 2e-5 and np.abs(b1 - br).max() < 2e-5
        o = oracle.Sim(d, nx, ny, nz, tau=0.6, T0=0.1, thermal=True)
        o.set_force(acc)
        o.set_emitted(f0, b0)
        o.step(1)
        of, ob = o.emitted()
        assert normwise(f1, of) < 2e-6 and np.abs(b1 - ob).max() < 2e-6


WALL_TILE = 151  # the staged kernel's walls tile


@pytest.mark.parametrize("moving", [False, True])
@pytest.mark.parametrize("d,shape", [(3, (20, 32, 64)), (3, (9, 16, 96)), (2, (1, 40, 256)), (2, (1, 17, 384))])
def test_staged_walls_tile_matches_generic_and_oracle(d, shape, moving):
    """The staged kernel's walls tile (half-way bounce-back at the first and
    last plane of the march, the site's own variance on bounced populations,
    image planes beyond the walls for the gradient; a body force; walls at
    rest or moving): equal to the generic kernel on FP32 storage after
    several steps, over chunk lengths that do and do not divide the march
    (chunk ends at the walls and inside); one step from an identical state
    equal to the FP64 oracle to the FP32 storage precision."""
    nz, ny, nx = shape
    rho, u, T = random_fields(d, shape, 41, 0.1)
    acc = [2e-4, -1e-4, 0.0][:d]
    # tangential wall velocities: the upper wall moves along x (and y in 3D)
    uw = ([0.0] * d, [0.02, -0.01, 0.0] if d == 3 else [0.02, 0.0]) if moving else None

    def make(tile, chunk):
        g = lbm.Simulation(d, nx, ny, nz, tau=0.6, T0=0.1, thermal=True, bc="walls", dtype="f32", tile=tile,
                           chunk=chunk)
        if uw is not None:
            g.set_wall_velocity(*uw)
        g.set_force(acc)
        g.init(rho, u, T)
        return g

    ref = make(0, 4)
    ref.step(7)
    fr, br = ref.emitted()
    for chunk in (3, 8):
        g = make(WALL_TILE, chunk)
        g.step(6)
        assert g.launch_config()[0] == WALL_TILE
        f0, b0 = g.emitted()
        g.step(1)
        f1, b1 = g.emitted()
        assert normwise(f1, fr) < 2e-5 and np.abs(b1 - br).max() < 2e-5
        o = oracle.Sim(d, nx, ny, nz, tau=0.6, T0=0.1, thermal=True, bc="walls")
        if uw is not None:
            o.set_wall_velocity(*uw)
        o.set_force(acc)
        o.set_emitted(f0, b0)
        o.step(1)
        of, ob = o.emitted()
        assert normwise(f1, of) < 2e-6 and np.abs(b1 - ob).max() < 2e-6


def test_walled_fp32_lattice_tunes_onto_the_walls_tile():
    """The autotuner times the walls tile beside the generic kernel's tiles
    for a walled FP32 lattice and keeps the faster (the walls tile on a
    256 x 64 x 32 channel)."""
    g = lbm.Simulation(3, 256, 64, 32, tau=0.6, T0=0.1, bc="walls", dtype="f32")
    g.init(1.0, np.zeros((3, 32, 64, 256)), 0.1)
    g.set_force([1e-5, 0.0, 0.0])
    g.step(2)
    assert g.launch_config()[0] == WALL_TILE


@pytest.mark.parametrize("d,shape", [(2, (1, 23, 70)), (3, (13, 11, 37))])
def test_walls_chunks_bitwise(d, shape):
    """Chunk lengths along the wall-normal axis (1, 5 and the whole axis)
    give the same bits: the wall images at chunk ends and lattice ends are
    the same numbers."""
    rho, u, T = random_fields(d, shape, 5, 0.1)
    ref = None
    for chunk in (1, 5, 64):
        g = lbm.Simulation(d, shape[2], shape[1], shape[0], tau=0.6, T0=0.1, thermal=True, bc="walls",
                           tile=0, chunk=chunk)
        g.init(rho, u, T)
        g.set_force([1e-4] * d)
        g.set_wall_velocity([0.02] + [0.0] * (d - 1), [-0.01] + [0.0] * (d - 1))
        g.step(9)
        f, b = g.emitted()
        if ref is None:
            ref = (f, b)
        else:
            assert np.array_equal(f, ref[0]) and np.array_equal(b, ref[1])


@pytest.mark.parametrize("thermal", [False, True])
@pytest.mark.parametrize("d", [2, 3])
def test_moving_walls_fp64(d, thermal):
    """Moving walls (Sec. III.D) with a force normal to them, against the
    oracle: the bounced populations' wall momentum and the reflected image
    velocity."""
    shape = (1, 70, 300) if d == 2 else (24, 20, 40)
    steps = 60 if d == 2 else 20
    acc = (1e-4, -2e-4) if d == 2 else (0.0, 1e-4, -2e-4)
    lo = (0.02, 0.0) if d == 2 else (0.01, 0.02, 0.0)
    hi = (-0.01, 0.0) if d == 2 else (-0.01, 0.0, 0.0)
    g, o = pair(d, shape, random_fields(d, shape, 6, 0.1), 0.6, 0.1, thermal, "walls", acc, uw=(lo, hi))
    g.step(steps)
    o.step(steps)
    assert_parity(g, o)


def test_couette_gravity_fp32_matches_oracle():
    """FP32 storage, D2Q9 channel 64 x 32, walls at 0 and U, gravity normal
    to them: the steady profile equals the FP64 oracle's (one column) to
    1e-3 U."""
    H, U, T, tau, g = 32, 0.02, 0.1, 0.6, -1e-3
    steps = int(8 * H * H / (T * tau))
    sim = lbm.Simulation(2, 64, H, tau=tau, T0=T, bc="walls", dtype="f32")
    sim.set_wall_velocity([0.0, 0.0], [U, 0.0])
    sim.init(1.0, np.zeros((2, 1, H, 64)), T)
    sim.set_force([0.0, g])
    sim.step(steps)
    _, u, _ = sim.moments()
    o = oracle.Sim(2, 1, H, tau=tau, T0=T, bc="walls")
    o.set_wall_velocity([0.0, 0.0], [U, 0.0])
    o.init(1.0, np.zeros((2, 1, H, 1)), T)
    o.set_force([0.0, g])
    o.step(steps)
    _, uo, _ = o.moments()
    assert np.abs(u[0] - uo[0]).max() < 1e-3 * U


def test_wall_velocity_rejects_normal_component_and_no_walls():
    w = lbm.Simulation(2, 16, 16, bc="walls")
    with pytest.raises(Exception):
        w.set_wall_velocity([0.0, 0.01], [0.0, 0.0])
    p = lbm.Simulation(2, 16, 16)
    with pytest.raises(Exception):
        p.set_wall_velocity([0.01, 0.0], [0.0, 0.0])


def test_walls_reject_1d():
    with pytest.raises(Exception):
        lbm.Simulation(1, 64, bc="walls")
