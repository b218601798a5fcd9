"""The MRT collision (Appendix B, Table M basis) on the GPU against the FP64
oracle, through the C ABI (needs a GB300).

FP64 storage: 1e-12 norm-wise on rho, T and the emitted populations and
1e-12 absolute on u, as for the SRT step.  FP32 storage: one step from an
identical emitted state agrees to 2e-6 of the population scale.
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


def fields(shape, seed, T0):
    rng = np.random.default_rng(seed)
    return (1 + 0.05 * rng.random(shape), 0.05 * rng.standard_normal((3,) + shape),
            T0 * (1 + 0.05 * rng.random(shape)))


@pytest.mark.parametrize("thermal,bc", [(False, "periodic"), (True, "periodic"), (True, "walls")])
def test_mrt_fp64_parity(thermal, bc):
    """D3Q19 40 x 20 x 24 (ragged tiles, several chunks), rates s3 = 1.3,
    s4 = 1.6, a body force, 20 steps."""
    shape = (24, 20, 40)
    fl = fields(shape, 21, 0.1)
    g = lbm.Simulation(3, 40, 20, 24, tau=0.6, T0=0.1, bc=bc, thermal=thermal)
    o = oracle.Sim(3, 40, 20, 24, tau=0.6, T0=0.1, thermal=thermal, bc=bc)
    for x in (g, o):
        x.set_mrt(1.3, 1.6)
        x.init(*fl)
        x.set_force([1e-4, -5e-5, 2e-5] if bc == "periodic" else [1e-4, -5e-5, 0.0])
    g.step(20)
    o.step(20)
    assert g.launch_config()[2] == "step_kernel"
    gr, gu, gT = g.moments()
    orr, ou, oT = o.moments()
    assert normwise(gr, orr) < TOL
    assert np.abs(gu - ou).max() < TOL
    assert normwise(gT, oT) < TOL
    gf, gb = g.emitted()
    of, ob = o.emitted()
    assert normwise(gf, of) < TOL
    assert np.abs(gb - ob).max() < TOL


def test_mrt_equal_rates_is_srt_on_gpu():
    shape = (13, 11, 37)
    fl = fields(shape, 22, 0.1)
    out = []
    for mrt in (False, True):
        g = lbm.Simulation(3, 37, 11, 13, tau=0.6, T0=0.1, thermal=True, tile=0, chunk=5)
        if mrt:
            g.set_mrt(1 / 1.1, 1 / 1.1)
        g.init(*fl)
        g.step(15)
        out.append(g.emitted()[0])
    assert np.abs(out[0] - out[1]).max() < 1e-13


def test_mrt_fp32_one_step():
    shape = (16, 16, 32)
    fl = fields(shape, 23, 0.1)
    o = oracle.Sim(3, 32, 16, 16, tau=0.6, T0=0.1)
    o.set_mrt(1.2, 1.5)
    o.init(*fl)
    f0, b0 = o.emitted()
    g = lbm.Simulation(3, 32, 16, 16, tau=0.6, T0=0.1, dtype="f32")
    g.set_mrt(1.2, 1.5)
    g.init(*fl)
    g.set_emitted(f0, b0)
    o.set_emitted(f0, b0)
    g.step(1)
    o.step(1)
    tile, _, kernel = g.launch_config()
    assert kernel == "step_kernel" or tile == EXT_TILE
    assert normwise(g.emitted()[0], o.emitted()[0]) < 2e-6


EXT_TILE = 150  # the staged kernel's force/MRT tile


@pytest.mark.parametrize("force", [False, True])
@pytest.mark.parametrize("shape", [(20, 32, 64), (9, 16, 96)])
def test_mrt_staged_tile_matches_generic_and_oracle(shape, force):
    """The staged kernel's force/MRT tile with the MRT collision (and a body
    force): equal to the generic kernel up to FP32 rounding after several
    steps, over chunk lengths that do and do not divide the march; one step
    from an identical state equal to the FP64 oracle to the FP32 storage
    precision."""
    nz, ny, nx = shape
    fl = fields(shape, 24, 0.1)
    acc = [1e-4, -5e-5, 2e-5]

    def make(tile, chunk):
        g = lbm.Simulation(3, nx, ny, nz, tau=0.6, T0=0.1, thermal=True, dtype="f32", tile=tile, chunk=chunk)
        g.set_mrt(1.2, 1.5)
        if force:
            g.set_force(acc)
        g.init(*fl)
        return g

    ref = make(0, 4)
    ref.step(7)
    fr, br = ref.emitted()
    for chunk in (3, 8):
        g = make(EXT_TILE, chunk)
        g.step(6)
        assert g.launch_config()[0] == EXT_TILE
        f0, b0 = g.emitted()
        g.step(1)
        f1, b1 = g.emitted()
        assert normwise(f1, fr) < 2e-5 and np.abs(b1 - br).max() < 2e-5
        o = oracle.Sim(3, nx, ny, nz, tau=0.6, T0=0.1, thermal=True)
        o.set_mrt(1.2, 1.5)
        if force:
            o.set_force(acc)
        o.set_emitted(f0, b0)
        o.step(1)
        of, ob = o.emitted()
        assert normwise(f1, of) < 2e-6 and np.abs(b1 - ob).max() < 2e-6


def test_mrt_rejects_other_lattices():
    with pytest.raises(Exception):
        lbm.Simulation(2, 16, 16).set_mrt(1.2, 1.2)
    with pytest.raises(Exception):
        lbm.Simulation(3, 8, 8, 8, model="standard").set_mrt(1.2, 1.2)
    with pytest.raises(Exception):
        lbm.Simulation(3, 8, 8, 8).set_mrt(2.5, 1.2)
