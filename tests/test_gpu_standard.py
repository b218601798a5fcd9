"""The standard-lattice comparator on the GPU against the FP64 oracle,
through the C ABI (needs a GB300).

FP64 storage: 1e-12 norm-wise on rho, T and the emitted populations and 1e-12
absolute on u, as for the bump scheme.  FP32 storage at the size the
benchmark times (D3Q19 256^3): sampled windows advanced one step by the
oracle agree to 2e-6 of the population scale.
"""
import numpy as np
import pytest

import oracle
from _parity import check_windows, normwise
from paper_2501_00620_gb300 import workloads as W

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


def fields(d, shape, seed, T):
    rng = np.random.default_rng(seed)
    return (1 + 0.05 * rng.random(shape), 0.05 * rng.standard_normal((d,) + shape),
            T * (1 + 0.05 * rng.random(shape)))


@pytest.mark.parametrize("d,shape,T0", [(1, (1, 1, 300), 1 / 3), (2, (1, 70, 300), 0.25),
                                        (3, (24, 20, 40), 1 / 3)])
def test_standard_fp64_parity(d, shape, T0):
    """Ragged extents (no tile divides them); 50 steps; moments, emitted
    populations and the conservation diagnostics."""
    nz, ny, nx = shape
    fl = fields(d, shape, 7 + d, T0)
    g = lbm.Simulation(d, nx, ny, nz, tau=0.6, T0=T0, dtype="f64", model="standard")
    g.init(*fl)
    o = oracle.Sim(d, nx, ny, nz, tau=0.6, T0=T0, model="standard")
    o.init(*fl)
    g.step(50)
    o.step(50)
    assert g.launch_config()[2] == "std_step_kernel"
    gr, gu, gT = g.moments()
    orr, ou, oT = o.moments()
    assert normwise(gr, orr) < TOL
    assert np.abs(gu - ou).max() < TOL
    assert normwise(gT, oT) < TOL
    gf, _ = g.emitted()
    of, _ = o.emitted()
    assert normwise(gf, of) < TOL
    gd, od = g.diagnostics(), o.diagnostics()
    assert np.abs(gd - od).max() / abs(od[0]) < 1e-13


@pytest.mark.parametrize("d", [1, 2, 3])
def test_standard_tiny_lattices(d):
    shape = {1: (1, 1, 2), 2: (1, 1, 5), 3: (2, 1, 3)}[d]
    fl = fields(d, shape, 3, 1 / 3)
    g = lbm.Simulation(d, shape[2], shape[1], shape[0], tau=0.7, T0=1 / 3, model="standard")
    g.init(*fl)
    o = oracle.Sim(d, shape[2], shape[1], shape[0], tau=0.7, T0=1 / 3, model="standard")
    o.init(*fl)
    g.step(10)
    o.step(10)
    assert normwise(g.emitted()[0], o.emitted()[0]) < TOL


def test_standard_full_size_fp32_windows():
    """The comparator's benchmark configuration (D3Q19 256^3, FP32)."""
    c = W.CONFIGS["std3d"]
    rho, u, T = W.fields_for("std3d")
    g = lbm.Simulation(3, c["nx"], c["ny"], c["nz"], tau=c["tau"], T0=c["T0"], dtype="f32", model="standard")
    g.init(rho, u, T)
    g.step(4)
    f0, b0 = g.emitted()
    g.step(1)
    f1, b1 = g.emitted()
    wf, _ = check_windows(3, f0, b0, f1, b1, c["tau"], c["T0"], False, n_windows=8, model="standard")
    assert wf < 2e-6
    assert np.isfinite(g.diagnostics()).all()


@pytest.mark.parametrize("dtype,tol", [("f32", 2e-6), ("f16", 2e-3), ("bf16", 1.6e-2)])
def test_standard_one_step_storage_precision(dtype, tol):
    """One step from an identical emitted state agrees with the oracle to the
    storage precision."""
    shape = (1, 33, 70)
    fl = fields(2, shape, 11, 1 / 3)
    o = oracle.Sim(2, 70, 33, tau=0.6, T0=1 / 3, model="standard")
    o.init(*fl)
    f0, b0 = o.emitted()
    g = lbm.Simulation(2, 70, 33, tau=0.6, T0=1 / 3, dtype=dtype, model="standard")
    g.init(*fl)
    g.set_emitted(f0, b0)
    o.set_emitted(f0, b0)
    g.step(1)
    o.step(1)
    assert normwise(g.emitted()[0], o.emitted()[0]) < tol


def test_standard_rejects_walls_and_force():
    with pytest.raises(Exception):
        lbm.Simulation(2, 16, 16, bc="walls", model="standard")
    g = lbm.Simulation(2, 16, 16, model="standard")
    with pytest.raises(Exception):
        g.set_force([1e-4, 0.0])
