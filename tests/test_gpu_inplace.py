"""The in-place step (lbm_opts.inplace: one population buffer, two passes per
step on the AA access pattern) against the A-B fused step and the FP64 oracle
(needs a GB300): the emitted state after odd and even step counts (the
buffer alternates between the emitted layout and the arrived populations),
the moments and the diagnostics; checkpoints after even step counts; and the
smaller device footprint."""
import os
import tempfile

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


@pytest.fixture(autouse=True)
def _library_loaded():
    if lbm is None:
        raise _IMPORT_ERROR


def fields(d, shape, seed=31):
    rng = np.random.default_rng(seed)
    rho = 1 + 0.05 * rng.random(shape)
    u = 0.03 * rng.standard_normal((d,) + shape)
    T = 0.1 * (1 + 0.05 * rng.random(shape))
    return rho, u, T


@pytest.mark.parametrize("d,shape", [(2, (1, 20, 36)), (3, (10, 12, 14)), (1, (1, 1, 50))])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("thermal", [True, False])
def test_inplace_equals_ab_and_oracle(d, shape, dtype, thermal):
    nz, ny, nx = shape
    rho, u, T = fields(d, shape)
    a = lbm.Simulation(d, nx, ny, nz, tau=0.6, T0=0.1, thermal=thermal, dtype=dtype, inplace=True)
    b = lbm.Simulation(d, nx, ny, nz, tau=0.6, T0=0.1, thermal=thermal, dtype=dtype, tile=0, chunk=4)
    for s in (a, b):
        s.init(rho, u, T)
    tol = 1e-12 if dtype == "f64" else 2e-5
    for n in (1, 4, 3, 6):  # odd and even totals: 1, 5, 8, 14
        a.step(n)
        b.step(n)
        fa, ba = a.emitted()
        fb, bb = b.emitted()
        assert normwise(fa, fb) < tol and np.abs(ba - bb).max() < tol, a.nstep
        ma, mb = a.moments(), b.moments()
        assert normwise(ma[0], mb[0]) < tol and np.abs(ma[1] - mb[1]).max() < tol and normwise(ma[2], mb[2]) < tol
        da, db = a.diagnostics(), b.diagnostics()
        # FP32: the two kernels round differently (states within 2e-5), and so do their sums
        assert np.abs(da - db).max() <= (1e-12 if dtype == "f64" else 1e-6) * db[0]
    assert a.launch_config()[2] == "aa_collide_kernel"
    if dtype == "f64":
        o = oracle.Sim(d, nx, ny, nz, tau=0.6, T0=0.1, thermal=thermal)
        o.init(rho, u, T)
        o.step(a.nstep)
        fo, bo = o.emitted()
        fa, ba = a.emitted()
        assert normwise(fa, fo) < 1e-12 and np.abs(ba - bo).max() < 1e-12
    a.close()
    b.close()


def test_inplace_checkpoint_after_even_steps():
    d, shape = 3, (8, 8, 16)
    rho, u, T = fields(d, shape)
    a = lbm.Simulation(3, 16, 8, 8, tau=0.6, T0=0.1, thermal=True, dtype="f32", inplace=True)
    a.init(rho, u, T)
    a.step(3)
    with tempfile.TemporaryDirectory() as tmp:
        p = os.path.join(tmp, "ck.bin")
        with pytest.raises(lbm.LBMError) as e:
            a.save(p)
        assert e.value.status == lbm.LBM_EINVAL
        a.step(1)
        a.save(p)
        c = lbm.Simulation(3, 16, 8, 8, tau=0.6, T0=0.1, thermal=True, dtype="f32", inplace=True)
        c.load(p)
    a.step(5)
    c.step(5)
    fa, ba = a.emitted()
    fc, bc = c.emitted()
    assert np.array_equal(fa, fc) and np.array_equal(ba, bc)
    a.close()
    c.close()


def test_inplace_takes_less_device_memory():
    import torch
    dev = torch.device("cuda", 0)
    n = 128
    used = {}
    for inplace in (False, True):
        torch.cuda.synchronize(dev)
        free0 = torch.cuda.mem_get_info(dev)[0]
        s = lbm.Simulation(3, n, n, n, tau=0.6, T0=0.1, dtype="f32", inplace=inplace)
        torch.cuda.synchronize(dev)
        used[inplace] = free0 - torch.cuda.mem_get_info(dev)[0]
        s.close()
    N = n ** 3
    # A-B: 2 (19 + 6) floats per site; in place: 19 + 2 x 6 + (3 + 6) floats per site
    assert used[False] >= 2 * 25 * 4 * N and used[True] <= used[False] - 0.15 * 200 * N


def test_inplace_refusals():
    with pytest.raises(lbm.LBMError):
        lbm.Simulation(2, 16, 16, tau=0.6, T0=0.1, bc="fixed", inplace=True)
    with pytest.raises(lbm.LBMError):
        lbm.Simulation(2, 16, 16, tau=0.6, T0=0.1, dtype="f16", inplace=True)
    s = lbm.Simulation(3, 8, 8, 8, tau=0.6, T0=0.1, inplace=True)
    with pytest.raises(lbm.LBMError):
        s.set_mrt(1.2, 1.2)
    with pytest.raises(lbm.LBMError):
        s.set_force([1e-5, 0, 0])
    s.close()
