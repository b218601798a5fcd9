"""The cluster-resident multi-step kernel (lbm_opts.cluster: a small periodic
D2Q9 lattice held in the shared memory of one thread-block cluster, many steps
per launch, neighbour rows through distributed shared memory) against the
generic kernel's single steps and the FP64 oracle (needs a GB300): every
variant, bands of unequal height and widths that are no multiple of a warp,
launch lengths that do not divide the step count, thermal and isothermal;
the per-step diagnostics history; refusal of lattices that do not fit; and the
switch away from it when a setting only the generic kernel has is turned on."""
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


def fields(shape, seed=41):
    rng = np.random.default_rng(seed)
    rho = 1 + 0.05 * rng.random(shape)
    u = 0.03 * rng.standard_normal((2,) + shape)
    T = 0.1 * (1 + 0.05 * rng.random(shape))
    return rho, u, T


# (ny, nx): 16 equal bands of 4 rows; 37 rows in bands of 2 and 3 (37 = 16 x 2
# + 5); 20 rows in bands of 1 and 2 -- every band's neighbour rows live in
# other blocks; widths 64, 50 and 96
SHAPES = [(64, 64), (37, 50), (20, 96)]


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("ny,nx", SHAPES)
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("thermal", [True, False])
def test_cluster_kernel_matches_generic_and_oracle(variant, ny, nx, dtype, thermal):
    shape = (1, ny, nx)
    rho, u, T = fields(shape)
    c = lbm.Simulation(2, nx, ny, 1, tau=0.6, T0=0.1, thermal=thermal, dtype=dtype, cluster=1 + variant,
                       steps_per_launch=10)
    r = lbm.Simulation(2, nx, ny, 1, tau=0.6, T0=0.1, thermal=thermal, dtype=dtype, tile=0, chunk=4,
                       steps_per_launch=1)
    for s in (c, r):
        s.init(rho, u, T)
    tol = 1e-12 if dtype == "f64" else 2e-5
    for n in (1, 23):  # 1 step, then 10 + 10 + 3 per launch
        c.step(n)
        r.step(n)
        fc, bc = c.emitted()
        fr, br = r.emitted()
        assert normwise(fc, fr) < (tol if n > 1 or dtype == "f64" else 2e-6), c.nstep
        assert np.abs(bc - br).max() < tol
    tile, _, kernel = c.launch_config()
    assert kernel == "step_cluster_kernel" and tile == 300 + variant
    # moments and the per-step diagnostics history of every step
    mc, mr = c.moments(), r.moments()
    assert normwise(mc[0], mr[0]) < tol and np.abs(mc[1] - mr[1]).max() < tol and normwise(mc[2], mr[2]) < tol
    hc, hr = c.diagnostics_history(), r.diagnostics_history()
    assert len(hc) == 24 and hc[-1, 0] == 23
    np.testing.assert_allclose(hc, hr, rtol=1e-12 if dtype == "f64" else 2e-8,
                               atol=(1e-12 if dtype == "f64" else 1e-6) * hr[0, 1])
    if dtype == "f64":
        o = oracle.Sim(2, nx, ny, 1, tau=0.6, T0=0.1, thermal=thermal)
        o.init(rho, u, T)
        o.step(c.nstep)
        fo, bo = o.emitted()
        assert normwise(fc, fo) < 1e-12 and np.abs(bc - bo).max() < 1e-12
    c.close()
    r.close()


def test_cluster_kernel_refuses_what_does_not_fit():
    # 512^2 FP64 needs about 30 MB: far beyond one cluster's shared memory
    s = lbm.Simulation(2, 512, 512, 1, tau=0.6, T0=0.1, dtype="f64", cluster=1)
    s.init(*fields((1, 512, 512)))
    with pytest.raises(lbm.LBMError) as e:
        s.step(2)
    assert e.value.status == lbm.LBM_EINVAL
    s.close()
    # fewer rows than blocks in the cluster
    s = lbm.Simulation(2, 64, 8, 1, tau=0.6, T0=0.1, dtype="f32", cluster=1)
    s.init(*fields((1, 8, 64)))
    with pytest.raises(lbm.LBMError):
        s.step(2)
    s.close()
    with pytest.raises(lbm.LBMError):
        lbm.Simulation(2, 64, 64, 1, tau=0.6, T0=0.1, dtype="f32", cluster=9)


def test_cluster_kernel_leaves_for_the_generic_kernel_when_forced():
    """A body force is a generic-kernel setting: the lattice leaves the
    cluster kernel, and its steps equal the generic kernel's."""
    shape = (1, 32, 64)
    rho, u, T = fields(shape)
    c = lbm.Simulation(2, 64, 32, 1, tau=0.6, T0=0.1, dtype="f64", thermal=True, cluster=1, steps_per_launch=8)
    r = lbm.Simulation(2, 64, 32, 1, tau=0.6, T0=0.1, dtype="f64", thermal=True, tile=0, chunk=4,
                       steps_per_launch=1)
    for s in (c, r):
        s.init(rho, u, T)
        s.step(8)
    assert c.launch_config()[2] == "step_cluster_kernel"
    for s in (c, r):
        s.set_force([1e-5, 0.0])
        s.step(5)
    assert c.launch_config()[2] != "step_cluster_kernel"
    fc, bc = c.emitted()
    fr, br = r.emitted()
    assert normwise(fc, fr) < 1e-12 and np.abs(bc - br).max() < 1e-12
    c.close()
    r.close()


@pytest.mark.parametrize("n", [64, 128])
def test_autotuned_small_lattice_matches_generic(n):
    """Whatever the steps-per-launch autotuner picks for a small FP32 lattice
    (graph replays of single steps, the cooperative multi-step kernel or the
    cluster kernel), the result is the generic kernel's within FP32
    rounding."""
    shape = (1, n, n)
    rho, u, T = fields(shape, seed=43)
    a = lbm.Simulation(2, n, n, 1, tau=0.6, T0=0.1, thermal=True, dtype="f32")
    r = lbm.Simulation(2, n, n, 1, tau=0.6, T0=0.1, thermal=True, dtype="f32", tile=0, chunk=4,
                       steps_per_launch=1)
    for s in (a, r):
        s.init(rho, u, T)
        s.step(100)
    fa, ba = a.emitted()
    fr, br = r.emitted()
    assert normwise(fa, fr) < 2e-5 and np.abs(ba - br).max() < 2e-5, a.launch_config()
    a.close()
    r.close()
