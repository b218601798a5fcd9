"""Domain decomposition on one GPU: a lattice split into k slabs along its
slowest axis (lbm_opts.halo = 2), stepped one step at a time with the halo
exchange after every step, equals the undecomposed lattice bit for bit -- the
same kernel and tile, the same per-site arithmetic -- in FP64 and FP32, on
the generic, staged, pair and strip kernels, periodic and fixed-state in x;
the summed slab diagnostics equal the lattice's; and the multi-process form
(pack into a message, unpack on the other side) gives the same bits as the
in-process exchange.  (Needs a GB300.)"""
import numpy as np
import pytest

from paper_2501_00620_gb300 import decomp
from paper_2501_00620_gb300 import workloads as W

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


def fields(d, shape, bc):
    rng = np.random.default_rng(29)
    nz, ny, nx = shape
    if bc == "fixed":
        rho, _, T = W.riemann_1d(nx)
        rho = np.broadcast_to(rho, shape) * (1 + 0.01 * rng.random(shape))
        T = np.broadcast_to(T, shape) * (1 + 0.01 * rng.random(shape))
        u = 0.01 * rng.standard_normal((d,) + shape)
        return rho, u, T, W.T_UNIT_RIEMANN, 0.55
    rho = 1 + 0.05 * rng.random(shape)
    u = 0.03 * rng.standard_normal((d,) + shape)
    T = 0.1 * (1 + 0.05 * rng.random(shape))
    return rho, u, T, 0.1, 0.6


def slab_sims(d, shape, k, dtype, tile, bc, rho, u, T, T0, tau):
    nz, ny, nx = shape
    n = nz if d == 3 else ny
    sims, bounds = [], []
    for r in range(k):
        lo, hi = decomp.slab_bounds(n, k, r)
        planes = hi - lo + 2 * decomp.HALO
        ext = (nx, ny, planes) if d == 3 else (nx, planes, 1)
        s = lbm.Simulation(d, *ext, tau=tau, T0=T0, bc=bc, dtype=dtype, thermal=True, tile=tile, chunk=4,
                           halo=decomp.HALO)
        s.init(*decomp.slab_fields(rho, u, T, lo, hi))
        sims.append(s)
        bounds.append((lo, hi))
    return sims, bounds


CASES = [(3, (24, 16, 64), "f64", 0, "periodic"), (3, (24, 16, 64), "f32", 104, "periodic"),
         (3, (24, 16, 64), "f32", 200, "periodic"), (3, (24, 16, 64), "f32", 0, "fixed"),
         (3, (24, 16, 64), "f32", 104, "fixed"), (2, (1, 24, 256), "f64", 0, "periodic"),
         (2, (1, 24, 256), "f32", 200, "periodic"), (2, (1, 24, 256), "f32", 3, "fixed"),
         (2, (1, 24, 256), "f16", 101, "periodic")]


@pytest.mark.parametrize("d,shape,dtype,tile,bc", CASES)
@pytest.mark.parametrize("k", [2, 3, 4])
def test_slabs_equal_the_whole_lattice(d, shape, dtype, tile, bc, k):
    nz, ny, nx = shape
    rho, u, T, T0, tau = fields(d, shape, bc)
    whole = lbm.Simulation(d, nx, ny, nz, tau=tau, T0=T0, bc=bc, dtype=dtype, thermal=True, tile=tile, chunk=4)
    whole.init(rho, u, T)
    sims, bounds = slab_sims(d, shape, k, dtype, tile, bc, rho, u, T, T0, tau)
    steps = 6
    for _ in range(steps):
        for s in sims:
            s.step(1)
        lbm.lbm_halo_exchange(sims)
    whole.step(steps)
    fw, bw = whole.emitted()
    dw = whole.diagnostics()
    ax = 1 if d == 3 else 2  # plane axis of the (Q, nz, ny, nx) state arrays
    h = decomp.HALO
    parts_f, parts_b, diag = [], [], np.zeros(d + 2)
    for s, (lo, hi) in zip(sims, bounds):
        assert s.launch_config()[0] == whole.launch_config()[0] == tile
        f, b = s.emitted()
        parts_f.append(np.take(f, np.arange(h, h + hi - lo), axis=ax))
        parts_b.append(np.take(b, np.arange(h, h + hi - lo), axis=ax))
        diag += s.diagnostics()
        s.close()
    fs, bs = np.concatenate(parts_f, axis=ax), np.concatenate(parts_b, axis=ax)
    assert np.array_equal(fs, fw) and np.array_equal(bs, bw)
    # diagnostics: FP64 sums (1e-12); the 32/16-bit kernels sum FP32
    # deviations per thread, whose rounding depends on the partition into
    # blocks (their contract: 1e-9 of the exact sums of the stored state)
    tol = 1e-12 if dtype == "f64" else 1e-9
    assert abs(diag[0] - dw[0]) <= tol * dw[0]
    assert np.abs(diag[1:] - dw[1:]).max() <= 10 * tol * dw[0]
    whole.close()


def test_pack_unpack_equals_in_process_exchange():
    """The messages of the multi-process path (lbm_halo_pack into device
    memory, lbm_halo_unpack on the receiving slab, here two slabs of one
    process with torch buffers in between) give the same bits as
    lbm_halo_exchange."""
    import torch
    d, shape, bc = 3, (16, 16, 64), "periodic"
    rho, u, T, T0, tau = fields(d, shape, bc)
    A, _ = slab_sims(d, shape, 2, "f32", 104, bc, rho, u, T, T0, tau)
    B, _ = slab_sims(d, shape, 2, "f32", 104, bc, rho, u, T, T0, tau)
    nbytes = A[0].halo_bytes()
    assert nbytes == 2 * (19 * 4 + 6 * 4) * 16 * 64  # two planes of 19 populations and 6 variance components
    dev = torch.device("cuda", 0)
    for _ in range(4):
        for s in A + B:
            s.step(1)
        lbm.lbm_halo_exchange(A)
        msgs = {}
        for r, s in enumerate(B):
            for side in (0, 1):
                m = torch.empty(nbytes, dtype=torch.uint8, device=dev)
                s.halo_pack(side, m.data_ptr())
                msgs[r, side] = m
            s.sync()
        for r, s in enumerate(B):
            # low halo <- the high planes of the slab below, high <- the low planes above
            s.halo_unpack(0, msgs[(r - 1) % 2, 1].data_ptr())
            s.halo_unpack(1, msgs[(r + 1) % 2, 0].data_ptr())
            s.sync()
    for a, b in zip(A, B):
        fa, ba = a.emitted()
        fb, bb = b.emitted()
        assert np.array_equal(fa, fb) and np.array_equal(ba, bb)


def test_halo_option_is_validated():
    with pytest.raises(lbm.LBMError) as e:
        lbm.Simulation(1, 64, tau=0.6, T0=0.1, halo=2)
    assert e.value.status == lbm.LBM_EINVAL
    with pytest.raises(lbm.LBMError):
        lbm.Simulation(3, 16, 16, 4, tau=0.6, T0=0.1, halo=2)  # no owned plane
    with pytest.raises(lbm.LBMError):
        lbm.Simulation(2, 16, 16, 1, tau=0.6, T0=0.1, bc="walls", halo=2)
    s = lbm.Simulation(3, 16, 16, 8, tau=0.6, T0=0.1)
    assert s.halo_bytes() == 0
    with pytest.raises(lbm.LBMError):
        s.halo_pack(0, 0)
    s.close()
