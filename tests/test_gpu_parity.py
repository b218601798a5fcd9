"""GPU path vs the FP64 oracle, through the C ABI (needs a GB300).

Tolerances:
* FP64 storage: 1e-12 norm-wise (max |gpu - oracle| / max |oracle| per field)
  on rho, T and the emitted populations, and 1e-12 on u in units of the
  lattice speed c, after the full step counts of the 1D configurations and
  after tens of steps on multi-tile 2D/3D lattices.  The only differences are
  rounding order and fused multiply-adds.  u is a difference of O(1)
  populations divided by rho, so its round-off floor is absolute (~1e-16 c
  per step): for the 1D sound wave (|u| ~ 6e-4 c) the two sides' rounding
  alone reaches ~2e-12 relative to max|u| after a few hundred steps.
* FP32 / FP16 / BF16 storage: one step from an identical emitted state, the
  populations must agree to the storage precision (FP32 2e-6, FP16 2e-3,
  BF16 1.6e-2 of the population scale); longer runs are reported, bounded
  loosely.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
from _parity import check_windows, normwise
from paper_2501_00620_gb300 import workloads as W

try:
    from paper_2501_00620_gb300 import lbm
except ImportError as _e:  # collected where the library is not built; the tests then fail loudly
    lbm = None
    _IMPORT_ERROR = _e

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _library_loaded():
    if lbm is None:
        raise _IMPORT_ERROR

FP64_TOL = 1e-12


def run_pair(d, shape, fields, tau, T0, thermal, bc, steps, dtype="f64", **kw):
    nz, ny, nx = shape
    g = lbm.Simulation(d, nx, ny, nz, tau=tau, T0=T0, bc=bc, dtype=dtype, thermal=thermal, **kw)
    g.init(*fields)
    o = oracle.Sim(d, nx, ny, nz, tau=tau, T0=T0, thermal=thermal, bc=bc)
    o.init(*fields)
    g.step(steps)
    o.step(steps)
    return g, o


def assert_fp64_parity(g, o, tol=FP64_TOL):
    gr, gu, gT = g.moments()
    orr, ou, oT = o.moments()
    assert normwise(gr, orr) < tol
    assert np.abs(gu - ou).max() < tol          # units of c = 1
    assert normwise(gT, oT) < tol
    gf, gb = g.emitted()
    of, ob = o.emitted()
    assert normwise(gf, of) < tol
    # bbar is stored as bbar + c^2/3 (the full per-axis variance), so its
    # round-off floor is absolute in units of c^2 (bbar ~ 1e-10 at T = c^2/3)
    assert np.abs(gb - ob).max() < tol


def test_sound1d_full_fp64():
    c = W.CONFIGS["sound1d"]
    g, o = run_pair(1, (1, 1, c["nx"]), W.fields_for("sound1d"), c["tau"], c["T0"], c["thermal"],
                    c["bc"], c["steps"])
    assert_fp64_parity(g, o)


def test_riemann1d_fp64():
    """Config 2 (two-state Riemann problem, thermal, fixed-state ends).  The
    run is ill-conditioned: the under-resolved shock (cell Reynolds number
    ~10 at tau = 0.55) amplifies rounding differences -- the oracle alone
    amplifies a 1e-8 per-step perturbation ~50x per 500 steps (see
    test_oracle_dynamics.py::test_riemann_amplifies_rounding).  So the GPU
    matches the oracle to 1e-12 while the two roundings are still
    indistinguishable (100 steps) and to the amplified level at the stated
    5000 steps (measured: ~4e-9 in rho, up to ~1e-7 transiently)."""
    c = W.CONFIGS["riemann1d"]
    fields = W.fields_for("riemann1d")
    g, o = run_pair(1, (1, 1, c["nx"]), fields, c["tau"], c["T0"], c["thermal"], c["bc"], 100)
    assert_fp64_parity(g, o)
    g.step(c["steps"] - 100)
    o.step(c["steps"] - 100)
    gr, gu, gT = g.moments()
    orr, ou, oT = o.moments()
    assert normwise(gr, orr) < 1e-6 and np.abs(gu - ou).max() < 1e-6 and normwise(gT, oT) < 1e-6
    # the first step after the start has a transiently negative moment
    # temperature at the jump (the oracle shows the same): reported, not fatal
    assert g.flags() == 2


def test_riemann1d_fp32_error():
    """Config 2 with FP32 populations: the storage rounding (~6e-8) is
    amplified by the shock like any perturbation; the error against the FP64
    oracle is ~1e-4 after 250 steps and the FP32 run leaves the stable regime
    by ~2000 steps (the oracle does the same under 1e-8 injected noise)."""
    c = W.CONFIGS["riemann1d"]
    g, o = run_pair(1, (1, 1, c["nx"]), W.fields_for("riemann1d"), c["tau"], c["T0"], c["thermal"],
                    c["bc"], 250, dtype="f32")
    gr, gu, gT = g.moments()
    orr, ou, oT = o.moments()
    assert normwise(gr, orr) < 5e-4 and np.abs(gu - ou).max() < 2e-3 and normwise(gT, oT) < 5e-3


@pytest.mark.parametrize("thermal,bc", [(True, "periodic"), (False, "periodic"), (True, "fixed")])
def test_2d_ragged_fp64(thermal, bc):
    """D2Q9 on 300 x 70 (tiles of 128-512 plus a ragged tail; several chunks)."""
    nx, ny = 300, 70
    if bc == "fixed":
        rho, u, T = W.riemann_1d(nx)
        rho = np.repeat(rho, ny, axis=1)
        T = np.repeat(T, ny, axis=1)
        u = np.zeros((2, 1, ny, nx))
        T0 = W.T_UNIT_RIEMANN
        tau = 0.55
    else:
        r, uu, TT = W.taylor_green_pulse_2d(300)
        rho, T = r[:, :ny, :], TT[:, :ny, :]
        u = uu[:, :, :ny, :]
        T0, tau = 0.1, 0.6
    g, o = run_pair(2, (1, ny, nx), (rho, u, T), tau, T0, thermal, bc, 60)
    assert_fp64_parity(g, o)


@pytest.mark.parametrize("thermal", [False, True])
def test_3d_ragged_fp64(thermal):
    """D3Q19 on 40 x 20 x 24 (x, y tiles with ragged tails, several z chunks)."""
    rho, u, T = W.solenoidal_3d(40, k0=2.0, T0=0.05, thermal=thermal)
    rho, T, u = rho[:24, :20, :], T[:24, :20, :], u[:, :24, :20, :]
    g, o = run_pair(3, (24, 20, 40), (rho, u, T), 0.52, 0.05, thermal, "periodic", 20)
    assert_fp64_parity(g, o)


def test_3d_fixed_state_fp64():
    nx, ny, nz = 36, 10, 6
    rho, _, T = W.riemann_1d(nx)
    rho = np.broadcast_to(rho, (nz, ny, nx)).copy()
    T = np.broadcast_to(T, (nz, ny, nx)).copy()
    g, o = run_pair(3, (nz, ny, nx), (rho, np.zeros((3, nz, ny, nx)), T), 0.55, W.T_UNIT_RIEMANN,
                    True, "fixed", 15)
    assert_fp64_parity(g, o)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_tiny_lattices(d):
    """Degenerate extents (1 and 2 sites per axis) wrap correctly."""
    shape = {1: (1, 1, 2), 2: (1, 1, 5), 3: (2, 1, 3)}[d]
    rng = np.random.default_rng(d)
    rho = 1 + 0.05 * rng.random(shape)
    u = 0.05 * rng.standard_normal((d,) + shape)
    g, o = run_pair(d, shape, (rho, u, 0.2), 0.7, 0.2, True, "periodic", 10)
    assert_fp64_parity(g, o)


@pytest.mark.parametrize("d", [2, 3])
def test_variants_and_chunks(d):
    """For a given tile variant every chunk length gives the same bits; the
    tile variants (separate template instantiations, where the compiler may
    contract multiply-adds differently) agree to a few units in the last
    place."""
    shape = (1, 33, 70) if d == 2 else (13, 11, 37)
    rng = np.random.default_rng(0)
    rho = 1 + 0.05 * rng.random(shape)
    u = 0.03 * rng.standard_normal((d,) + shape)
    ref = None
    nv = 2 if d == 3 else 3
    for v in range(nv):
        vref = None
        for chunk in (1, 5, 64):
            g = lbm.Simulation(d, shape[2], shape[1], shape[0], tau=0.6, T0=0.1, thermal=True,
                               tile=v, chunk=chunk)
            g.init(rho, u, 0.1)
            g.step(7)
            f, b = g.emitted()
            if vref is None:
                vref = (f, b)
            else:
                assert np.array_equal(f, vref[0]) and np.array_equal(b, vref[1])
        if ref is None:
            ref = vref
        else:
            assert np.abs(vref[0] - ref[0]).max() < 1e-15 and np.abs(vref[1] - ref[1]).max() < 1e-15


def test_graphs_equal_direct_launches():
    rho, u, T = W.taylor_green_pulse_2d(64)
    out = []
    for graphs in (True, False):
        g = lbm.Simulation(2, 64, 64, tau=0.6, T0=0.1, thermal=True, use_graphs=graphs)
        g.init(rho, u, T)
        g.step(37)
        g.step(40)
        out.append(g.emitted())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_diagnostics_vs_oracle_and_conservation():
    rng = np.random.default_rng(3)
    shape = (6, 10, 12)
    rho = 1 + 0.1 * rng.random(shape)
    u = 0.05 * rng.standard_normal((3,) + shape)
    T = 0.1 * (1 + 0.1 * rng.random(shape))
    g, o = run_pair(3, shape, (rho, u, T), 0.6, 0.1, True, "periodic", 0)
    d0 = g.diagnostics()
    np.testing.assert_allclose(d0, o.diagnostics(), rtol=1e-13, atol=1e-13 * d0[0])
    g.step(200)
    o.step(200)
    d1 = g.diagnostics()
    np.testing.assert_allclose(d1, o.diagnostics(), rtol=1e-12, atol=1e-12 * d0[0])
    assert abs(d1[0] - d0[0]) / d0[0] < 1e-13
    assert np.abs(d1[1:4] - d0[1:4]).max() / d0[0] < 1e-13
    assert abs(d1[4] - d0[4]) / d0[4] < 1e-12
    # the per-step history recorded by the step kernel
    h = g.diagnostics_history()
    assert len(h) == 200 and h[0, 0] == 0 and h[-1, 0] == 199
    assert np.abs(h[:, 1] - d0[0]).max() / d0[0] < 1e-13


def test_checkpoint_resume_bitwise():
    rho, u, T = W.taylor_green_pulse_2d(96)
    a = lbm.Simulation(2, 96, 96, tau=0.6, T0=0.1, thermal=True, dtype="f32")
    a.init(rho, u, T)
    a.step(30)
    b = lbm.Simulation(2, 96, 96, tau=0.6, T0=0.1, thermal=True, dtype="f32")
    b.init(rho, u, T)
    b.step(15)
    with tempfile.TemporaryDirectory() as d:
        p = os.path.join(d, "ck.bin")
        b.save(p)
        c = lbm.Simulation(2, 96, 96, tau=0.6, T0=0.1, thermal=True, dtype="f32")
        c.load(p)
    c.step(15)
    fa, ba = a.emitted()
    fc, bc_ = c.emitted()
    assert np.array_equal(fa, fc) and np.array_equal(ba, bc_)
    assert c.nstep == 30


def test_checkpoint_refuses_other_model_and_bad_parameters():
    """lbm_load refuses a bump-scheme checkpoint on a comparator simulation
    (same planes, other meaning), and a header whose tau or T0 is not finite
    and > 0 (a corrupt or foreign file), before touching the state."""
    import struct
    rho, u, T = W.taylor_green_pulse_2d(32)
    a = lbm.Simulation(2, 32, 32, tau=0.6, T0=1 / 3, dtype="f32")
    a.init(rho, u, T)
    a.step(2)
    with tempfile.TemporaryDirectory() as d:
        p = os.path.join(d, "ck.bin")
        a.save(p)
        s = lbm.Simulation(2, 32, 32, tau=0.6, T0=1 / 3, dtype="f32", model="standard")
        with pytest.raises(lbm.LBMError) as e:
            s.load(p)
        assert e.value.status == lbm.LBM_EINVAL and "model" in str(e.value)
        raw = bytearray(open(p, "rb").read())
        # header: magic[8], 8 ints, then tau and T0 as doubles
        for off, bad in ((40, 0.0), (40, float("nan")), (48, -0.1), (48, float("inf"))):
            q = os.path.join(d, "bad.bin")
            patched = bytearray(raw)
            patched[off:off + 8] = struct.pack("<d", bad)
            open(q, "wb").write(bytes(patched))
            b = lbm.Simulation(2, 32, 32, tau=0.6, T0=1 / 3, dtype="f32")
            b.init(rho, u, T)
            with pytest.raises(lbm.LBMError) as e:
                b.load(q)
            assert e.value.status == lbm.LBM_EIO
            b.close()
        s.close()
    a.close()


def test_state_roundtrip():
    rho, u, T = W.taylor_green_pulse_2d(32)
    g = lbm.Simulation(2, 32, 32, tau=0.6, T0=0.1, thermal=True)
    g.init(rho, u, T)
    g.step(3)
    f, b = g.emitted()
    h = lbm.Simulation(2, 32, 32, tau=0.6, T0=0.1, thermal=True)
    h.init(rho, u, T)
    h.set_emitted(f, b)
    f2, b2 = h.emitted()
    assert np.array_equal(f, f2) and np.array_equal(b, b2)


def test_unstable_state_is_reported_not_faulted():
    """A violent start (u ~ c at T << 1/3) drives T negative; the library
    reports LBM_EUNSTABLE and the process keeps a working context."""
    n = 64
    u = np.zeros((1, 1, 1, n))
    u[0, 0, 0, : n // 2] = 0.9
    g = lbm.Simulation(1, n, tau=0.55, T0=0.02, thermal=True)
    g.init(1.0, u, 0.02)
    g.step(50)
    with pytest.raises(lbm.LBMError) as e:
        g.sync()
    assert e.value.status == lbm.LBM_EUNSTABLE
    g.close()
    ok = lbm.Simulation(1, 16, tau=0.8, T0=1 / 3)
    ok.init(1.0, np.zeros((1, 1, 1, 16)), 1 / 3)
    ok.step(5)
    ok.sync()


@pytest.mark.parametrize("dtype,tol", [("f32", 2e-6), ("f16", 2e-3), ("bf16", 1.6e-2)])
def test_one_step_storage_precision_2d(dtype, tol):
    """From an identical emitted state, one GPU step in the storage dtype
    matches the oracle's FP64 step to the storage precision."""
    rho, u, T = W.taylor_green_pulse_2d(256)
    g = lbm.Simulation(2, 256, 256, tau=0.6, T0=0.1, thermal=True, dtype=dtype)
    g.init(rho, u, T)
    g.step(5)
    f0, b0 = g.emitted()
    g.step(1)
    f1, b1 = g.emitted()
    wf, wb = check_windows(2, f0, b0, f1, b1, 0.6, 0.1, True)
    assert wf < tol and wb < max(tol, 2e-6)


@pytest.mark.parametrize("name", ["tgv2d", "turb3d"])
def test_full_size_sampled_windows(name):
    """The configurations the benchmark times (full size, FP32, autotuned
    launch): after a few steps, random windows of the GPU state are advanced
    one step by the oracle and compared with the GPU's next state."""
    c = W.CONFIGS[name]
    rho, u, T = W.fields_for(name)
    g = lbm.Simulation(c["d"], c["nx"], c["ny"], c["nz"], tau=c["tau"], T0=c["T0"],
                       thermal=c["thermal"], dtype=c["dtype"])
    g.init(rho, u, T)
    g.step(4)
    f0, b0 = g.emitted()
    g.step(1)
    f1, b1 = g.emitted()
    wf, wb = check_windows(c["d"], f0, b0, f1, b1, c["tau"], c["T0"], c["thermal"], n_windows=8)
    assert wf < 2e-6 and wb < 2e-6
    d = g.diagnostics()
    assert np.isfinite(d).all()


def test_full_size_2d_fp64_windows():
    c = W.CONFIGS["tgv2d"]
    rho, u, T = W.fields_for("tgv2d")
    g = lbm.Simulation(2, c["nx"], c["ny"], tau=c["tau"], T0=c["T0"], thermal=c["thermal"], dtype="f64")
    g.init(rho, u, T)
    g.step(3)
    f0, b0 = g.emitted()
    g.step(1)
    f1, b1 = g.emitted()
    wf, wb = check_windows(2, f0, b0, f1, b1, c["tau"], c["T0"], c["thermal"], n_windows=8)
    assert wf < FP64_TOL and wb < FP64_TOL


TMA_BASE = 100


@pytest.mark.parametrize("d,shape,ntma,bc", [
    (2, (1, 40, 256), 4, "periodic"), (2, (1, 24, 128), 4, "fixed"),
    (3, (20, 32, 64), 5, "periodic"), (3, (9, 16, 64), 5, "fixed")])
@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_staged_variants_match_generic(d, shape, ntma, bc, dtype):
    """The staged kernel -- populations pulled from global memory, variance
    planes staged by bulk tensor copies, halos patched at the domain edges --
    computes what the generic kernel computes,
    up to FP32 rounding, for every tile shape and several chunk lengths,
    periodic and fixed-state; and one step of it matches the FP64 oracle
    to the storage precision."""
    nz, ny, nx = shape
    rng = np.random.default_rng(7)
    if bc == "fixed":
        rho, _, T = W.riemann_1d(nx)
        rho = np.broadcast_to(rho, shape).copy()
        T = np.broadcast_to(T, shape).copy()
        u = np.zeros((d,) + shape)
        T0, tau, thermal = W.T_UNIT_RIEMANN, 0.55, True
    else:
        rho = 1 + 0.05 * rng.random(shape)
        u = 0.03 * rng.standard_normal((d,) + shape)
        T = 0.1 * (1 + 0.05 * rng.random(shape))
        T0, tau, thermal = 0.1, 0.6, True
    ref = lbm.Simulation(d, nx, ny, nz, tau=tau, T0=T0, bc=bc, dtype=dtype, thermal=thermal, tile=0, chunk=4)
    ref.init(rho, u, T)
    ref.step(7)
    fr, br = ref.emitted()
    tol = 2e-5 if dtype == "f32" else 4e-3
    for k in range(ntma):
        for chunk in (3, 8):
            g = lbm.Simulation(d, nx, ny, nz, tau=tau, T0=T0, bc=bc, dtype=dtype, thermal=thermal,
                               tile=TMA_BASE + k, chunk=chunk)
            g.init(rho, u, T)
            g.step(6)
            f0, b0 = g.emitted()
            g.step(1)
            f1, b1 = g.emitted()
            g.sync()
            assert normwise(f1, fr) < tol and np.abs(b1 - br).max() < tol
            if bc == "periodic":
                wf, wb = check_windows(d, f0, b0, f1, b1, tau, T0, thermal, n_windows=3, half=4)
                assert wf < (2e-6 if dtype == "f32" else 2e-3) and wb < 2e-6


@pytest.mark.parametrize("d,shape", [(3, (32, 32, 64)), (2, (1, 64, 256))])
def test_fp32_diagnostics_match_exact_state_sums(d, shape):
    """The staged kernel sums the diagnostics per thread in FP32 as
    deviations from the rest state.  The mass of a state is the sum of all
    stored populations (the pull is a permutation), and the momentum that sum
    weighted by e_i plus half the summed gradient correction, which vanishes
    on a periodic lattice up to FP32 rounding of the antisymmetric sums.
    Checked against FP64 sums of the stored FP32 state: the only error left is
    the FP32 rounding of each site's rho and j."""
    nz, ny, nx = shape
    rng = np.random.default_rng(11)
    rho = 1 + 0.05 * rng.random(shape)
    u = 0.03 * rng.standard_normal((d,) + shape)
    T = 0.1 * (1 + 0.05 * rng.random(shape))
    for k in range(5 if d == 3 else 4):  # every staged tile of the lattice
        g = lbm.Simulation(d, nx, ny, nz, tau=0.6, T0=0.1, thermal=True, dtype="f32",
                           tile=TMA_BASE + k, chunk=8)
        g.init(rho, u, T)
        g.step(5)
        f, _ = g.emitted()
        diag = g.diagnostics()
        mass = f.sum()
        # per site the kernel's rho is an FP32 number near 1 (rounding <= 2^-24);
        # summed over N sites the error grows like sqrt(N) 2^-24: 1e-9 relative
        # is four standard deviations at N = 65536
        assert abs(diag[0] - mass) / mass < 1e-9
        e, _ = oracle.lattice(d)  # velocity order of the emitted planes
        mom = np.array([(e[:, a].reshape((-1,) + (1,) * (f.ndim - 1)) * f).sum() for a in range(d)])
        assert np.abs(diag[1:1 + d] - mom).max() / mass < 1e-8
        g.close()


PAIR_BASE = 200
N_PAIR = {2: 3, 3: 3}  # pair-kernel tiles per lattice


@pytest.mark.parametrize("d,shape", [(3, (24, 32, 64)), (3, (9, 8, 128)), (2, (1, 40, 256)), (2, (1, 24, 128))])
@pytest.mark.parametrize("thermal", [True, False])
def test_pair_kernel_matches_generic(d, shape, thermal):
    """The pair kernel (two x-adjacent sites per thread in packed FP32x2,
    8-byte population accesses, TMA-staged variance planes, tensor-memory
    hand-off) computes what the generic kernel computes up to FP32 rounding,
    for several chunk lengths and one or several tiles per axis; one step of
    it matches the FP64 oracle to the storage precision on sampled windows;
    and its diagnostics equal FP64 sums of the stored state."""
    nz, ny, nx = shape
    rng = np.random.default_rng(13)
    rho = 1 + 0.05 * rng.random(shape)
    u = 0.03 * rng.standard_normal((d,) + shape)
    T = 0.1 * (1 + 0.05 * rng.random(shape))
    T0, tau = 0.1, 0.6
    ref = lbm.Simulation(d, nx, ny, nz, tau=tau, T0=T0, dtype="f32", thermal=thermal, tile=0, chunk=4)
    ref.init(rho, u, T)
    ref.step(7)
    fr, br = ref.emitted()
    # chunk 20: a segment of 22 planes, so the pipeline barriers of the
    # warp-specialized form serve three planes each
    for k, chunk in [(k, c) for k in range(N_PAIR[d]) for c in (3, 8, 20)]:
        g = lbm.Simulation(d, nx, ny, nz, tau=tau, T0=T0, dtype="f32", thermal=thermal,
                           tile=PAIR_BASE + k, chunk=chunk)
        g.init(rho, u, T)
        g.step(6)
        assert g.launch_config()[0] == PAIR_BASE + k
        f0, b0 = g.emitted()
        g.step(1)
        f1, b1 = g.emitted()
        diag = g.diagnostics()
        g.sync()
        assert normwise(f1, fr) < 2e-5 and np.abs(b1 - br).max() < 2e-5
        wf, wb = check_windows(d, f0, b0, f1, b1, tau, T0, thermal, n_windows=3, half=4)
        assert wf < 2e-6 and wb < 2e-6
        mass = f1.sum()
        assert abs(diag[0] - mass) / mass < 1e-9
        e, _ = oracle.lattice(d)
        mom = np.array([(e[:, a].reshape((-1,) + (1,) * (f1.ndim - 1)) * f1).sum() for a in range(d)])
        assert np.abs(diag[1:1 + d] - mom).max() / mass < 1e-8
        g.close()


@pytest.mark.parametrize("dtype,tol_gen,tol_one", [("f16", 4e-3, 2e-3), ("bf16", 3e-2, 1.6e-2)])
@pytest.mark.parametrize("shape", [(1, 40, 256), (1, 17, 384)])
def test_pair_kernel_16bit_matches_generic(dtype, tol_gen, tol_one, shape):
    """The D2Q9 pair kernel on FP16 / BF16 shifted population storage (4-byte
    accesses of two adjacent 16-bit populations, FP32 variance) computes what
    the generic kernel computes on the same storage up to rounding, for every
    pair tile and chunk lengths that do and do not divide the march; one step
    from an identical state matches the FP64 oracle to the storage
    precision."""
    nz, ny, nx = shape
    rng = np.random.default_rng(19)
    rho = 1 + 0.05 * rng.random(shape)
    u = 0.03 * rng.standard_normal((2,) + shape)
    T = 0.1 * (1 + 0.05 * rng.random(shape))
    T0, tau = 0.1, 0.6
    ref = lbm.Simulation(2, nx, ny, 1, tau=tau, T0=T0, dtype=dtype, thermal=True, tile=0, chunk=4)
    ref.init(rho, u, T)
    ref.step(7)
    fr, br = ref.emitted()
    for k, chunk in [(k, c) for k in range(N_PAIR[2]) for c in (3, 8)]:
        g = lbm.Simulation(2, nx, ny, 1, tau=tau, T0=T0, dtype=dtype, thermal=True, tile=PAIR_BASE + k,
                           chunk=chunk)
        g.init(rho, u, T)
        g.step(6)
        assert g.launch_config()[0] == PAIR_BASE + k
        f0, b0 = g.emitted()
        g.step(1)
        f1, b1 = g.emitted()
        assert normwise(f1, fr) < tol_gen and np.abs(b1 - br).max() < tol_gen
        wf, wb = check_windows(2, f0, b0, f1, b1, tau, T0, True, n_windows=3, half=4)
        assert wf < tol_one and wb < 2e-6


def test_pair_kernel_moments_match_generic():
    """lbm_moments through the pair kernel (write_state off, FP64 moments
    out) gives the corrected u and T of the generic kernel up to FP32
    rounding."""
    shape = (12, 16, 128)
    rng = np.random.default_rng(17)
    rho = 1 + 0.05 * rng.random(shape)
    u = 0.03 * rng.standard_normal((3,) + shape)
    T = 0.1 * (1 + 0.05 * rng.random(shape))
    out = []
    for tile in (0, PAIR_BASE):
        g = lbm.Simulation(3, 128, 16, 12, tau=0.6, T0=0.1, dtype="f32", thermal=True, tile=tile, chunk=4)
        g.init(rho, u, T)
        g.step(4)
        out.append(g.moments())
        g.close()
    for a, b in zip(out[0], out[1]):
        assert np.abs(a - b).max() < 2e-5


@pytest.mark.parametrize("tile", [TMA_BASE + 4, PAIR_BASE, PAIR_BASE + 2])
def test_bounded_copy_wait_times_out_and_context_survives(tile):
    """A staged kernel whose first variance copy in one block is armed on its
    transaction barrier but never issued (the LBM_DEBUG_MISSING_COPY switch;
    nothing is left in flight) gives up after the bounded wait, drains,
    frees its tensor memory and returns: the host sees LBM_ETIMEOUT, and the
    same context then runs ordinary steps that equal a fresh simulation's."""
    shape = (12, 16, 64)
    rng = np.random.default_rng(23)
    rho = 1 + 0.05 * rng.random(shape)
    u = 0.03 * rng.standard_normal((3,) + shape)
    T = 0.1 * np.ones(shape)
    g = lbm.Simulation(3, 64, 16, 12, tau=0.6, T0=0.1, dtype="f32", tile=tile, chunk=4)
    g.init(rho, u, T)
    g.step(1)  # tuned onto the requested tile
    assert g.launch_config()[0] == tile
    g.set_debug(lbm.LBM_DEBUG_MISSING_COPY)
    g.step(1)
    with pytest.raises(lbm.LBMError) as e:
        g.sync()
        g.diagnostics()
    assert e.value.status == lbm.LBM_ETIMEOUT
    g.set_debug(0)
    g.init(rho, u, T)
    g.step(3)
    f, b = g.emitted()
    ref = lbm.Simulation(3, 64, 16, 12, tau=0.6, T0=0.1, dtype="f32", tile=tile, chunk=4)
    ref.init(rho, u, T)
    ref.step(3)
    fr, br = ref.emitted()
    assert np.array_equal(f, fr) and np.array_equal(b, br)
    g.close()
    ref.close()


@pytest.mark.parametrize("d", [1, 2, 3])
def test_small_t_fp64_recovery(d):
    """T0 = 0.02 with |u| ~ 0.3 (T << |u|^2): the FP32 temperature
    T = (Ebar - rho |u|^2)/(d rho) cancels (relative error ~1e-7 here).  With
    the FP64 recovery on (lbm_set_small_t) the transport, rho, j0 and Ebar
    of the site are FP64 sums of the stored FP32 values, so what is left of
    the error against the FP64 oracle on the same stored state is the FP32
    rounding of the gradient sums F, G (Eqs. 59, 61; on a uniform lattice
    their FP32 sums cancel only to ~eps |u| |rho b|): measured 3e-8 / 2e-9 /
    2e-8 against 4e-7 / 2e-7 / 1e-7 in 1D / 2D / 3D.  Velocity and density
    agree either way."""
    n = 16
    shape = (n,) * d + (1,) * (3 - d)
    shape = shape[::-1]
    rho = np.full(shape, 1.03)
    u = np.zeros((d,) + shape)
    for c, v in enumerate((0.27, 0.11, -0.07)[:d]):
        u[c] = v
    T = np.full(shape, 0.02)
    nz, ny, nx = shape
    g = lbm.Simulation(d, nx, ny, nz, tau=0.6, T0=0.02, thermal=True, dtype="f32", tile=0, chunk=4)
    g.init(rho, u, T)
    g.step(2)
    f, b = g.emitted()
    o = oracle.Sim(d, nx, ny, nz, tau=0.6, T0=0.02, thermal=True)
    o.set_emitted(f, b)
    orho, ou, oT = o.moments()
    _, _, T_off = g.moments()
    g.set_small_t(1.0)
    grho, gu, T_on = g.moments()
    err_on = np.abs(T_on - oT).max() / np.abs(oT).max()
    err_off = np.abs(T_off - oT).max() / np.abs(oT).max()
    assert err_on < 1e-7 and err_on < err_off / 3, (err_on, err_off)
    assert np.abs(grho - orho).max() < 1e-6 and np.abs(gu - ou).max() < 1e-6
    # the step with the recovery on stays a valid step of the same lattice
    g.step(2)
    f2, b2 = g.emitted()
    o.step(2)
    fo, bo = o.emitted()
    assert normwise(f2, fo) < 1e-6 and np.abs(b2 - bo).max() < 1e-6
    g.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_2d_multi_step_launch_equals_single_steps(dtype):
    """Small D2 lattices may run many steps per cooperative launch (the
    generic kernel's 128-site strips with a grid-wide barrier between
    steps): the same bits as single launches of the same tile in FP64 (FP32:
    the two kernels are compiled apart and may contract multiply-adds
    differently, so within FP32 rounding), and the per-step diagnostics
    history is recorded for every step."""
    shape = (1, 64, 96)
    rng = np.random.default_rng(37)
    rho = 1 + 0.05 * rng.random(shape)
    u = 0.03 * rng.standard_normal((2,) + shape)
    T = 0.1 * (1 + 0.05 * rng.random(shape))
    m = lbm.Simulation(2, 96, 64, 1, tau=0.6, T0=0.1, thermal=True, dtype=dtype, steps_per_launch=16)
    r = lbm.Simulation(2, 96, 64, 1, tau=0.6, T0=0.1, thermal=True, dtype=dtype, tile=1, chunk=4,
                       steps_per_launch=1)
    for s in (m, r):
        s.init(rho, u, T)
        s.step(48)
    assert m.launch_config()[2] == "step_multi_kernel"
    fm, bm = m.emitted()
    fr, br = r.emitted()
    if dtype == "f64":
        assert np.array_equal(fm, fr) and np.array_equal(bm, br)
    else:
        assert normwise(fm, fr) < 2e-6 and np.abs(bm - br).max() < 2e-6
    h = m.diagnostics_history()
    assert len(h) == 48 and h[-1, 0] == 47
    # momentum and energy as fractions of the mass (FP32: the per-site
    # gradient terms round differently in the two compilations)
    np.testing.assert_allclose(h, r.diagnostics_history(), rtol=1e-12 if dtype == "f64" else 2e-8,
                               atol=(1e-12 if dtype == "f64" else 1e-9) * h[0, 1])
    m.close()
    r.close()


STRIP_TILE = 3


@pytest.mark.parametrize("shape,bc", [((1, 70, 300), "periodic"), ((1, 33, 520), "fixed"),
                                      ((1, 3, 40), "periodic"), ((1, 1, 17), "periodic")])
@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_strip_variant_matches_generic(shape, bc, dtype):
    """The D2Q9 strip kernel (254-site strips of any extent, variance rows
    staged with plain loads) computes what the generic kernel computes up to
    FP32 rounding: ragged strips, fixed-state reservoirs, one to three rows;
    and one step of it matches the FP64 oracle to the storage precision."""
    nz, ny, nx = shape
    rng = np.random.default_rng(5)
    if bc == "fixed":
        rho, _, T = W.riemann_1d(nx)
        rho = np.broadcast_to(rho, shape).copy()
        T = np.broadcast_to(T, shape).copy()
        u = np.zeros((2,) + shape)
        T0, tau, thermal = W.T_UNIT_RIEMANN, 0.55, True
    else:
        rho = 1 + 0.05 * rng.random(shape)
        u = 0.03 * rng.standard_normal((2,) + shape)
        T = 0.1 * (1 + 0.05 * rng.random(shape))
        T0, tau, thermal = 0.1, 0.6, True
    ref = lbm.Simulation(2, nx, ny, 1, tau=tau, T0=T0, bc=bc, dtype=dtype, thermal=thermal, tile=0, chunk=4)
    ref.init(rho, u, T)
    ref.step(7)
    fr, br = ref.emitted()
    tol = 2e-5 if dtype == "f32" else 4e-3
    for chunk in (3, 16):
        g = lbm.Simulation(2, nx, ny, 1, tau=tau, T0=T0, bc=bc, dtype=dtype, thermal=thermal,
                           tile=STRIP_TILE, chunk=chunk)
        g.init(rho, u, T)
        g.step(6)
        f0, b0 = g.emitted()
        g.step(1)
        f1, b1 = g.emitted()
        assert g.launch_config()[0] == STRIP_TILE
        g.sync()
        assert normwise(f1, fr) < tol and np.abs(b1 - br).max() < tol
        if bc == "periodic" and ny >= 11:
            wf, wb = check_windows(2, f0, b0, f1, b1, tau, T0, thermal, n_windows=3, half=4)
            assert wf < tol and wb < max(tol, 2e-6)
        g.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_steps_per_launch_equal_single_steps(dtype):
    """Several steps per cooperative launch (1D lattices) give the same bits
    as one step per launch -- the tile body and its arithmetic are the same --
    and record one diagnostics entry per step."""
    rho, u, T = W.riemann_1d(1000)
    out = []
    for spl in (1, 16, 0):
        g = lbm.Simulation(1, 1000, tau=0.55, T0=W.T_UNIT_RIEMANN, bc="fixed", thermal=True, dtype=dtype,
                           steps_per_launch=spl)
        g.init(rho, u, T)
        g.step(37)
        g.step(5)
        out.append((g.emitted(), g.diagnostics_history()))
        g.close()
    (f1, b1), h1 = out[0]
    for (f, b), h in out[1:]:
        assert np.array_equal(f, f1) and np.array_equal(b, b1)
        assert len(h) == 42 and np.array_equal(h, h1)


def test_init_refuses_non_positive_fields_and_keeps_state():
    """lbm_init checks rho > 0 and T > 0 on the device; a refused call leaves
    the state of the previous lbm_init untouched."""
    d, nx = 2, 64
    rho, u, T = W.taylor_green_pulse_2d(n=64, T0=0.2)
    ny = nx
    g = lbm.Simulation(d, nx, ny, 1, tau=0.6, T0=0.2, bc="periodic", dtype="f64")
    g.init(rho, u, T)
    g.step(3)
    before = g.emitted()
    for field, k, bad in (("rho", 17, -1.0), ("T", nx * ny - 1, 0.0), ("rho", 5, np.nan)):
        r2, T2 = rho.copy(), T.copy()
        (r2 if field == "rho" else T2).reshape(-1)[k] = bad
        with pytest.raises(lbm.LBMError):
            g.init(r2, u, T2)
        after = g.emitted()
        for x, y in zip(before, after):
            assert np.array_equal(x, y)
    g.init(rho, u, T)  # a valid call still works
    g.step(1)
    g.close()
