"""Host logic of the domain-decomposed path (slabs along the slowest axis):
the slab plan, the two-phase point-to-point halo exchange and the FP64
all-reduce of the diagnostics, run by 2 and 3 CPU ranks under gloo with
numpy slabs standing in for the library's pack / unpack of device planes.
After one exchange every rank's halo planes hold the planes the whole
periodic lattice has there, and the reduced sums equal the lattice's."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2501_00620_gb300 import decomp  # noqa: E402

NZ, NY, NX, NPL = 11, 3, 4, 5  # global planes, plane shape, "population planes" per message


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _lattice():
    rng = np.random.default_rng(3)
    return rng.standard_normal((NPL, NZ, NY, NX))


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A = _lattice()
        lo, hi = decomp.slab_bounds(NZ, world, rank)
        h = decomp.HALO
        # the slab as the library holds it: owned planes plus halo planes,
        # whose contents are garbage until the exchange
        slab = np.full((NPL, hi - lo + 2 * h, NY, NX), np.nan)
        slab[:, h:h + hi - lo] = A[:, lo:hi]
        n = slab.shape[1]

        def pack(side):
            p = h if side == 0 else n - 2 * h
            return torch.from_numpy(np.ascontiguousarray(slab[:, p:p + h]).ravel().copy())

        def unpack(side, msg):
            p = 0 if side == 0 else n - h
            slab[:, p:p + h] = msg.numpy().reshape(NPL, h, NY, NX)

        decomp.exchange_halos(dist, rank, world, pack, unpack,
                              lambda: torch.empty(NPL * h * NY * NX, dtype=torch.float64))
        want = A[:, np.arange(lo - h, hi + h) % NZ]
        halo_ok = bool(np.array_equal(slab, want))
        local = [A[0, lo:hi].sum(), A[1, lo:hi].sum(), A[2, lo:hi].sum()]
        total = decomp.reduce_diagnostics(dist, local)
        out.put((rank, lo, hi, halo_ok, total.tolist()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_halo_exchange_schedule_and_diagnostics_allreduce(world):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    A = _lattice()
    want_total = [A[0].sum(), A[1].sum(), A[2].sum()]
    covered = []
    for rank, lo, hi, halo_ok, total in res:
        assert halo_ok, rank
        np.testing.assert_allclose(total, want_total, rtol=1e-13)
        covered += list(range(lo, hi))
    assert covered == list(range(NZ))  # the slabs tile the axis once


def test_slab_plan_and_fields():
    """Slabs tile the axis in order, sizes differ by at most one plane; the
    slab fields are the lattice's planes with periodic halos (2D and 3D)."""
    for n, w in [(11, 2), (11, 3), (24, 4), (5, 5)]:
        b = [decomp.slab_bounds(n, w, r) for r in range(w)]
        assert b[0][0] == 0 and b[-1][1] == n and all(b[i][1] == b[i + 1][0] for i in range(w - 1))
        sizes = [hi - lo for lo, hi in b]
        assert max(sizes) - min(sizes) <= 1
    rng = np.random.default_rng(1)
    rho3, u3, T3 = rng.random((6, 2, 3)), rng.random((3, 6, 2, 3)), rng.random((6, 2, 3))
    r, u, T = decomp.slab_fields(rho3, u3, T3, 4, 6)
    idx = [2, 3, 4, 5, 0, 1]
    assert np.array_equal(r, rho3[idx]) and np.array_equal(u, u3[:, idx]) and np.array_equal(T, T3[idx])
    rho2, u2, T2 = rng.random((1, 7, 3)), rng.random((2, 1, 7, 3)), rng.random((1, 7, 3))
    r, u, T = decomp.slab_fields(rho2, u2, T2, 0, 2)
    idx = [5, 6, 0, 1, 2, 3]
    assert np.array_equal(r, rho2[:, idx]) and np.array_equal(u, u2[:, :, idx]) and np.array_equal(T, T2[:, idx])
