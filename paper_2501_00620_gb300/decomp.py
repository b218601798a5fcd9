"""Domain decomposition of one lattice into slabs along its slowest axis
(y in 2D, z in 3D), one slab per process (rank) or several per process.

The step is a nearest-neighbour stencil whose gradient term (the gradient of
rho b, Eqs. 59, 61, 68 of arXiv 2501.00620) reaches two sites away, so each
slab carries two halo planes at each face (lbm_opts.halo = 2) that hold the
neighbouring slabs' emitted state and are refreshed after every step:
point-to-point messages between neighbouring ranks (lbm_halo_pack on one
side, lbm_halo_unpack on the other), and one FP64 all-reduce of the dim + 2
conservation sums for the lattice's diagnostics.  Every step of the path
runs in the library; this module only plans the slabs and moves the
messages with torch.distributed (NCCL between GPUs, gloo on CPU).
"""
import numpy as np

HALO = 2


def slab_bounds(n, world, rank):
    """Owned planes [lo, hi) of `rank` among `world` slabs of an n-plane axis
    (the first n % world slabs take one plane more)."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def neighbours(rank, world):
    """Ranks below and above along the periodic slowest axis."""
    return (rank - 1) % world, (rank + 1) % world


def slab_fields(rho, u, T, lo, hi, halo=HALO):
    """Initial fields of the slab [lo, hi) plus `halo` planes on each side
    (periodic wrap), from the whole lattice's fields (rho, T: (nz, ny, nx);
    u: (d, nz, ny, nx); in 2D the slowest axis is ny with nz = 1)."""
    d = u.shape[0]
    ax = 0 if d == 3 else 1  # axis of the plane index in rho / T
    n = rho.shape[ax]
    idx = np.arange(lo - halo, hi + halo) % n
    take = lambda a, axis: np.ascontiguousarray(np.take(a, idx, axis=axis))
    return take(rho, ax), take(u, ax + 1), take(T, ax)


def exchange_halos(dist, rank, world, pack, unpack, make_buffer):
    """One halo exchange among `world` ranks.  pack(side) returns this rank's
    message for side 0 (its low owned planes, for the rank below) or 1 (its
    high owned planes, for the rank above) as a tensor; unpack(side, msg)
    writes a received message into the halo on that side; make_buffer()
    returns an empty message tensor.  Two phases, each a batch of one send
    and one receive per rank, so that the messages between two ranks match
    even where both neighbours are the same rank (world = 2): first every
    rank sends its high planes up and receives its low halo from below, then
    it sends its low planes down and receives its high halo from above."""
    lower, upper = neighbours(rank, world)
    if world == 1:
        unpack(0, pack(1))
        unpack(1, pack(0))
        return
    for send_side, recv_side, to, frm in ((1, 0, upper, lower), (0, 1, lower, upper)):
        msg = pack(send_side)
        buf = make_buffer()
        ops = [dist.P2POp(dist.isend, msg, to), dist.P2POp(dist.irecv, buf, frm)]
        for r in dist.batch_isend_irecv(ops):
            r.wait()
        unpack(recv_side, buf)


def reduce_diagnostics(dist, local, device="cpu"):
    """Sum of every rank's dim + 2 conservation sums (mass, momentum, energy
    of its owned sites), in FP64: the lattice's diagnostics."""
    import torch
    t = torch.as_tensor(np.asarray(local, dtype=np.float64), device=device).clone()
    if dist is not None:
        dist.all_reduce(t)
    return t.cpu().numpy()


class SlabRun:
    """One rank's slab of a decomposed lattice on its GPU: a Simulation with
    halo planes, initialised from the whole lattice's fields, stepped one step
    at a time with a halo exchange (NCCL) after each step."""

    def __init__(self, dist, rank, world, dim, nx, ny, nz, fields, device=0, **sim_kwargs):
        import torch
        from . import lbm
        self.dist, self.rank, self.world, self.dim = dist, rank, world, dim
        n = nz if dim == 3 else ny
        self.lo, self.hi = slab_bounds(n, world, rank)
        planes = self.hi - self.lo + 2 * HALO
        if dim == 3:
            self.sim = lbm.Simulation(3, nx, ny, planes, halo=HALO, device=device, **sim_kwargs)
        else:
            self.sim = lbm.Simulation(2, nx, planes, 1, halo=HALO, device=device, **sim_kwargs)
        self.sim.init(*slab_fields(*fields, self.lo, self.hi))
        self.dev = torch.device("cuda", device)
        self.nbytes = self.sim.halo_bytes()
        self.torch = torch

    def _pack(self, side):
        buf = self.torch.empty(self.nbytes, dtype=self.torch.uint8, device=self.dev)
        self.sim.halo_pack(side, buf.data_ptr())
        self.sim.sync()  # the message is complete before NCCL reads it
        return buf

    def _unpack(self, side, buf):
        self.torch.cuda.current_stream(self.dev).synchronize()  # received before the library reads it
        self.sim.halo_unpack(side, buf.data_ptr())

    def step(self, n=1):
        for _ in range(n):
            self.sim.step(1)
            exchange_halos(self.dist, self.rank, self.world, self._pack, self._unpack,
                           lambda: self.torch.empty(self.nbytes, dtype=self.torch.uint8, device=self.dev))
        self.sim.sync()

    def diagnostics(self):
        return reduce_diagnostics(self.dist, self.sim.diagnostics(), device=self.dev)

    def owned(self, a, axis):
        """The owned planes of a slab array (halo planes dropped)."""
        return np.take(a, np.arange(HALO, HALO + self.hi - self.lo), axis=axis)
