"""Slab partitioning of a periodic lattice across ranks (the multi-GPU layout; the paper
leaves multi-GPU runs to future work, Sec. 3.3).

The grid is split along its last axis (z in 3D, y in 2D) into equal slabs, one per rank. Each
rank holds its slab in a liblb context whose last dimension has one ghost layer at each end;
the context steps all its layers as an ordinary periodic grid, and after every step the
populations that cross each face move to the neighbouring ranks' ghost layers
(``lb_halo_pack`` / ``lb_halo_unpack``: 3 slots of one row for D2Q9, 5 or 9 slots of one plane
for D3Q19 / D3Q27). The global sums add the ranks' interior sums in FP64 (``lb_reduce_slab`` and
one all-reduce of six doubles).

Transports move the packed face buffers: ``DistTransport`` sends them with torch.distributed
point-to-point calls (NCCL between GPUs, gloo on the CPU) into the receiving rank's own
buffers; ``LocalTransport`` with ``step_local`` serves several slabs held by one process (one
device) with device-to-device copies, for tests.
Argument marshalling and message ordering only: every step of the method runs in liblb.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from .lattice import Lattice


def slab_bounds(n_last: int, world: int, rank: int):
    """First layer and number of layers of rank's slab of a last axis of n_last layers."""
    if n_last % world:
        raise ValueError(f"{n_last} layers do not split into {world} equal slabs")
    m = n_last // world
    return rank * m, m


def with_ghosts(a, first: int, count: int, axis_len: int, d: int):
    """The layers [first - 1, first + count] (periodic) of a field laid out [..., N] with the
    last axis slowest: the slab's own layers plus one ghost layer at each end."""
    a = np.asarray(a) if not isinstance(a, torch.Tensor) else a
    lead = a.shape[:-1]
    layers = a.reshape(*lead, axis_len, -1)
    idx = [(first - 1 + k) % axis_len for k in range(count + 2)]
    if isinstance(layers, torch.Tensor):
        out = layers[..., torch.tensor(idx, device=layers.device), :]
    else:
        out = layers[..., idx, :]
    return out.reshape(*lead, -1)


def interior(a, count: int):
    """The slab's own layers of a local field [..., N_local] (ghost layers dropped)."""
    lead = a.shape[:-1]
    layers = a.reshape(*lead, count + 2, -1)
    return layers[..., 1:count + 1, :].reshape(*lead, -1)


class DistTransport:
    """Face buffers over torch.distributed: the high face's buffer goes to rank + 1, the low
    face's to rank - 1 (periodic), each received into this rank's own buffer. Two messages per
    neighbour pair with distinct tags, so two ranks (each other's upper and lower neighbour)
    need no special case; one rank sends to itself by a local copy."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)

    def exchange(self, send_lo, send_hi, recv_lo, recv_hi):
        if self.world == 1:
            recv_lo.copy_(send_hi)
            recv_hi.copy_(send_lo)
            return
        dist = self.dist
        up, down = (self.rank + 1) % self.world, (self.rank - 1) % self.world
        ops = [dist.P2POp(dist.isend, send_hi, up, self.group, tag=0),
               dist.P2POp(dist.irecv, recv_lo, down, self.group, tag=0),
               dist.P2POp(dist.isend, send_lo, down, self.group, tag=1),
               dist.P2POp(dist.irecv, recv_hi, up, self.group, tag=1)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()

    def allreduce_sum(self, t):
        """Sum of t over the ranks. NCCL reduces device tensors only: a host tensor goes through
        the rank's current CUDA device and comes back."""
        if t.device.type == "cpu" and self.dist.get_backend(self.group) == "nccl":
            d = t.to(torch.device("cuda", torch.cuda.current_device()))
            self.dist.all_reduce(d, op=self.dist.ReduceOp.SUM, group=self.group)
            t.copy_(d.cpu())
            return t
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t


class LocalTransport:
    """Slabs of several ranks held by one process (one device), for tests: rank r of `world`
    gets an endpoint; step_local() steps them together."""

    def __init__(self, world: int):
        self.world = world

    def endpoint(self, rank: int):
        return _LocalEndpoint(self.world, rank)


class _LocalEndpoint:
    def __init__(self, world: int, rank: int):
        self.world, self.rank = world, rank


def step_local(slabs, n: int = 1):
    """n steps of the slabs of one process (slabs[r] is rank r): every slab steps, every slab
    packs its faces, the buffers move to the neighbours, every slab unpacks."""
    w = len(slabs)
    for _ in range(int(n)):
        for sl in slabs:
            sl.lat.step(1)
        for sl in slabs:
            sl.pack()
        for r, sl in enumerate(slabs):
            sl.bufs[2].copy_(slabs[(r - 1) % w].bufs[1])  # from the lower neighbour's high face
            sl.bufs[3].copy_(slabs[(r + 1) % w].bufs[0])  # from the upper neighbour's low face
        for sl in slabs:
            sl.unpack()


class SlabLattice:
    """One rank's slab of a periodic grid of global dims, split along the last axis.

    Arrays passed in and returned are the slab's own layers in the library's node order
    (x fastest), i.e. the rank's contiguous part of the global arrays. All ranks must call
    step() and reduce() together."""

    def __init__(self, stencil: str, global_dims, tau: float, collision: str, transport, storage: str = "f32",
                 nodes_per_thread: int = 0, device: int | None = None):
        self.stencil = stencil
        self.gdims = tuple(int(v) for v in global_dims)
        if len(self.gdims) == 2:
            self.gdims = (*self.gdims, 1)
        self.d = 2 if stencil == "D2Q9" else 3
        ax = self.d - 1
        self.axis_len = self.gdims[ax]
        self.t = transport
        self.first, self.count = slab_bounds(self.axis_len, transport.world, transport.rank)
        ldims = list(self.gdims)
        ldims[ax] = self.count + 2
        self.ldims = tuple(ldims)
        self.lat = Lattice(stencil, self.ldims, tau, collision, storage=storage, layout="ab",
                           nodes_per_thread=nodes_per_thread, device=device, graphs=False)
        self.N_global = int(np.prod(self.gdims))
        nb = ctypes.c_int64()
        _lib.check(self.lat._lib.lb_halo_bytes(self.lat.handle, ctypes.byref(nb)), "lb_halo_bytes")
        self.bufs = [torch.empty(int(nb.value), dtype=torch.uint8, device=self.lat.device) for _ in range(4)]

    def close(self):
        self.lat.close()

    def _ghosted(self, a):
        return with_ghosts(a, self.first, self.count, self.axis_len, self.d)

    def init_from_moments(self, rho_global, u_global):
        """f^eq of the global moments (rho[N], u[d][N] of the whole grid): the slab's layers and
        its ghost layers, so that no exchange is needed before the first step."""
        self.lat.init_from_moments(self._ghosted(rho_global), self._ghosted(u_global))
        return self

    def pack(self):
        """The crossing populations of both faces into the send buffers (on the lattice's stream)."""
        lib, h = self.lat._lib, self.lat.handle
        _lib.check(lib.lb_halo_pack(h, 0, self.bufs[0].data_ptr()), "lb_halo_pack")
        _lib.check(lib.lb_halo_pack(h, 1, self.bufs[1].data_ptr()), "lb_halo_pack")

    def unpack(self):
        """The received buffers into both ghost layers (on the lattice's stream)."""
        lib, h = self.lat._lib, self.lat.handle
        _lib.check(lib.lb_halo_unpack(h, 0, self.bufs[2].data_ptr()), "lb_halo_unpack")
        _lib.check(lib.lb_halo_unpack(h, 1, self.bufs[3].data_ptr()), "lb_halo_unpack")

    def exchange(self):
        """pack, move the face buffers through the transport (on torch's current stream, ordered
        after the lattice's), unpack."""
        self.pack()
        cur = torch.cuda.current_stream(self.lat.device)
        cur.wait_stream(self.lat.stream)
        self.t.exchange(*self.bufs)
        self.lat.stream.wait_stream(cur)
        self.unpack()

    def step(self, n: int = 1):
        """n steps of Eq. 1 on the slab, each followed by the face exchange (all ranks together)."""
        for _ in range(int(n)):
            self.lat.step(1)
            self.exchange()
        return self

    def get_populations(self, dtype=torch.float64, device=None):
        return interior(self.lat.get_populations(dtype, device), self.count)

    def moments(self, dtype=torch.float64, device=None):
        rho, u = self.lat.moments(dtype, device)
        return interior(rho, self.count), interior(u, self.count)

    def local_sums(self) -> np.ndarray:
        """The slab's unnormalised FP64 sums (lb_reduce_slab over its own layers)."""
        out = (ctypes.c_double * 6)()
        _lib.check(self.lat._lib.lb_reduce_slab(self.lat.handle, 1, self.count, out), "lb_reduce_slab")
        return np.array(list(out))

    def reduce(self) -> np.ndarray:
        """lb_reduce of the whole grid: the ranks' sums added in FP64 by one all-reduce."""
        t = torch.tensor(self.local_sums(), dtype=torch.float64)
        if self.t.world > 1:
            t = self.t.allreduce_sum(t)
        return normalise_sums(t.numpy(), self.N_global)


def normalise_sums(s, N: int) -> np.ndarray:
    """The lb_reduce convention from summed raw sums: E = (1/2N) sum |u|^2, E_rho likewise."""
    s = np.array(s, dtype=np.float64)
    s[4] = 0.5 * s[4] / N
    s[5] = 0.5 * s[5] / N
    return s


def allreduce_gradient(g: torch.Tensor, group=None) -> torch.Tensor:
    """Sum of the ranks' parameter gradients (data-parallel training: each rank runs its share
    of a batch's rollouts); g is summed in place in FP64 and returned in its own dtype."""
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return g
    acc = g.detach().to(torch.float64)
    dist.all_reduce(acc, op=dist.ReduceOp.SUM, group=group)
    g.copy_(acc.to(g.dtype))
    return g
