"""The sharded step across processes: one slab of the mesh per rank (the domain decomposition
of Sec. 5), its halo exchanged by torch.distributed point-to-point operations.

The partition and the halo are those of the library's in-process form (ridg_shard_*): the
mesh is cut along its slowest axis into slabs of nearly equal numbers of layers (the first
n mod count slabs one layer more); with a nonzero velocity a along that axis every slab
carries the two layers upstream of it (below it for a > 0, above for a < 0) and, per step,
receives them from its upstream neighbour's outermost interior layers before stepping its
locally periodic mesh.  A rank's local array holds its layers in that order: the halo first
for a > 0, last for a < 0.  With gloo the layers are CPU tensors; with NCCL they would be
views of each slab's device state on the slab's stream.
"""
from __future__ import annotations


def partition(n: int, count: int):
    """(first layer, layers) of every slab: as even as possible, the extra layers first."""
    if count < 1 or n < 2 * count:
        raise ValueError("every slab needs at least two layers")
    base, extra = divmod(n, count)
    out, g = [], 0
    for i in range(count):
        k = base + (1 if i < extra else 0)
        out.append((g, k))
        g += k
    return out


def halo_layers(a: float) -> int:
    """Halo depth along the slab axis: two layers upstream, none without flux along it."""
    return 2 if a != 0 else 0


def neighbours(rank: int, ws: int, a: float):
    """(upstream rank, downstream rank) along the slab axis (periodic)."""
    if a > 0:
        return (rank - 1) % ws, (rank + 1) % ws
    return (rank + 1) % ws, (rank - 1) % ws


def local_layers(first: int, nloc: int, n: int, a: float):
    """Global layer of every local layer of a slab (halo included, periodic)."""
    h = halo_layers(a)
    start = first - h if a > 0 else first
    return [(start + l) % n for l in range(nloc + h)]


class SlabExchange:
    """The per-step halo exchange of one rank's slab: send the two outermost interior layers
    downstream, receive the two halo layers from upstream (one batched isend / irecv)."""

    def __init__(self, rank: int, ws: int, a: float, nloc: int):
        self.rank, self.ws, self.a, self.nloc = rank, ws, a, nloc
        self.h = halo_layers(a)
        self.up, self.down = neighbours(rank, ws, a)

    def send_slice(self):
        # a > 0: the last two interior layers (local h + nloc - 2, h + nloc - 1);
        # a < 0: the first two (local 0, 1)
        return slice(self.h + self.nloc - 2, self.h + self.nloc) if self.a > 0 else slice(0, 2)

    def halo_slice(self):
        return slice(0, 2) if self.a > 0 else slice(self.nloc, self.nloc + 2)

    def exchange(self, q):
        """q: the local layers, shape (layers, per-layer values); halo filled in place."""
        if self.h == 0:
            return
        send = q[self.send_slice()].contiguous()
        if self.ws == 1:
            q[self.halo_slice()] = send
            return
        import torch
        import torch.distributed as dist
        recv = torch.empty_like(send)
        reqs = dist.batch_isend_irecv([dist.P2POp(dist.isend, send, self.down),
                                       dist.P2POp(dist.irecv, recv, self.up)])
        for r in reqs:
            r.wait()
        q[self.halo_slice()] = recv
