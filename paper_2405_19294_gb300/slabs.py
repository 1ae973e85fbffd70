"""The even-odd operator on a lattice split in time over the ranks of a process
group: the halo-ready geometry of Sec. 2 (bulk sites and receive buffers,
the directions that need the neighbours masked until their data arrive, send
buffers filled from the boundary sites with half-spinors).

Every rank holds one time slab, an ``hr.Lattice`` created with ``t0`` and
``T_global`` (slab k of n covers [k T/n, (k+1) T/n)).  One application of
Dhat_p runs two hops, each as

    begin  -- fill the send buffers from the boundary, bulk hop with the
              face-crossing t hops masked (on the GPU, in libhr)
    exchange -- send_down to the rank below, where it becomes receive-up;
              send_up to the rank above, where it becomes receive-down
              (periodic in rank order)
    end    -- add the face terms from the receive buffers (libhr)

The exchange is the only collective: point-to-point sends of the two face
buffers (NCCL between GPUs, gloo on the host).  With one rank the buffers are
simply swapped in place.  Any object with the methods ``domain_hop_begin``,
``domain_hop_end``, ``new_halo`` and ``new_field`` of ``hr.Lattice`` can
serve as the slab.
"""
from __future__ import annotations


def exchange_faces(send_up, send_down, recv_up, recv_down, group=None):
    """recv_up <- send_down of the rank above; recv_down <- send_up of the rank below."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        recv_up.copy_(send_down)
        recv_down.copy_(send_up)
        return
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    up = dist.get_global_rank(group, (rank + 1) % world) if group is not None else (rank + 1) % world
    down = dist.get_global_rank(group, (rank - 1) % world) if group is not None else (rank - 1) % world
    # per peer the two messages are matched in issue order: first the
    # send_down / receive-up pair, then send_up / receive-down (with two ranks
    # the peer above and below is the same process)
    ops = [dist.P2POp(dist.isend, send_down, down, group, tag=0),
           dist.P2POp(dist.irecv, recv_up, up, group, tag=0),
           dist.P2POp(dist.isend, send_up, up, group, tag=1),
           dist.P2POp(dist.irecv, recv_down, down, group, tag=1)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()


class SlabDirac:
    """Dhat_p on this rank's time slab, coupled to the other ranks' slabs."""

    def __init__(self, slab, prec: int, nrhs: int = 1, group=None):
        self.slab, self.prec, self.nrhs, self.group = slab, prec, nrhs, group
        self.bufs = [slab.new_halo(prec, nrhs) for _ in range(4)]  # send_up, send_down, recv_up, recv_down
        self.tmp = None

    def apply(self, out, inp, parity: int, m0: float, dagger: bool = False):
        """out = Dhat_parity inp (internal fields of this slab, both of the given parity)."""
        s, (su, sd, ru, rd) = self.slab, self.bufs
        q = 1 - parity
        if self.tmp is None:
            self.tmp = s.new_field(q, self.prec, self.nrhs)
        for stage in (0, 1):
            o = self.tmp if stage == 0 else out
            ih = inp if stage == 0 else self.tmp
            op = q if stage == 0 else parity
            s.domain_hop_begin(o, ih, inp if stage else None, op, m0, self.prec, stage, su, sd,
                               nrhs=self.nrhs, dagger=dagger)
            exchange_faces(su, sd, ru, rd, self.group)
            s.domain_hop_end(o, op, m0, self.prec, stage, ru, rd, nrhs=self.nrhs, dagger=dagger)
        return out
