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
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        recv_up.copy_(send_down)
        recv_down.copy_(send_up)
        return
    if send_up.is_cuda and dist.get_backend(group) == "gloo":
        # gloo moves host tensors only: stage the faces through host memory
        host = [t.cpu() for t in (send_up, send_down)] + [torch.empty_like(t, device="cpu") for t in (recv_up, recv_down)]
        exchange_faces(*host, group=group)
        recv_up.copy_(host[2])
        recv_down.copy_(host[3])
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


def global_sum(values, group=None, device=None):
    """Sum per-rank FP64 scalars over the ranks of the group: one all-reduce of
    the whole list (the only collective of a CG iteration besides the faces)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, group=group)
    return t.tolist()


def slab_cg(sd: SlabDirac, x, b, parity: int, m0: float, tol: float, maxit: int = 10000, group=None,
            device=None):
    """Conjugate gradient (Sec. 3.3) on Dhat_p^+ Dhat_p x = b over the slabs of
    all ranks of the group, x0 = 0.

    ``x`` and ``b`` are this rank's internal fields (parity p, the precision and
    right-hand sides of ``sd``).  Every operator application exchanges the slab
    faces (SlabDirac); every global scalar -- |b|^2, <p, M p> = |Dhat p|^2 and
    |r|^2 -- is this rank's partial sum all-reduced in FP64 over the group
    (``device``: where the reduction tensor lives, e.g. the GPU for NCCL).  The
    vector updates run on the slab (``axpby``, in libhr for a GPU slab).
    Stopping rule as the library's CG: the recursive |r| <= tol |b| per rhs,
    then the true residual b - M x (restart from it if it is still above).
    Returns (iterations, true relative residual per rhs)."""
    s, prec, nr = sd.slab, sd.prec, sd.nrhs
    r = s.new_field(parity, prec, nr)
    p = s.new_field(parity, prec, nr)
    t = s.new_field(parity, prec, nr)
    Mp = s.new_field(parity, prec, nr)
    ones, zeros = [1.0] * nr, [0.0] * nr
    s.axpby(b, x, zeros, zeros, parity, prec, nr)     # x = 0
    s.axpby(b, r, ones, zeros, parity, prec, nr)      # r = b
    s.axpby(b, p, ones, zeros, parity, prec, nr)      # p = b
    bb = global_sum(s.norm2(b, parity, prec, nr), group, device)
    stop = [tol * tol * v for v in bb]
    rr = list(bb)

    def apply_M(out, inp):
        sd.apply(t, inp, parity, m0)
        sd.apply(out, t, parity, m0, dagger=True)

    it = 0
    while it < maxit:
        active = [rr[k] > stop[k] for k in range(nr)]
        sd.apply(t, p, parity, m0)
        pAp = global_sum(s.norm2(t, parity, prec, nr), group, device)
        sd.apply(Mp, t, parity, m0, dagger=True)
        alpha = [rr[k] / pAp[k] if active[k] and pAp[k] > 0 else 0.0 for k in range(nr)]
        s.axpby(p, x, alpha, ones, parity, prec, nr)
        s.axpby(Mp, r, [-a for a in alpha], ones, parity, prec, nr)
        rr_new = global_sum(s.norm2(r, parity, prec, nr), group, device)
        it += 1
        if all(rr_new[k] <= stop[k] for k in range(nr)):
            apply_M(Mp, x)                                 # true residual r = b - M x
            s.axpby(b, r, ones, zeros, parity, prec, nr)
            s.axpby(Mp, r, [-1.0] * nr, ones, parity, prec, nr)
            rt = global_sum(s.norm2(r, parity, prec, nr), group, device)
            if all(rt[k] <= stop[k] for k in range(nr)):
                return it, [(rt[k] / bb[k]) ** 0.5 if bb[k] > 0 else 0.0 for k in range(nr)]
            s.axpby(r, p, ones, zeros, parity, prec, nr)   # restart from the true residual
            rr = rt
            continue
        beta = [rr_new[k] / rr[k] if active[k] else 1.0 for k in range(nr)]
        s.axpby(r, p, [1.0 if active[k] else 0.0 for k in range(nr)], beta, parity, prec, nr)
        rr = rr_new
    raise RuntimeError(f"slab_cg: no convergence in {maxit} iterations")
