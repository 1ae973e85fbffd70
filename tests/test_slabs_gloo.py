"""Time-slab decomposition over a process group on the host: two (and one)
gloo ranks each hold one slab (a host stand-in of libhr's slab), run
``slabs.SlabDirac`` with its face exchange, and together reproduce the
oracle's Dhat on the whole lattice."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import sun
from oracle.dirac import Geometry, WilsonOperator
from paper_2405_19294_gb300 import inputs, slabs
from slab_fake import FakeSlab

T, L, N, REP, M0 = 8, 4, 2, "fund", -0.3


def _problem():
    g = Geometry(T, L)
    U = sun.reunitarise(sun.links_from_algebra(inputs.algebra_coefficients(0, T, L, N), 1.0, N))
    op = WilsonOperator(U, N, REP, g, M0, 0.0)
    psi = inputs.gaussian_spinor(3, T, L, op.d, nrhs=2)
    return g, op, psi


def _run_slab(rank, world, port, parity, dagger, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g, op, psi = _problem()
        Tl = T // world
        slab = FakeSlab(op.UR, T, L, rank * Tl, Tl)
        sd = slabs.SlabDirac(slab, prec=0, nrhs=2)
        V3 = L ** 3
        inp = torch.from_numpy(np.ascontiguousarray(psi[:, rank * Tl * V3:(rank + 1) * Tl * V3]))
        out = slab.new_field(parity, 0, 2)
        sd.apply(out, inp, parity, M0, dagger=dagger)
        q.put((rank, out.numpy()))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [1, 2, 4])
@pytest.mark.parametrize("parity,dagger", [(0, False), (1, True)])
def test_slab_dirac_over_gloo_matches_oracle(world, parity, dagger):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_run_slab, args=(r, world, port, parity, dagger, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.concatenate([parts[r] for r in range(world)], axis=1)
    g, op, psi = _problem()
    mask = g.parity == parity
    for r in range(2):
        ref = op.apply_schur(psi[r], parity, dagger=dagger)
        assert np.max(np.abs(got[r][mask] - ref[mask])) < 1e-12 * np.max(np.abs(ref))


def test_single_process_exchange_swaps_buffers():
    """Without a process group the faces go back to the same slab (periodic)."""
    su, sd = torch.arange(6.0), torch.arange(6.0) + 10
    ru, rd = torch.zeros(6), torch.zeros(6)
    slabs.exchange_faces(su, sd, ru, rd)
    assert torch.equal(ru, sd) and torch.equal(rd, su)


def _run_slab_cg(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g, op, psi = _problem()
        Tl = T // world
        slab = FakeSlab(op.UR, T, L, rank * Tl, Tl)
        sd = slabs.SlabDirac(slab, prec=0, nrhs=2)
        V3 = L ** 3
        b = torch.from_numpy(np.ascontiguousarray(psi[:, rank * Tl * V3:(rank + 1) * Tl * V3]))
        x = slab.new_field(0, 0, 2)
        it, res = slabs.slab_cg(sd, x, b, 0, M0, 1e-10)
        q.put((rank, x.numpy(), it, res))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [1, 2, 4])
def test_slab_cg_over_gloo_matches_oracle(world):
    """CG on Dhat^+ Dhat over the time slabs of `world` gloo ranks (face exchange
    per operator application, one FP64 all-reduce per global sum) against the
    oracle's CG on the whole lattice, to a true residual of 1e-10."""
    from oracle import solvers
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_run_slab_cg, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = {}
    for _ in range(world):
        rank, x, it, res = q.get(timeout=300)
        parts[rank] = (x, it, res)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    its = {parts[r][1] for r in range(world)}
    assert len(its) == 1                          # every rank ran the same iterations
    assert all(v <= 1e-10 for v in parts[0][2])
    got = np.concatenate([parts[r][0] for r in range(world)], axis=1)
    g, op, psi = _problem()
    ev = g.parity == 0
    for r in range(2):
        b = np.where(ev[:, None, None], psi[r], 0)
        M = lambda v: op.apply_schur(op.apply_schur(v, 0), 0, dagger=True)
        res = np.linalg.norm(b - M(got[r])) / np.linalg.norm(b)
        assert res <= 1.05e-10, res
        x_ref, _, _ = solvers.cg(M, b, 1e-12)
        assert np.linalg.norm(got[r][ev] - x_ref[ev]) <= 1e-8 * np.linalg.norm(x_ref[ev])
