"""Time-slab decomposition on the GPU: n slabs of one lattice (hr_domains_dphi,
device-to-device exchange) and the begin / end entry points with
caller-owned buffers reproduce the oracle's Dhat of the whole lattice in all
three precisions, both parities and the adjoint."""
import numpy as np
import pytest

from gpu_helpers import TOL, from_complex, oracle_operator, rel_err, to_complex
from oracle.dirac import Geometry
from paper_2405_19294_gb300 import inputs, slabs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _slabs(hr, T, L, N, rep, n, eps=1.0, seed=0):
    a = inputs.algebra_coefficients(seed, T, L, N)
    Tl, V3 = T // n, L ** 3
    lats = []
    for k in range(n):
        lat = hr.Lattice(Tl, L, N, rep, t0=k * Tl, T_global=T)
        ak = torch.from_numpy(np.ascontiguousarray(a[k * Tl * V3:(k + 1) * Tl * V3])).cuda()
        U = torch.empty((lat.V, 4, N, N, 2), dtype=torch.float64, device="cuda")
        lat.links_from_algebra(U, ak, eps, True)
        lat.represent_links(U, True, 0.0)
        lats.append(lat)
    return lats


def _pack(lat, psi_slab, parity, prec):
    f = lat.new_field(parity, prec)
    lat.pack(f, from_complex(psi_slab), parity, prec)
    return f


def _unpack(lat, f, parity, prec):
    out = torch.zeros((1, lat.V, 4, lat.d, 2), dtype=torch.float64, device="cuda")
    lat.unpack(out, f, parity, prec)
    return to_complex(out)[0]


@pytest.mark.parametrize("N,rep", [(3, "fund"), (2, "adj"), (3, "sym"), (4, "fund")])
@pytest.mark.parametrize("n", [1, 2, 4])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_domains_dphi_matches_oracle(hr, N, rep, n, prec):
    T, L, m0 = 8, 4, -0.3
    lats = _slabs(hr, T, L, N, rep, n)
    op = oracle_operator(T, L, N, rep, 1.0, m0, 0.0)
    psi = inputs.gaussian_spinor(4, T, L, lats[0].d)[0]
    V3, Tl = L ** 3, T // n
    g = op.geom
    for parity, dagger in ((0, 0), (1, 1), (0, 1)):
        ins = [_pack(l, psi[None, k * Tl * V3:(k + 1) * Tl * V3], parity, prec) for k, l in enumerate(lats)]
        outs = [l.new_field(parity, prec) for l in lats]
        hr.domains_dphi(lats, outs, ins, parity, m0, prec, dagger=bool(dagger))
        got = np.concatenate([_unpack(l, outs[k], parity, prec) for k, l in enumerate(lats)])
        ref = op.apply_schur(psi, parity, dagger=bool(dagger))
        mask = g.parity == parity
        assert rel_err(got, ref, mask) < TOL[prec], (parity, dagger)
        assert np.all(got[~mask] == 0)


@pytest.mark.parametrize("prec", [0, 1])
def test_slab_dirac_begin_end_two_slabs_one_process(hr, prec):
    """The caller-owned-buffer path: two slabs, the exchange done by hand."""
    T, L, N, rep, m0 = 8, 6, 3, "fund", -0.4
    lats = _slabs(hr, T, L, N, rep, 2)
    op = oracle_operator(T, L, N, rep, 1.0, m0, 0.0)
    psi = inputs.gaussian_spinor(5, T, L, N)[0]
    V3, Tl = L ** 3, T // 2
    ins = [_pack(l, psi[None, k * Tl * V3:(k + 1) * Tl * V3], 0, prec) for k, l in enumerate(lats)]
    tmps = [l.new_field(1, prec) for l in lats]
    outs = [l.new_field(0, prec) for l in lats]
    bufs = [[l.new_halo(prec) for _ in range(4)] for l in lats]
    for stage in (0, 1):
        for k, l in enumerate(lats):
            o, ih = (tmps[k], ins[k]) if stage == 0 else (outs[k], tmps[k])
            l.domain_hop_begin(o, ih, ins[k] if stage else None, 1 - stage, m0, prec, stage,
                               bufs[k][0], bufs[k][1])
        for k in range(2):
            bufs[k][2].copy_(bufs[(k + 1) % 2][1])   # receive-up <- send-down of the slab above
            bufs[k][3].copy_(bufs[(k + 1) % 2][0])   # receive-down <- send-up of the slab below
        for k, l in enumerate(lats):
            o = tmps[k] if stage == 0 else outs[k]
            l.domain_hop_end(o, 1 - stage, m0, prec, stage, bufs[k][2], bufs[k][3])
    got = np.concatenate([_unpack(l, outs[k], 0, prec) for k, l in enumerate(lats)])
    ref = op.apply_schur(psi, 0)
    assert rel_err(got, ref, op.geom.parity == 0) < TOL[prec]


def test_slab_dirac_single_rank(hr):
    """slabs.SlabDirac on one rank (one slab covering the lattice) equals hr_dphi."""
    T, L, N, rep, m0 = 8, 4, 3, "sym", -0.3
    lat = _slabs(hr, T, L, N, rep, 1)[0]
    op = oracle_operator(T, L, N, rep, 1.0, m0, 0.0)
    psi = inputs.gaussian_spinor(6, T, L, lat.d)[0]
    f = _pack(lat, psi[None], 0, 1)
    out = lat.new_field(0, 1)
    slabs.SlabDirac(lat, prec=1).apply(out, f, 0, m0)
    assert rel_err(_unpack(lat, out, 0, 1), op.apply_schur(psi, 0), op.geom.parity == 0) < TOL[1]


def test_slab_errors(hr):
    with pytest.raises(hr.HrError):
        hr.Lattice(3, 4, 3, "fund", t0=0, T_global=8)      # odd slab
    with pytest.raises(hr.HrError):
        hr.Lattice(4, 4, 3, "fund", t0=6, T_global=8)      # past the end
    lats = _slabs(hr, 8, 4, 3, "fund", 2)
    f = [l.new_field(0, 1) for l in lats]
    with pytest.raises(hr.HrError):
        hr.domains_dphi(lats[::-1], [l.new_field(0, 1) for l in lats[::-1]], f[::-1], 0, -0.3, 1)  # out of order
    lat = hr.Lattice(4, 4, 3, "fund", t0=0, T_global=8)
    U = torch.zeros((lat.V, 4, 3, 3, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(hr.HrError):
        lat.represent_links(U, False, 1.0)                  # clover on a slab


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_axpby(hr, prec):
    """hr_axpby: y = a x + b y per rhs, against NumPy on the unpacked fields."""
    T, L, N, rep = 4, 4, 3, "sym"
    lat = _slabs(hr, T, L, N, rep, 1)[0]
    psi = inputs.gaussian_spinor(7, T, L, lat.d, nrhs=3)
    phi = inputs.gaussian_spinor(8, T, L, lat.d, nrhs=3)
    x, y = lat.new_field(0, prec, 3), lat.new_field(0, prec, 3)
    lat.pack(x, from_complex(psi), 0, prec, 3)
    lat.pack(y, from_complex(phi), 0, prec, 3)

    def back(f):
        out = torch.zeros((3, lat.V, 4, lat.d, 2), dtype=torch.float64, device="cuda")
        lat.unpack(out, f, 0, prec, 3)
        return to_complex(out)
    xs, ys = back(x), back(y)
    a, b = [0.5, -2.0, 0.0], [1.5, 0.25, 0.0]
    lat.axpby(x, y, a, b, 0, prec, 3)
    got = back(y)
    ev = Geometry(T, L).parity == 0
    for r in range(3):
        ref = a[r] * xs[r] + b[r] * ys[r]
        if r == 2:
            assert np.all(got[r][ev] == 0)
        else:
            assert rel_err(got[r], ref, ev) < {0: 1e-15, 1: 1e-7, 2: 1e-3}[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_slab_cg_on_one_slab(hr, prec):
    """slabs.slab_cg driving libhr (hr_axpby, hr_norm2, the slab hops) on one slab
    that spans the lattice: FP64 true residual of the oracle's operator <= 1e-10
    (FP64 fields), or the FP32 floor (FP32 fields)."""
    T, L, N, rep, m0 = 8, 4, 3, "fund", -0.3
    lat = _slabs(hr, T, L, N, rep, 1)[0]
    op = oracle_operator(T, L, N, rep, 1.0, m0, 0.0)
    ev = op.geom.parity == 0
    b = np.where(ev[:, None, None], inputs.gaussian_spinor(9, T, L, lat.d)[0], 0)
    fb = _pack(lat, b[None], 0, prec)
    fx = lat.new_field(0, prec)
    sd = slabs.SlabDirac(lat, prec)
    tol = 1e-10 if prec == 0 else 1e-4
    it, res = slabs.slab_cg(sd, fx, fb, 0, m0, tol)
    x = _unpack(lat, fx, 0, prec)
    r = b - op.apply_schur(op.apply_schur(x, 0), 0, dagger=True)
    true = np.linalg.norm(r) / np.linalg.norm(b)
    assert res[0] <= tol and true <= (1.05e-10 if prec == 0 else 2e-4), (it, res, true)


def _slab_cg_rank(rank, world, port, q):
    import os
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2405_19294_gb300 import hr
        T, L, N, rep, m0 = 8, 4, 3, "fund", -0.3
        Tl, V3 = T // world, L ** 3
        lat = _slabs(hr, T, L, N, rep, world)[rank]      # this rank's slab (all built, one kept)
        ev = Geometry(T, L).parity == 0
        b = np.where(ev[:, None, None], inputs.gaussian_spinor(9, T, L, lat.d)[0], 0)
        fb = _pack(lat, b[None, rank * Tl * V3:(rank + 1) * Tl * V3], 0, 0)
        fx = lat.new_field(0, 0)
        it, res = slabs.slab_cg(slabs.SlabDirac(lat, 0), fx, fb, 0, m0, 1e-10)
        q.put((rank, _unpack(lat, fx, 0, 0), it, res))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_slab_cg_two_processes(hr, world):
    """slabs.slab_cg over two gloo ranks, each a separate process driving libhr's slab
    kernels (bulk hop with masked faces, face packing and completion, hr_axpby,
    hr_norm2) on this GPU; the faces and the FP64 all-reduces go through the host.
    The kernels of the two processes never wait on each other.  The assembled
    solution meets the oracle's whole-lattice residual bound."""
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_slab_cg_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = dict((r, (x, it, res)) for r, x, it, res in (q.get(timeout=300) for _ in procs))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert len({parts[r][1] for r in parts}) == 1
    T, L, N, rep, m0 = 8, 4, 3, "fund", -0.3
    op = oracle_operator(T, L, N, rep, 1.0, m0, 0.0)
    x = np.concatenate([parts[r][0] for r in range(world)])
    ev = op.geom.parity == 0
    b = np.where(ev[:, None, None], inputs.gaussian_spinor(9, T, L, 3)[0], 0)
    r = b - op.apply_schur(op.apply_schur(x, 0), 0, dagger=True)
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.05e-10
