"""GPU (C ABI) vs FP64 oracle parity on lattices that span several thread
blocks and end in a ragged tail: links, represented links, clover blocks,
pack/unpack codes, the operator in all three precisions and both parities,
its adjoint, and the norm reduction."""
import numpy as np
import pytest

from gpu_helpers import TOL, from_complex, gpu_lattice, oracle_links, oracle_operator, rel_err, to_complex
from oracle import dirac, sun
from oracle.dirac import Geometry
from paper_2405_19294_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SMALL = [(2, "fund"), (3, "fund"), (2, "adj"), (3, "sym"), (4, "asym"), (3, "adj"), (4, "fund"),
         (5, "fund"), (6, "fund"), (3, "asym")]


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6])
def test_links_from_algebra(hr, N):
    T, L = 4, 4
    lat, U = gpu_lattice(hr, T, L, N, "fund", 1.0, 0.0)
    Ug = to_complex(U.view(lat.V, 4, N, N, 2))
    Uo = oracle_links(T, L, N, 1.0)
    assert np.max(np.abs(Ug - Uo)) < 1e-13
    # without reunitarisation: still SU(N) to rounding (scaling and squaring of exp)
    lat2, U2 = gpu_lattice(hr, T, L, N, "fund", 1.0, 0.0, reunitarise=False)
    Uo2 = oracle_links(T, L, N, 1.0, reunitarise=False)
    assert np.max(np.abs(to_complex(U2) - Uo2)) < 1e-13


@pytest.mark.parametrize("N,rep", SMALL + [(6, "adj"), (6, "sym"), (5, "asym")])
def test_represented_links(hr, N, rep):
    T, L = 4, 2
    lat, _ = gpu_lattice(hr, T, L, N, rep, 1.0, 0.0)
    d = lat.d
    UR = torch.empty((lat.V, 4, d, d, 2), dtype=torch.float64, device="cuda")
    lat.export_represented_links(UR)
    g = Geometry(T, L)
    ref = dirac.represented_field(oracle_links(T, L, N, 1.0), N, rep, g)
    assert np.max(np.abs(to_complex(UR) - ref)) < 1e-13


def _pack_roundtrip(hr, lat, psi, parity, prec, nrhs=1):
    f = lat.new_field(parity, prec, nrhs)
    lat.pack(f, from_complex(psi), parity, prec, nrhs)
    out = torch.zeros((nrhs, lat.V, 4, lat.d, 2), dtype=torch.float64, device="cuda")
    lat.unpack(out, f, parity, prec, nrhs)
    return to_complex(out)


@pytest.mark.parametrize("parity", [0, 1, 2])
def test_pack_codes(hr, parity):
    T, L, N, rep = 6, 4, 3, "sym"
    lat, _ = gpu_lattice(hr, T, L, N, rep, 1.0, 0.0)
    psi = inputs.gaussian_spinor(3, T, L, lat.d, nrhs=2)
    g = Geometry(T, L)
    mask = np.ones(g.V, bool) if parity == 2 else g.parity == parity
    r64 = _pack_roundtrip(hr, lat, psi, parity, 0, 2)
    assert np.array_equal(r64[:, mask], psi[:, mask])
    assert np.all(r64[:, ~mask] == 0)
    r32 = _pack_roundtrip(hr, lat, psi, parity, 1, 2)
    ref32 = psi.real.astype(np.float32).astype(np.float64) + 1j * psi.imag.astype(np.float32).astype(np.float64)
    assert np.array_equal(r32[:, mask], ref32[:, mask])
    # FP16 code is bit-exact against the oracle's encoding
    r16 = _pack_roundtrip(hr, lat, psi, parity, 2, 2)
    h, s = dirac.encode_fp16(dirac.spinor_site_reals(psi))
    ref16 = dirac.spinor_from_site_reals(dirac.decode_fp16(h, s), lat.d)
    assert np.array_equal(r16[:, mask], ref16[:, mask])


def _gpu_apply(lat, psi, parity, m0, csw, prec, dagger, nrhs=1):
    fin = lat.new_field(parity, prec, nrhs)
    fout = lat.new_field(parity, prec, nrhs)
    lat.pack(fin, from_complex(psi), parity, prec, nrhs)
    lat.dphi(fout, fin, parity, m0, csw, prec, nrhs, dagger)
    out = torch.zeros((nrhs, lat.V, 4, lat.d, 2), dtype=torch.float64, device="cuda")
    lat.unpack(out, fout, parity, prec, nrhs)
    lat.synchronize()
    return to_complex(out)


def _oracle_apply(op, psi, parity, dagger):
    if parity == 2:
        return op.apply(psi, dagger=bool(dagger))
    return op.apply_schur(psi, parity, dagger=bool(dagger))


@pytest.mark.parametrize("N,rep", SMALL)
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_dphi_parity(hr, N, rep, prec):
    # 6^3 x 10: V/2 = 1080 sites -> 9 blocks of 128 with a ragged last block
    T, L, m0, eps = 10, 6, -0.3, 1.0
    lat, _ = gpu_lattice(hr, T, L, N, rep, eps, 0.0)
    op = oracle_operator(T, L, N, rep, eps, m0, 0.0)
    psi = inputs.gaussian_spinor(1, T, L, lat.d)
    g = op.geom
    for parity in (0, 1, 2):
        for dagger in (0, 1):
            got = _gpu_apply(lat, psi, parity, m0, 0.0, prec, dagger)[0]
            ref = _oracle_apply(op, psi[0], parity, dagger)
            mask = np.ones(g.V, bool) if parity == 2 else g.parity == parity
            err = rel_err(got, ref, mask)
            assert err < TOL[prec], (parity, dagger, err)
            if parity != 2:
                assert np.all(got[~mask] == 0)


@pytest.mark.parametrize("N,rep", [(2, "fund"), (3, "fund"), (2, "adj"), (3, "sym"), (4, "asym"), (3, "adj")])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_dphi_clover_parity(hr, N, rep, prec):
    T, L, m0, csw, eps = 6, 4, -0.35, 1.0, 1.0
    lat, _ = gpu_lattice(hr, T, L, N, rep, eps, csw)
    op = oracle_operator(T, L, N, rep, eps, m0, csw)
    psi = inputs.gaussian_spinor(2, T, L, lat.d)
    g = op.geom
    for parity in (0, 1, 2):
        for dagger in (0, 1):
            got = _gpu_apply(lat, psi, parity, m0, csw, prec, dagger)[0]
            ref = _oracle_apply(op, psi[0], parity, dagger)
            mask = np.ones(g.V, bool) if parity == 2 else g.parity == parity
            assert rel_err(got, ref, mask) < TOL[prec], (parity, dagger)


@pytest.mark.parametrize("N,rep", [(2, "fund"), (3, "sym"), (2, "adj")])
def test_clover_blocks(hr, N, rep):
    T, L, m0, csw = 4, 4, -0.35, 1.3
    lat, _ = gpu_lattice(hr, T, L, N, rep, 1.0, csw)
    op = oracle_operator(T, L, N, rep, 1.0, m0, csw)
    d = lat.d
    A = torch.empty((lat.V, 2, 2 * d, 2 * d, 2), dtype=torch.float64, device="cuda")
    lat.export_clover(A, m0, inverse=False)
    Ag = to_complex(A)
    Ao = op.A
    for b in range(2):
        blk = Ao[:, 2 * b * d:(2 * b + 2) * d, 2 * b * d:(2 * b + 2) * d]
        assert np.max(np.abs(Ag[:, b] - blk)) < 1e-13
    # off-diagonal chirality blocks of the oracle's A vanish
    assert np.max(np.abs(Ao[:, :2 * d, 2 * d:])) < 1e-14
    lat.export_clover(A, m0, inverse=True)
    Ig = to_complex(A)
    for b in range(2):
        blk = Ao[:, 2 * b * d:(2 * b + 2) * d, 2 * b * d:(2 * b + 2) * d]
        assert np.max(np.abs(Ig[:, b] - np.linalg.inv(blk))) < 1e-12


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("parity", [0, 2])
def test_norm2(hr, prec, parity):
    T, L, N, rep = 6, 6, 3, "fund"
    lat, _ = gpu_lattice(hr, T, L, N, rep, 1.0, 0.0)
    nrhs = 3
    psi = inputs.gaussian_spinor(4, T, L, lat.d, nrhs)
    f = lat.new_field(parity, prec, nrhs)
    lat.pack(f, from_complex(psi), parity, prec, nrhs)
    got = lat.norm2(f, parity, prec, nrhs)
    back = _pack_roundtrip(hr, lat, psi, parity, prec, nrhs)
    g = Geometry(T, L)
    mask = np.ones(g.V, bool) if parity == 2 else g.parity == 0
    for r in range(nrhs):
        ref = np.sum(np.abs(back[r, mask]) ** 2)
        assert abs(got[r] - ref) <= 1e-6 * ref if prec else abs(got[r] - ref) <= 1e-13 * ref
    # deterministic: bit-identical on repeat
    assert lat.norm2(f, parity, prec, nrhs) == got


def test_multi_rhs_dphi_matches_single(hr):
    """Every multi-rhs launch shape gives each rhs the single-rhs result to the FP32
    rounding level (the kernels differ in summation order, register budget and, for
    the tensor-core kernel, the TF32 splitting)."""
    T, L, N, rep, m0 = 4, 4, 3, "fund", -0.4
    lat, _ = gpu_lattice(hr, T, L, N, rep, 1.0, 0.0)
    psi = inputs.gaussian_spinor(5, T, L, lat.d, nrhs=3)
    ones = [_gpu_apply(lat, psi[r:r + 1], 0, m0, 0.0, 1, 0, nrhs=1)[0] for r in range(3)]
    mask = Geometry(T, L).parity == 0
    for sh in lat.shape_candidates(1, nrhs=3):
        lat.set_shape(1, sh, nrhs=3)
        many = _gpu_apply(lat, psi, 0, m0, 0.0, 1, 0, nrhs=3)
        for r in range(3):
            assert rel_err(many[r], ones[r], mask) < 1e-6, sh


def test_errors_are_reported(hr):
    with pytest.raises(hr.HrError):
        hr.Lattice(3, 4, 3, "fund")        # odd T
    with pytest.raises(hr.HrError):
        hr.Lattice(4, 4, 2, "asym")        # trivial singlet
    with pytest.raises(hr.HrError):
        hr.Lattice(4, 4, 13, "fund")       # N out of range
    lat = hr.Lattice(4, 4, 3, "fund")
    f = lat.new_field(0, 1)
    with pytest.raises(hr.HrError):
        lat.dphi(lat.new_field(0, 1), f, 0, -0.4, 0.0, 1)   # links not loaded
    lat2, _ = gpu_lattice(hr, 4, 4, 3, "fund", 1.0, 0.0)
    with pytest.raises(hr.HrError):
        lat2.dphi(lat2.new_field(0, 1), lat2.new_field(0, 1), 0, -0.4, 1.0, 1)  # csw mismatch


LARGE = [(4, "sym"), (6, "asym"), (6, "sym"), (4, "adj"), (5, "adj"), (6, "adj"), (5, "asym")]


@pytest.mark.parametrize("N,rep", LARGE)
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_dphi_parity_large_representations(hr, N, rep, prec):
    """d_R = 10 ... 35: the colour-split kernel (several thread blocks, ragged tail)."""
    T, L, m0, eps = 4, 6, -0.3, 1.0
    lat, _ = gpu_lattice(hr, T, L, N, rep, eps, 0.0)
    op = oracle_operator(T, L, N, rep, eps, m0, 0.0)
    psi = inputs.gaussian_spinor(1, T, L, lat.d)
    g = op.geom
    for parity in (0, 2):
        for dagger in (0, 1):
            got = _gpu_apply(lat, psi, parity, m0, 0.0, prec, dagger)[0]
            ref = _oracle_apply(op, psi[0], parity, dagger)
            mask = np.ones(g.V, bool) if parity == 2 else g.parity == parity
            err = rel_err(got, ref, mask)
            assert err < TOL[prec], (parity, dagger, err)


@pytest.mark.parametrize("N,rep", [(3, "fund"), (3, "adj"), (3, "sym"), (4, "sym"), (6, "asym"), (5, "adj"), (4, "adj"),
                                   (6, "sym"), (6, "adj")])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_every_tuner_shape_is_correct(hr, N, rep, prec):
    """Each candidate launch shape of the autotuner, pinned in turn, matches the oracle."""
    T, L, m0, eps = 4, 6, -0.3, 1.0
    lat, _ = gpu_lattice(hr, T, L, N, rep, eps, 0.0)
    op = oracle_operator(T, L, N, rep, eps, m0, 0.0)
    psi = inputs.gaussian_spinor(7, T, L, lat.d)
    ref = _oracle_apply(op, psi[0], 0, 0)
    mask = op.geom.parity == 0
    shapes = lat.shape_candidates(prec)
    assert len(shapes) >= 1
    for sh in shapes:
        lat.set_shape(prec, sh)
        got = _gpu_apply(lat, psi, 0, m0, 0.0, prec, 0)[0]
        assert rel_err(got, ref, mask) < TOL[prec], sh
        assert lat.tuned_shape(prec) == sh


def test_autotuner_records_a_choice(hr):
    lat, _ = gpu_lattice(hr, 8, 8, 3, "fund", 1.0, 0.0)
    psi = inputs.gaussian_spinor(8, 8, 8, 3)
    _gpu_apply(lat, psi, 0, -0.4, 0.0, 1, 0)
    sh = lat.tuned_shape(1)
    assert sh is not None and sh in lat.shape_candidates(1)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_pack_unpack_direct_from_pinned_host(hr, prec):
    """Page-locked host buffers are read / written by the kernels in place (no staging copy)."""
    import ctypes
    T, L, N, rep = 6, 4, 3, "fund"
    lat, _ = gpu_lattice(hr, T, L, N, rep, 1.0, 0.0)
    psi = inputs.gaussian_spinor(9, T, L, lat.d, nrhs=2)
    host = torch.from_numpy(np.stack([psi.real, psi.imag], -1)).pin_memory()
    dev = host.cuda()
    f_host, f_dev = lat.new_field(0, prec, 2), lat.new_field(0, prec, 2)
    lat.pack(f_host, host, 0, prec, 2)
    lat.pack(f_dev, dev, 0, prec, 2)
    torch.cuda.synchronize()
    assert torch.equal(f_host, f_dev)
    out_host = torch.zeros_like(host).pin_memory()
    out_dev = torch.zeros_like(dev)
    lat.unpack(out_host, f_dev, 0, prec, 2)
    lat.unpack(out_dev, f_dev, 0, prec, 2)
    torch.cuda.synchronize()
    assert torch.equal(out_host, out_dev.cpu())
    # pageable host memory is refused by the C ABI (nothing is launched)
    page = np.zeros(host.numel(), dtype=np.float64)
    lib = hr.lib_handle()
    rc = lib.hr_pack_spinor(lat._h, ctypes.c_void_p(f_dev.data_ptr()), ctypes.c_void_p(page.ctypes.data), 0, prec, 2)
    assert rc == -1


@pytest.mark.parametrize("N,rep,csw", [(3, "fund", 0.0), (3, "sym", 1.0), (2, "adj", 0.0), (3, "adj", 1.0),
                                       (6, "adj", 0.0), (5, "fund", 1.0), (3, "fund", 1.0)])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_every_multi_rhs_shape_is_correct(hr, N, rep, csw, prec):
    """Several right-hand sides at once, every candidate shape (incl. the link-staging kernel)."""
    T, L, m0, eps, nrhs = 4, 6, -0.35, 1.0, 5
    lat, _ = gpu_lattice(hr, T, L, N, rep, eps, csw)
    op = oracle_operator(T, L, N, rep, eps, m0, csw)
    psi = inputs.gaussian_spinor(12, T, L, lat.d, nrhs)
    mask = op.geom.parity == 0
    refs = [_oracle_apply(op, psi[r], 0, 0) for r in range(nrhs)]
    shapes = lat.shape_candidates(prec, nrhs=nrhs, clover=csw != 0.0)
    assert len(shapes) >= 1
    for sh in shapes:
        lat.set_shape(prec, sh, nrhs=nrhs, clover=csw != 0.0)
        got = _gpu_apply(lat, psi, 0, m0, csw, prec, 0, nrhs=nrhs)
        for r in range(nrhs):
            assert rel_err(got[r], refs[r], mask) < TOL[prec], (sh, r)


def test_torch_caching_allocator_backs_library_buffers(hr):
    """hr_set_allocator: the links, rows layout and Schur intermediate come from
    PyTorch's pool and go back to it when the lattice is destroyed."""
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    hr.use_torch_allocator(True)
    try:
        lat, U = gpu_lattice(hr, 8, 8, 4, "sym", 1.0, 0.0)
        links_bytes = 2 * 4 * lat.d * lat.d * lat.Vh * (16 + 8 + 4)
        grown = torch.cuda.memory_allocated() - before
        assert grown >= links_bytes
        op = oracle_operator(8, 8, 4, "sym", 1.0, -0.3, 0.0)
        psi = inputs.gaussian_spinor(3, 8, 8, lat.d)
        got = _gpu_apply(lat, psi, 0, -0.3, 0.0, 1, 0)[0]
        assert rel_err(got, op.apply_schur(psi[0], 0), op.geom.parity == 0) < TOL[1]
        del U
        lat.close()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() - before < links_bytes // 4
    finally:
        hr.use_torch_allocator(False)
    lat2, _ = gpu_lattice(hr, 4, 4, 3, "fund", 1.0, 0.0)   # back on cudaMalloc
    lat2.close()


@pytest.mark.parametrize("N,rep", [(3, "fund"), (2, "adj"), (3, "adj"), (3, "sym"), (5, "fund"), (4, "adj"),
                                   (6, "adj")])
def test_fp16_error_stays_near_storage_rounding(hr, N, rep):
    """FP16 Dhat keeps the error of FP16 storage: the half2 projection and the
    FP16 x FP16 -> FP32 products (site kernel; rows kernel for real links) add
    one FP16 rounding of the half-spinor, measured at about 3e-4 relative.  A
    bound of 1e-3, well inside the 5e-3 parity tolerance, catches an
    accumulation that slipped to FP16."""
    T, L, m0, eps = 4, 6, -0.3, 1.0
    lat, _ = gpu_lattice(hr, T, L, N, rep, eps, 0.0)
    op = oracle_operator(T, L, N, rep, eps, m0, 0.0)
    psi = inputs.gaussian_spinor(3, T, L, lat.d)
    mask = op.geom.parity == 0
    ref = _oracle_apply(op, psi[0], 0, 0)
    for sh in lat.shape_candidates(2):
        lat.set_shape(2, sh)
        got = _gpu_apply(lat, psi, 0, m0, 0.0, 2, 0)[0]
        assert rel_err(got, ref, mask) < 1e-3, sh


@pytest.mark.parametrize("N,rep,T,csw", [(2, "fund", 2, 0.0), (3, "fund", 2, 1.0), (2, "adj", 2, 0.0),
                                         (3, "sym", 4, 0.0)])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_dphi_parity_smallest_lattice(hr, N, rep, T, csw, prec):
    """L = 2 (and T = 2): the forward and backward neighbours coincide, so the
    two hops of each direction land on the same site and must both be added;
    V/2 = 4 T sites, one ragged tile."""
    L, m0, eps = 2, -0.3, 1.0
    lat, _ = gpu_lattice(hr, T, L, N, rep, eps, csw)
    op = oracle_operator(T, L, N, rep, eps, m0, csw)
    psi = inputs.gaussian_spinor(5, T, L, lat.d)
    g = op.geom
    for parity in (0, 1, 2):
        for dagger in (0, 1):
            got = _gpu_apply(lat, psi, parity, m0, csw, prec, dagger)[0]
            ref = _oracle_apply(op, psi[0], parity, dagger)
            mask = np.ones(g.V, bool) if parity == 2 else g.parity == parity
            assert rel_err(got, ref, mask) < TOL[prec], (parity, dagger)


TC_SHAPE = (0, 0, 0, 66, 0)    # tensor-core multi-rhs kernel (16 sites per block)


@pytest.mark.parametrize("N,rep,csw", [(3, "sym", 1.0), (4, "asym", 0.0), (4, "fund", 1.0), (3, "fund", 0.0),
                                       (5, "fund", 0.0)])
@pytest.mark.parametrize("prec", [1, 2])
def test_tensor_core_multi_rhs(hr, N, rep, csw, prec):
    """The tensor-core multi-rhs kernel against the oracle: 12 rhs (three 4-rhs MMA
    tiles) and 17 rhs (a full 16-rhs block plus a block of one), Schur and full
    operator, both signs, on 6^4 (V/2 = 648 = 40.5 tiles of 16: a ragged last tile)."""
    T, L, m0, eps = 6, 6, -0.35, 1.0
    lat, _ = gpu_lattice(hr, T, L, N, rep, eps, csw)
    op = oracle_operator(T, L, N, rep, eps, m0, csw)
    g = op.geom
    assert TC_SHAPE in [tuple(s) for s in lat.shape_candidates(prec, nrhs=12, clover=csw != 0.0)]
    for nrhs, cases in ((12, ((0, 0), (0, 1), (2, 0))), (17, ((1, 1),))):
        psi = inputs.gaussian_spinor(13, T, L, lat.d, nrhs)
        lat.set_shape(prec, TC_SHAPE, nrhs=nrhs, clover=csw != 0.0)
        for parity, dagger in cases:
            got = _gpu_apply(lat, psi, parity, m0, csw, prec, dagger, nrhs=nrhs)
            mask = np.ones(g.V, bool) if parity == 2 else g.parity == parity
            for r in range(nrhs):
                ref = _oracle_apply(op, psi[r], parity, dagger)
                err = rel_err(got[r], ref, mask)
                assert err < (1e-6 if prec == 1 else 1e-3), (nrhs, parity, dagger, r, err)

