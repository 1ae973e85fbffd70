"""Float-float operator (HR_FF: each real an unevaluated hi + lo pair of FP32
numbers): the pack codes to 48 bits, Dhat / D against the FP64 oracle at the
FP64 tolerance and against the FP64 kernel to a few units of 2^-48, every
launch shape, and the mixed CG whose outer residuals run in float-float,
checked with the oracle's own residual over the whole lattice."""
import numpy as np
import pytest

from gpu_helpers import TOL, from_complex, gpu_lattice, oracle_operator, rel_err, to_complex
from oracle.dirac import Geometry
from paper_2405_19294_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FF = 3
# float-float against the FP64 kernel on the same inputs: each is within a few
# units of 2^-48 (float-float) or 2^-53 (FP64) of the exact result per term
FF_VS_F64 = 5e-14

CLASSES = [(2, "fund"), (3, "fund"), (2, "adj"), (3, "sym"), (4, "asym"), (3, "adj"), (4, "fund"),
           (5, "fund"), (6, "fund"), (3, "asym"), (7, "fund"), (8, "fund")]


def _apply(lat, psi, parity, m0, csw, prec, dagger, nrhs=1):
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


@pytest.mark.parametrize("parity", [0, 1, 2])
def test_pack_codes_ff(hr, parity):
    """hi = fl32(x), lo = fl32(x - hi): hi + lo is x to 2^-48, and unpacking adds them in FP64."""
    T, L, N, rep = 6, 4, 3, "sym"
    lat, _ = gpu_lattice(hr, T, L, N, rep, 1.0, 0.0)
    psi = inputs.gaussian_spinor(3, T, L, lat.d, nrhs=2)
    f = lat.new_field(parity, FF, 2)
    assert f.numel() == lat.new_field(parity, 0, 2).numel()  # the FP64 field size
    lat.pack(f, from_complex(psi), parity, FF, 2)
    out = torch.zeros((2, lat.V, 4, lat.d, 2), dtype=torch.float64, device="cuda")
    lat.unpack(out, f, parity, FF, 2)
    lat.synchronize()
    got = to_complex(out)
    mask = np.ones(lat.V, bool) if parity == 2 else Geometry(T, L).parity == parity
    for part in (np.real, np.imag):
        a, b = part(got[:, mask]), part(psi[:, mask])
        assert np.all(np.abs(a - b) <= 2.0 ** -47 * np.abs(b))
        assert not np.array_equal(a.astype(np.float32).astype(np.float64), a)  # more than FP32 survives
    assert np.all(got[:, ~mask] == 0)


@pytest.mark.parametrize("N,rep", CLASSES)
def test_dphi_ff_parity(hr, N, rep):
    # 6^3 x 10: V/2 = 1080 sites, several blocks and a ragged last block
    T, L, m0, eps = 10, 6, -0.3, 1.0
    lat, _ = gpu_lattice(hr, T, L, N, rep, eps, 0.0)
    op = oracle_operator(T, L, N, rep, eps, m0, 0.0)
    psi = inputs.gaussian_spinor(1, T, L, lat.d)
    g = op.geom
    for parity in (0, 1, 2):
        for dagger in (0, 1):
            got = _apply(lat, psi, parity, m0, 0.0, FF, dagger)[0]
            ref = _oracle_apply(op, psi[0], parity, dagger)
            mask = np.ones(g.V, bool) if parity == 2 else g.parity == parity
            assert rel_err(got, ref, mask) < TOL[0], (parity, dagger)
            f64 = _apply(lat, psi, parity, m0, 0.0, 0, dagger)[0]
            assert rel_err(got, f64, mask) < FF_VS_F64, (parity, dagger, rel_err(got, f64, mask))
            if parity != 2:
                assert np.all(got[~mask] == 0)


@pytest.mark.parametrize("N,rep", [(2, "fund"), (3, "fund"), (2, "adj"), (3, "sym"), (4, "asym")])
def test_dphi_ff_clover_parity(hr, N, rep):
    T, L, m0, csw, eps = 6, 4, -0.35, 1.0, 1.0
    lat, _ = gpu_lattice(hr, T, L, N, rep, eps, csw)
    op = oracle_operator(T, L, N, rep, eps, m0, csw)
    psi = inputs.gaussian_spinor(2, T, L, lat.d)
    g = op.geom
    for parity in (0, 1, 2):
        for dagger in (0, 1):
            got = _apply(lat, psi, parity, m0, csw, FF, dagger)[0]
            ref = _oracle_apply(op, psi[0], parity, dagger)
            mask = np.ones(g.V, bool) if parity == 2 else g.parity == parity
            assert rel_err(got, ref, mask) < TOL[0], (parity, dagger)
    # a new m0 rebuilds the clover blocks and their float-float copies
    got = _apply(lat, psi, 0, -0.2, csw, FF, 0)[0]
    ref = oracle_operator(T, L, N, rep, eps, -0.2, csw).apply_schur(psi[0], 0)
    assert rel_err(got, ref, g.parity == 0) < TOL[0]


def test_ff_links_follow_new_gauge_field(hr):
    """The float-float links are a copy made on first use: representing new links replaces it."""
    T, L, N, rep, m0 = 6, 4, 3, "fund", -0.3
    lat, _ = gpu_lattice(hr, T, L, N, rep, 1.0, 0.0, seed=0)
    psi = inputs.gaussian_spinor(4, T, L, lat.d)
    _apply(lat, psi, 0, m0, 0.0, FF, 0)
    a = inputs.algebra_coefficients(5, T, L, N)
    U = torch.empty((lat.V, 4, N, N, 2), dtype=torch.float64, device="cuda")
    lat.links_from_algebra(U, torch.from_numpy(a).cuda(), 1.0, True)
    lat.represent_links(U, True, 0.0)
    got = _apply(lat, psi, 0, m0, 0.0, FF, 0)[0]
    ref = oracle_operator(T, L, N, rep, 1.0, m0, 0.0, seed=5).apply_schur(psi[0], 0)
    assert rel_err(got, ref, Geometry(T, L).parity == 0) < TOL[0]


@pytest.mark.parametrize("N,rep", [(3, "fund"), (2, "adj"), (6, "fund"), (3, "adj"), (4, "sym"), (6, "adj")])
def test_every_ff_shape(hr, N, rep):
    T, L, m0 = (10, 6, -0.3) if N < 4 or rep == "fund" else (4, 6, -0.3)
    lat, _ = gpu_lattice(hr, T, L, N, rep, 1.0, 0.0)
    psi = inputs.gaussian_spinor(6, T, L, lat.d)
    mask = Geometry(T, L).parity == 0
    f64 = _apply(lat, psi, 0, m0, 0.0, 0, 0)[0]
    shapes = lat.shape_candidates(FF)
    assert shapes
    for sh in shapes:
        lat.set_shape(FF, sh)
        got = _apply(lat, psi, 0, m0, 0.0, FF, 0)[0]
        assert rel_err(got, f64, mask) < FF_VS_F64, sh


LARGE = [(4, "sym"), (6, "asym"), (4, "adj"), (6, "sym"), (5, "adj"), (6, "adj"), (9, "fund"), (12, "fund")]


@pytest.mark.parametrize("N,rep", LARGE)
def test_dphi_ff_parity_large_representations(hr, N, rep):
    """d_R = 9 ... 35: the rows kernel in float-float (several blocks, ragged tail)."""
    T, L, m0, eps = 4, 6, -0.3, 1.0
    lat, _ = gpu_lattice(hr, T, L, N, rep, eps, 0.0)
    op = oracle_operator(T, L, N, rep, eps, m0, 0.0)
    psi = inputs.gaussian_spinor(1, T, L, lat.d)
    g = op.geom
    for parity in (0, 2):
        for dagger in (0, 1):
            got = _apply(lat, psi, parity, m0, 0.0, FF, dagger)[0]
            ref = _oracle_apply(op, psi[0], parity, dagger)
            mask = np.ones(g.V, bool) if parity == 2 else g.parity == parity
            assert rel_err(got, ref, mask) < TOL[0], (parity, dagger)
            f64 = _apply(lat, psi, parity, m0, 0.0, 0, dagger)[0]
            assert rel_err(got, f64, mask) < FF_VS_F64, (parity, dagger, rel_err(got, f64, mask))


@pytest.mark.parametrize("inner", [1, 2])
@pytest.mark.parametrize("N,rep,csw", [(3, "fund", 0.0), (2, "adj", 0.0), (3, "sym", 1.0), (4, "sym", 0.0)])
def test_mixed_cg_ff_outer_oracle_residual(hr, inner, N, rep, csw):
    """The oracle's FP64 residual of the solution meets the target, the residual the
    library reports from its float-float arithmetic agrees with it, and the two outer
    arithmetics give the same x to within the tolerance."""
    T, L, m0, nr = 8, 4, -0.35, 2
    lat, _ = gpu_lattice(hr, T, L, N, rep, 1.0, csw)
    op = oracle_operator(T, L, N, rep, 1.0, m0, csw)
    ev = op.geom.parity == 0
    b = np.where(ev[None, :, None, None], inputs.gaussian_spinor(23, T, L, lat.d, nr), 0)
    fb = lat.new_field(0, 0, nr)
    lat.pack(fb, from_complex(b), 0, 0, nr)
    xs = {}
    for outer in (FF, 0):
        fx = lat.new_field(0, 0, nr)
        st = lat.cg_solve(fx, fb, 0, m0, csw, 1e-10, inner_prec=inner, nrhs=nr, outer_prec=outer)
        assert st["status"] == 0 and 0.0 < st["true_residual"] <= 1e-10, (outer, st)
        out = torch.zeros((nr, lat.V, 4, lat.d, 2), dtype=torch.float64, device="cuda")
        lat.unpack(out, fx, 0, 0, nr)
        lat.synchronize()
        xs[outer] = to_complex(out)
        worst = 0.0
        for k in range(nr):
            r = b[k] - op.apply_schur(op.apply_schur(xs[outer][k], 0), 0, dagger=True)
            worst = max(worst, np.linalg.norm(r) / np.linalg.norm(b[k]))
        assert worst <= 1.05e-10, (outer, worst, st)
        # the reported residual is the largest over the rhs, computed in the outer arithmetic
        assert abs(st["true_residual"] - worst) <= 0.05 * worst, (outer, worst, st)
    for k in range(nr):
        assert rel_err(xs[FF][k], xs[0][k], ev) < 1e-8


def test_ff_outer_falls_back_to_fp64_without_room(hr):
    """When the float-float link copies cannot be allocated (an allocator that refuses every
    request stands in for a full device), the mixed solve keeps FP64 outer residuals: it
    converges, and its residual is bit for bit the FP64-outer solve's (the reductions are
    deterministic)."""
    import ctypes as C
    T, L, N, rep, m0 = 8, 4, 3, "fund", -0.35
    lat, _ = gpu_lattice(hr, T, L, N, rep, 1.0, 0.0)
    ev = Geometry(T, L).parity == 0
    b = np.where(ev[None, :, None, None], inputs.gaussian_spinor(24, T, L, lat.d), 0)
    fb, fx = lat.new_field(0, 0), lat.new_field(0, 0)
    lat.pack(fb, from_complex(b), 0, 0)
    st64 = lat.cg_solve(fx, fb, 0, m0, 0.0, 1e-10, inner_prec=1, outer_prec=0)  # workspaces in place
    refuse = hr._ALLOC_FN(lambda nbytes, ctx: None)
    keep = hr._FREE_FN(lambda ptr, nbytes, ctx: None)
    assert hr._lib.hr_set_allocator(C.cast(refuse, C.c_void_p), C.cast(keep, C.c_void_p), None) == 0
    try:
        st = lat.cg_solve(fx, fb, 0, m0, 0.0, 1e-10, inner_prec=1, outer_prec=FF)
    finally:
        assert hr._lib.hr_set_allocator(None, None, None) == 0
    assert st["status"] == 0 and st["true_residual"] <= 1e-10
    assert st["true_residual"] == st64["true_residual"]
    # with room again, the same call runs in float-float (a different rounding of the same residual)
    st_ff = lat.cg_solve(fx, fb, 0, m0, 0.0, 1e-10, inner_prec=1, outer_prec=FF)
    assert st_ff["status"] == 0 and st_ff["true_residual"] <= 1e-10
    assert st_ff["true_residual"] != st64["true_residual"]
