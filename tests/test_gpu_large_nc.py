"""SU(N_c) fundamental fermions for N_c = 7 ... 12 (the large-N_c workload of
Sec. 3.1.2): links from the algebra, the operator in all three precisions with
every candidate launch shape of the autotuner (one-site-per-thread kernel
where it is built, the rows kernel otherwise), the clover term where the
site kernel exists, and a mixed-precision CG."""
import numpy as np
import pytest

from gpu_helpers import TOL, from_complex, gpu_lattice, oracle_links, oracle_operator, rel_err, to_complex
from paper_2405_19294_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("N", [7, 8, 9, 10, 11, 12])
def test_links_from_algebra_large_nc(hr, N):
    T, L = 4, 2
    lat, U = gpu_lattice(hr, T, L, N, "fund", 1.0, 0.0)
    Ug = to_complex(U.view(lat.V, 4, N, N, 2))
    assert np.max(np.abs(Ug - oracle_links(T, L, N, 1.0))) < 1e-13


def _gpu_apply(lat, psi, parity, m0, csw, prec, dagger):
    fin = lat.new_field(parity, prec, 1)
    fout = lat.new_field(parity, prec, 1)
    lat.pack(fin, from_complex(psi), parity, prec, 1)
    lat.dphi(fout, fin, parity, m0, csw, prec, 1, dagger)
    out = torch.zeros((1, lat.V, 4, lat.d, 2), dtype=torch.float64, device="cuda")
    lat.unpack(out, fout, parity, prec, 1)
    lat.synchronize()
    return to_complex(out)[0]


@pytest.mark.parametrize("N", [7, 8, 9, 10, 11, 12])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_dphi_large_nc_every_shape(hr, N, prec):
    # 4 x 6^3: V/2 = 432 sites -> 13.5 tiles of 32 (ragged tail)
    T, L, m0 = 4, 6, -0.3
    lat, _ = gpu_lattice(hr, T, L, N, "fund", 1.0, 0.0)
    op = oracle_operator(T, L, N, "fund", 1.0, m0, 0.0)
    psi = inputs.gaussian_spinor(5, T, L, N)[0]
    g = op.geom
    shapes = lat.shape_candidates(prec)
    assert len(shapes) >= 2
    for sh in shapes:
        lat.set_shape(prec, sh)
        for parity, dagger in ((0, 0), (1, 1), (2, 0)):
            got = _gpu_apply(lat, psi, parity, m0, 0.0, prec, dagger)
            ref = op.apply(psi, dagger=bool(dagger)) if parity == 2 else \
                op.apply_schur(psi, parity, dagger=bool(dagger))
            mask = np.ones(g.V, bool) if parity == 2 else g.parity == parity
            assert rel_err(got, ref, mask) < TOL[prec], (sh, parity, dagger)


@pytest.mark.parametrize("N", [7, 8])
def test_clover_large_nc(hr, N):
    T, L, m0, csw = 4, 4, -0.35, 1.0
    lat, _ = gpu_lattice(hr, T, L, N, "fund", 1.0, csw)
    op = oracle_operator(T, L, N, "fund", 1.0, m0, csw)
    psi = inputs.gaussian_spinor(6, T, L, N)[0]
    for prec in (0, 1):
        got = _gpu_apply(lat, psi, 0, m0, csw, prec, 0)
        ref = op.apply_schur(psi, 0)
        assert rel_err(got, ref, op.geom.parity == 0) < TOL[prec]


def test_cg_large_nc(hr):
    T, L, N, m0 = 4, 6, 10, -0.2
    lat, _ = gpu_lattice(hr, T, L, N, "fund", 1.0, 0.0)
    op = oracle_operator(T, L, N, "fund", 1.0, m0, 0.0)
    g = op.geom
    b = np.where((g.parity == 0)[:, None, None], inputs.gaussian_spinor(3, T, L, N)[0], 0)
    fb = lat.new_field(0, 0, 1)
    fx = lat.new_field(0, 0, 1)
    lat.pack(fb, from_complex(b), 0, 0, 1)
    st = lat.cg_solve(fx, fb, 0, m0, 0.0, 1e-10, inner_prec=1)
    out = torch.zeros((1, lat.V, 4, N, 2), dtype=torch.float64, device="cuda")
    lat.unpack(out, fx, 0, 0, 1)
    lat.synchronize()
    x = to_complex(out)[0]
    r = b - op.apply_schur(op.apply_schur(x, 0), 0, dagger=True)
    # the library stops on its own FP64 true residual <= 1e-10; the oracle's independent
    # evaluation of b - M x differs from it by rounding only, hence the 5 % margin
    assert st["true_residual"] <= 1e-10, st
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.05e-10, st


def test_lattice_rejects_large_nc_two_index(hr):
    with pytest.raises(hr.HrError):
        hr.Lattice(4, 4, 7, "adj")
    with pytest.raises(hr.HrError):
        hr.Lattice(4, 4, 13, "fund")
