"""GPU BiCGstab on the operator itself, against the FP64 oracle: the solution's
true residual |b - A x| / |b|, recomputed by the oracle, reaches the target,
for the Schur complement (both parities, with and without clover, several
right-hand sides) and the full operator."""
import numpy as np
import pytest

from gpu_helpers import from_complex, gpu_lattice, oracle_operator, to_complex
from paper_2405_19294_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _solve(hr, lat, b, parity, m0, csw, tol, inner, nrhs=1, outer=3):
    fb = lat.new_field(parity, 0, nrhs)
    fx = lat.new_field(parity, 0, nrhs)
    lat.pack(fb, from_complex(b), parity, 0, nrhs)
    st = lat.bicgstab_solve(fx, fb, parity, m0, csw, tol, inner_prec=inner, nrhs=nrhs, outer_prec=outer)
    out = torch.zeros((nrhs, lat.V, 4, lat.d, 2), dtype=torch.float64, device="cuda")
    lat.unpack(out, fx, parity, 0, nrhs)
    lat.synchronize()
    return to_complex(out), st


@pytest.mark.parametrize("N,rep,csw", [(3, "fund", 0.0), (3, "sym", 1.0), (2, "adj", 0.0), (6, "adj", 0.0)])
@pytest.mark.parametrize("inner,outer", [(0, 0), (1, 3), (1, 0)])  # outer residuals: 3 float-float, 0 FP64
def test_bicgstab_schur(hr, N, rep, csw, inner, outer):
    T, L, m0, nrhs = 6, 4, -0.35, 2
    lat, _ = gpu_lattice(hr, T, L, N, rep, 1.0, csw)
    op = oracle_operator(T, L, N, rep, 1.0, m0, csw)
    for parity in (0, 1):
        b = inputs.gaussian_spinor(3, T, L, lat.d, nrhs)
        b[:, op.geom.parity != parity] = 0
        x, st = _solve(hr, lat, b, parity, m0, csw, 1e-10, inner, nrhs, outer)
        assert 0.0 < st["true_residual"] <= 1e-10
        worst = 0.0
        for r in range(nrhs):
            res = np.linalg.norm(b[r] - op.apply_schur(x[r], parity)) / np.linalg.norm(b[r])
            assert res <= 1.05e-10, (parity, r, res, st)
            worst = max(worst, res)
        # the reported residual (outer arithmetic) is the oracle's, to rounding
        assert abs(st["true_residual"] - worst) <= 0.05 * worst, (parity, worst, st)


def test_bicgstab_full_operator(hr):
    T = L = 4
    lat, _ = gpu_lattice(hr, T, L, 2, "fund", 0.5, 0.0)
    op = oracle_operator(T, L, 2, "fund", 0.5, -0.2, 0.0)
    b = inputs.gaussian_spinor(1, T, L, 2)
    x, st = _solve(hr, lat, b, 2, -0.2, 0.0, 1e-10, 0)
    res = np.linalg.norm(b[0] - op.apply(x[0])) / np.linalg.norm(b[0])
    assert res <= 1.05e-10 and st["true_residual"] <= 1e-10


def test_bicgstab_rejects_fp16_inner(hr):
    lat, _ = gpu_lattice(hr, 4, 4, 3, "fund", 1.0, 0.0)
    fb, fx = lat.new_field(0, 0), lat.new_field(0, 0)
    with pytest.raises(hr.HrError):
        lat.bicgstab_solve(fx, fb, 0, -0.4, 0.0, 1e-10, inner_prec=2)
