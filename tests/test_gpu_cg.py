"""GPU conjugate gradient vs the FP64 oracle: the solution's true residual,
recomputed by the oracle, must reach the target, and the 4^4 SU(2) case is
compared with a dense LAPACK solve."""
import numpy as np
import pytest
import scipy.linalg

from gpu_helpers import from_complex, gpu_lattice, oracle_operator, to_complex
from paper_2405_19294_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _solve(hr, lat, b, parity, m0, csw, tol, inner, nrhs=1, inner_tol=0.0):
    fb = lat.new_field(parity, 0, nrhs)
    fx = lat.new_field(parity, 0, nrhs)
    lat.pack(fb, from_complex(b), parity, 0, nrhs)
    st = lat.cg_solve(fx, fb, parity, m0, csw, tol, inner_prec=inner, inner_tol=inner_tol, nrhs=nrhs)
    out = torch.zeros((nrhs, lat.V, 4, lat.d, 2), dtype=torch.float64, device="cuda")
    lat.unpack(out, fx, parity, 0, nrhs)
    lat.synchronize()
    return to_complex(out), st


def _normal(op, parity):
    if parity == 2:
        return lambda v: op.apply(op.apply(v), dagger=True)
    return lambda v: op.apply_schur(op.apply_schur(v, parity), parity, dagger=True)


def test_cg_full_su2_4x4_dense(hr):
    """SU(2) fundamental 4^4, eps 0.5, m0 -0.2, csw 0: plain FP64 CG on D^+D to 1e-10."""
    T = L = 4
    lat, _ = gpu_lattice(hr, T, L, 2, "fund", 0.5, 0.0)
    op = oracle_operator(T, L, 2, "fund", 0.5, -0.2, 0.0)
    b = inputs.gaussian_spinor(1, T, L, 2)
    x, st = _solve(hr, lat, b, 2, -0.2, 0.0, 1e-10, hr.F64)
    M = _normal(op, 2)
    res = np.linalg.norm(b[0] - M(x[0])) / np.linalg.norm(b[0])
    assert res <= 1.05e-10 and st["true_residual"] <= 1e-10
    # dense reference
    n = g_n = lat.V * 4 * 2
    cols = []
    for j in range(n):
        e = np.zeros(n, complex)
        e[j] = 1
        cols.append(M(e.reshape(lat.V, 4, 2)).ravel())
    Md = np.array(cols).T
    xd = scipy.linalg.solve(Md, b[0].ravel())
    assert np.linalg.norm(x[0].ravel() - xd) / np.linalg.norm(xd) < 1e-10 * np.linalg.cond(Md)
    assert st["outer_steps"] >= 1 and st["iterations"] > 5


@pytest.mark.parametrize("inner", [0, 1, 2])
def test_cg_even_schur(hr, inner):
    T, L, N, rep, m0 = 10, 6, 3, "fund", -0.4
    lat, _ = gpu_lattice(hr, T, L, N, rep, 1.0, 0.0)
    op = oracle_operator(T, L, N, rep, 1.0, m0, 0.0)
    b = inputs.gaussian_spinor(1, T, L, lat.d)
    b[0][op.geom.parity == 1] = 0
    x, st = _solve(hr, lat, b, 0, m0, 0.0, 1e-10, inner)
    M = _normal(op, 0)
    res = np.linalg.norm(b[0] - M(x[0])) / np.linalg.norm(b[0])
    assert res <= 1.05e-10, (res, st)
    assert np.all(x[0][op.geom.parity == 1] == 0)
    if inner != 0:
        assert st["outer_steps"] >= 2


@pytest.mark.parametrize("N,rep,inner", [(3, "sym", 1), (2, "adj", 2), (4, "asym", 2)])
def test_cg_multi_rhs_clover(hr, N, rep, inner):
    T, L, m0, csw, nrhs = 6, 4, -0.35, 1.0, 3
    lat, _ = gpu_lattice(hr, T, L, N, rep, 1.0, csw)
    op = oracle_operator(T, L, N, rep, 1.0, m0, csw)
    b = inputs.gaussian_spinor(1, T, L, lat.d, nrhs)
    b[:, op.geom.parity == 1] = 0
    x, st = _solve(hr, lat, b, 0, m0, csw, 1e-10, inner, nrhs=nrhs)
    M = _normal(op, 0)
    for r in range(nrhs):
        res = np.linalg.norm(b[r] - M(x[r])) / np.linalg.norm(b[r])
        assert res <= 1.05e-10, (r, res, st)
