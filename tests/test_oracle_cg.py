"""Pins of the oracle's conjugate gradient: dense LAPACK solves on small lattices.

The 4^4 SU(2) fundamental workload (dimension 2048) is solved densely with
LAPACK and compared with CG on D^dagger D; the even-odd route (Schur
complement on the even sites, reconstruction of the odd sites) must give the
same full-lattice solution.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import solvers, sun
from oracle.dirac import Geometry, WilsonOperator
from paper_2405_19294_gb300 import inputs


def _dense(apply, V, d):
    n = V * 4 * d
    cols = []
    for j in range(n):
        e = np.zeros(n, complex)
        e[j] = 1
        cols.append(apply(e.reshape(V, 4, d)).ravel())
    return np.array(cols).T


def _setup(N, rep, T, L, eps, m0, csw, seed_links=0, seed_src=1):
    g = Geometry(T, L)
    a = inputs.algebra_coefficients(seed_links, T, L, N)
    U = sun.reunitarise(sun.links_from_algebra(a, eps, N))
    op = WilsonOperator(U, N, rep, g, m0, csw)
    b = inputs.gaussian_spinor(seed_src, T, L, op.d)[0]
    return g, op, b


def test_cg_su2_fund_4x4_matches_lapack():
    """SU(2) fundamental, 4^4, eps = 0.5, m0 = -0.2, csw = 0, plain FP64 CG on D^+D to 1e-10."""
    g, op, b = _setup(2, "fund", 4, 4, 0.5, -0.2, 0.0)
    D = _dense(op.apply, g.V, op.d)
    x_ref = scipy.linalg.solve(D, b.ravel())
    x, it = solvers.solve_wilson_full(op, b, 1e-10)
    rel = np.linalg.norm(x.ravel() - x_ref) / np.linalg.norm(x_ref)
    cond = np.linalg.cond(D)
    assert rel < 1e-10 * cond
    assert np.linalg.norm(D @ x.ravel() - b.ravel()) / np.linalg.norm(b) < 1e-10 * cond
    # normal-equation residual that CG controls
    M = D.conj().T @ D
    rhs = D.conj().T @ b.ravel()
    assert np.linalg.norm(M @ x.ravel() - rhs) / np.linalg.norm(rhs) <= 1e-10
    assert 5 < it < 2000


@pytest.mark.parametrize("csw", [0.0, 1.0])
def test_even_odd_solve_reconstructs_full_solution(csw):
    g, op, b = _setup(3, "sym", 2, 4, 1.0, -0.3, csw)
    D = _dense(op.apply, g.V, op.d)
    x_ref = scipy.linalg.solve(D, b.ravel()).reshape(b.shape)
    x, _ = solvers.solve_wilson_eo(op, b, 1e-12)
    assert np.max(np.abs(x - x_ref)) / np.max(np.abs(x_ref)) < 1e-8


def test_cg_normal_equations_true_residual():
    g, op, b = _setup(2, "adj", 4, 2, 1.0, -0.3, 0.0)
    be = np.where((g.parity == 0)[:, None, None], b, 0)
    M = lambda v: op.apply_schur(op.apply_schur(v, 0), 0, dagger=True)
    x, it, res = solvers.cg(M, be, 1e-10)
    r = be - M(x)
    assert np.linalg.norm(r) / np.linalg.norm(be) <= 1e-10
    assert res <= 1e-10
    # odd sites stay untouched by the even Schur operator
    assert np.all(x[g.parity == 1] == 0)


@pytest.mark.parametrize("csw", [0.0, 1.0])
def test_bicgstab_schur_matches_lapack(csw):
    """BiCGstab on Dhat_e x = b directly reproduces the dense solution of the Schur system."""
    g, op, b = _setup(3, "fund", 4, 4, 1.0, -0.35, csw)
    ev = g.parity == 0
    be = np.where(ev[:, None, None], b, 0)
    A = lambda v: op.apply_schur(v, 0)
    x, it, res = solvers.bicgstab(A, be, 1e-10)
    assert res <= 1e-10
    Dm = _dense(lambda v: op.apply_schur(v, 0), g.V, op.d)
    n = 4 * op.d
    mask = np.repeat(ev, n)
    xd = scipy.linalg.solve(Dm[np.ix_(mask, mask)], be.ravel()[mask])
    assert np.linalg.norm(x.ravel()[mask] - xd) / np.linalg.norm(xd) < 1e-8
    # fewer operator applications than CG on the normal equations
    M = lambda v: op.apply_schur(op.apply_schur(v, 0), 0, dagger=True)
    rhs = op.apply_schur(be, 0, dagger=True)
    _, it_cg, _ = solvers.cg(M, rhs, 1e-10)
    assert 2 * it <= 2 * it_cg + 4


def test_bicgstab_nonhermitian_small_dense():
    """A random well-conditioned non-Hermitian matrix: BiCGstab against LAPACK."""
    rng = np.random.default_rng(33)
    n = 60
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A *= 0.5
    bb = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, it, res = solvers.bicgstab(lambda v: A @ v, bb, 1e-12)
    assert res <= 1e-12
    assert np.allclose(x, np.linalg.solve(A, bb), atol=1e-9)
