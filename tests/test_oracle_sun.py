"""Pins of the oracle's SU(N) layer against mathematics, not against itself.

Every group-theory identity below is independent of how ``oracle.sun`` builds
its matrices: Lie-algebra normalisation and completeness, the SU(2) closed
form of the exponential, scipy's Pade exponential, the QR factorisation, and
the characters and centre charges of each representation.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import sun
from paper_2405_19294_gb300 import inputs

NS = [2, 3, 4, 5, 6]
NS_FUND = NS + [7, 8, 10, 12]   # fundamental-only large-N_c workload
REPS = ["fund", "adj", "sym", "asym"]


def _random_sun(N, n, seed, eps=1.0):
    a = np.random.default_rng(seed).standard_normal((n, N * N - 1))
    return sun.reunitarise(sun.links_from_algebra(a, eps, N))


def _valid(N, rep):
    return not (N == 2 and rep == "asym")


@pytest.mark.parametrize("N", NS_FUND)
def test_generators_normalisation_and_completeness(N):
    T = sun.generators(N)
    assert T.shape == (N * N - 1, N, N)
    assert np.allclose(T, np.conj(np.swapaxes(T, 1, 2)), atol=1e-15)
    assert np.allclose(np.trace(T, axis1=1, axis2=2), 0, atol=1e-15)
    gram = np.einsum("aij,bji->ab", T, T)
    assert np.allclose(gram, 0.5 * np.eye(N * N - 1), atol=1e-14)
    # completeness: sum_a (T_a)_ij (T_a)_kl = (d_il d_jk - d_ij d_kl / N) / 2
    lhs = np.einsum("aij,akl->ijkl", T, T)
    I = np.eye(N)
    rhs = 0.5 * (np.einsum("il,jk->ijkl", I, I) - np.einsum("ij,kl->ijkl", I, I) / N)
    assert np.allclose(lhs, rhs, atol=1e-14)


def test_generators_su2_are_half_pauli():
    T = sun.generators(2)
    sx = np.array([[0, 1], [1, 0]])
    sy = np.array([[0, -1j], [1j, 0]])
    sz = np.array([[1, 0], [0, -1]])
    assert np.allclose(T, 0.5 * np.array([sx, sy, sz]), atol=1e-15)


def test_generators_su3_are_gell_mann():
    # textbook Gell-Mann matrices lambda_1..lambda_8
    l = np.zeros((8, 3, 3), complex)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    order = [0, 1, 3, 4, 5, 6, 2, 7]  # pairs (01),(02),(12) then the diagonals
    assert np.allclose(sun.generators(3), 0.5 * l[order], atol=1e-15)


def test_su2_link_closed_form():
    # exp(i theta n.sigma / 2) = cos(theta/2) + i sin(theta/2) n.sigma
    a = np.random.default_rng(1).standard_normal((50, 3))
    eps = 0.7
    U = sun.links_from_algebra(a, eps, 2)
    theta = eps * np.linalg.norm(a, axis=1)
    n = a / np.linalg.norm(a, axis=1)[:, None]
    sig = np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]])
    ns = np.einsum("xk,kij->xij", n, sig)
    ref = np.cos(theta / 2)[:, None, None] * np.eye(2) + 1j * np.sin(theta / 2)[:, None, None] * ns
    assert np.max(np.abs(U - ref)) < 1e-14


@pytest.mark.parametrize("N", NS_FUND)
def test_links_match_pade_expm_and_are_special_unitary(N):
    a = inputs.algebra_coefficients(7, 2, 2, N).reshape(-1, N * N - 1)[:40]
    eps = 1.0
    U = sun.links_from_algebra(a, eps, N)
    T = sun.generators(N)
    for i in range(len(a)):
        H = np.einsum("k,kij->ij", a[i], T)
        assert np.max(np.abs(U[i] - scipy.linalg.expm(1j * eps * H))) < 1e-13
    assert np.allclose(U @ np.conj(np.swapaxes(U, 1, 2)), np.eye(N), atol=1e-14)
    assert np.allclose(np.linalg.det(U), 1.0, atol=1e-13)


@pytest.mark.parametrize("N", NS_FUND)
def test_reunitarise_matches_qr_and_fixes_det(N):
    rng = np.random.default_rng(3)
    M = rng.standard_normal((30, N, N)) + 1j * rng.standard_normal((30, N, N))
    R = sun.reunitarise(M)
    assert np.allclose(R @ np.conj(np.swapaxes(R, 1, 2)), np.eye(N), atol=1e-13)
    assert np.allclose(np.linalg.det(R), 1.0, atol=1e-13)
    # Gram-Schmidt on rows = QR of M^dagger with positive diagonal R factor;
    # the determinant fix multiplies the last row by a phase only.
    for i in range(len(M)):
        Q, Rf = np.linalg.qr(M[i].conj().T)
        ph = np.diag(Rf) / np.abs(np.diag(Rf))
        Q = Q * ph[None, :]
        rows = Q.conj().T
        assert np.allclose(R[i, :-1], rows[:-1], atol=1e-12)
        ratio = R[i, -1] / rows[-1]
        assert np.allclose(np.abs(ratio), 1.0, atol=1e-12)
        assert np.allclose(ratio, ratio[0], atol=1e-12)


@pytest.mark.parametrize("N", NS_FUND)
def test_reunitarise_is_identity_on_sun(N):
    U = sun.links_from_algebra(np.random.default_rng(5).standard_normal((20, N * N - 1)), 1.0, N)
    assert np.max(np.abs(sun.reunitarise(U) - U)) < 1e-13


@pytest.mark.parametrize("N", NS)
@pytest.mark.parametrize("rep", REPS)
def test_represent_unitary_det1_identity(N, rep):
    if not _valid(N, rep):
        pytest.skip("SU(2) antisymmetric is the trivial singlet")
    d = sun.rep_dim(N, rep)
    U = _random_sun(N, 10, 11)
    R = sun.represent(U, N, rep)
    assert R.shape == (10, d, d)
    assert np.allclose(R @ np.conj(np.swapaxes(R, 1, 2)), np.eye(d), atol=1e-13)
    assert np.allclose(np.linalg.det(R), 1.0, atol=1e-12)
    one = sun.represent(np.eye(N, dtype=complex)[None], N, rep)
    assert np.allclose(one[0], np.eye(d), atol=1e-15)
    if rep == "adj":
        assert np.max(np.abs(R.imag)) == 0.0


@pytest.mark.parametrize("N", NS)
@pytest.mark.parametrize("rep", REPS)
def test_represent_homomorphism(N, rep):
    if not _valid(N, rep):
        pytest.skip()
    U = _random_sun(N, 8, 21)
    W = _random_sun(N, 8, 22)
    lhs = sun.represent(U @ W, N, rep)
    rhs = sun.represent(U, N, rep) @ sun.represent(W, N, rep)
    assert np.allclose(lhs, rhs, atol=1e-13)
    # (U^dagger)_R = (U_R)^dagger
    Ud = np.conj(np.swapaxes(U, 1, 2))
    assert np.allclose(sun.represent(Ud, N, rep),
                       np.conj(np.swapaxes(sun.represent(U, N, rep), 1, 2)), atol=1e-13)


@pytest.mark.parametrize("N", NS)
def test_represent_characters(N):
    U = _random_sun(N, 12, 31)
    tr = np.trace(U, axis1=1, axis2=2)
    tr2 = np.trace(U @ U, axis1=1, axis2=2)
    ch = {rep: np.trace(sun.represent(U, N, rep), axis1=1, axis2=2) for rep in REPS
          if _valid(N, rep)}
    assert np.allclose(ch["fund"], tr, atol=1e-13)
    assert np.allclose(ch["adj"], np.abs(tr) ** 2 - 1, atol=1e-12)
    assert np.allclose(ch["sym"], (tr ** 2 + tr2) / 2, atol=1e-12)
    if N > 2:
        assert np.allclose(ch["asym"], (tr ** 2 - tr2) / 2, atol=1e-12)
    if N == 3:
        assert np.allclose(ch["asym"], np.conj(tr), atol=1e-12)
    if N == 2:
        assert np.allclose(ch["sym"], ch["adj"], atol=1e-12)


@pytest.mark.parametrize("N", NS)
def test_represent_centre_charges(N):
    w = np.exp(2j * np.pi / N)
    Z = (w * np.eye(N))[None]
    assert np.allclose(sun.represent(Z, N, "fund")[0], w * np.eye(N), atol=1e-14)
    assert np.allclose(sun.represent(Z, N, "adj")[0], np.eye(N * N - 1), atol=1e-14)
    assert np.allclose(sun.represent(Z, N, "sym")[0], w ** 2 * np.eye(N * (N + 1) // 2),
                       atol=1e-14)
    if N > 2:
        assert np.allclose(sun.represent(Z, N, "asym")[0], w ** 2 * np.eye(N * (N - 1) // 2),
                           atol=1e-14)


def test_rep_dims():
    assert [sun.rep_dim(3, r) for r in REPS] == [3, 8, 6, 3]
    assert [sun.rep_dim(6, r) for r in REPS] == [6, 35, 21, 15]
