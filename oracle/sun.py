"""SU(N) group theory for the oracle: generators, links, representations.

The paper supports fermions "for general higher representations of SU(N_c)"
and calls the link field in representation R the "represented gauge field"
(Sec. 3.1, Sec. 3.1.2) without defining it.  The definitions used here are the
textbook ones:

* generators T_a: generalised Gell-Mann matrices, Hermitian, traceless,
  tr(T_a T_b) = delta_ab / 2;
* links: U = exp(i eps sum_k a_k T_k) with Gaussian a_k (the synthetic input);
* reunitarisation: Gram-Schmidt on the rows, then fix the determinant;
* U -> U_R: the fundamental is U itself, the adjoint acts on the algebra by
  conjugation, the 2-index (anti)symmetric representations act on (anti)
  symmetric tensors psi -> U psi U^T, each written in an orthonormal basis.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np


def rep_dim(N: int, rep: str) -> int:
    """d_R for rep in {fund, adj, sym, asym}."""
    if rep == "fund":
        return N
    if rep == "adj":
        return N * N - 1
    if rep == "sym":
        return N * (N + 1) // 2
    if rep == "asym":
        return N * (N - 1) // 2
    raise ValueError(rep)


def rep_is_real(rep: str) -> bool:
    """The adjoint representation of SU(N) is real; the others are complex."""
    return rep == "adj"


def generators(N: int) -> np.ndarray:
    """Generalised Gell-Mann generators of su(N), shape [N*N-1, N, N].

    Order: for each index pair (j, k), j < k, in lexicographic order, first the
    symmetric (E_jk + E_kj)/2 then the antisymmetric (-i E_jk + i E_kj)/2; then
    the diagonal ones diag(1, ..., 1, -m, 0, ..., 0) / sqrt(2 m (m+1)) for
    m = 1..N-1 (m ones).  For SU(2) this is sigma_x/2, sigma_y/2, sigma_z/2.
    """
    T = []
    for j in range(N):
        for k in range(j + 1, N):
            s = np.zeros((N, N), complex)
            s[j, k] = s[k, j] = 0.5
            a = np.zeros((N, N), complex)
            a[j, k] = -0.5j
            a[k, j] = 0.5j
            T.append(s)
            T.append(a)
    for m in range(1, N):
        dgl = np.zeros(N)
        dgl[:m] = 1.0
        dgl[m] = -m
        T.append(np.diag(dgl / np.sqrt(2.0 * m * (m + 1))).astype(complex))
    return np.array(T)


def algebra_matrix(a: np.ndarray, N: int) -> np.ndarray:
    """H = sum_k a_k T_k for a[..., N*N-1] (Hermitian, traceless)."""
    return np.einsum("...k,kij->...ij", a, generators(N))


def links_from_algebra(a: np.ndarray, eps: float, N: int) -> np.ndarray:
    """U = exp(i eps H), H = sum_k a_k T_k, for a[..., N*N-1].

    The exponential is evaluated through the eigendecomposition of the
    Hermitian H: H = W diag(lam) W^dagger  =>  U = W diag(exp(i eps lam)) W^dagger.
    """
    H = algebra_matrix(a, N)
    lam, W = np.linalg.eigh(H)
    ph = np.exp(1j * eps * lam)
    return np.einsum("...ik,...k,...jk->...ij", W, ph, W.conj())


def reunitarise(U: np.ndarray) -> np.ndarray:
    """Project N x N matrices onto SU(N).

    Modified Gram-Schmidt on the rows in order 0..N-1 (row i loses its
    components along the already-orthonormal rows 0..i-1, one at a time, then
    is normalised), then the last row is multiplied by conj(det U) so that the
    determinant becomes exactly 1 in exact arithmetic.
    """
    U = np.array(U, dtype=complex, copy=True)
    N = U.shape[-1]
    for i in range(N):
        for j in range(i):
            proj = np.sum(U[..., j, :].conj() * U[..., i, :], axis=-1)
            U[..., i, :] = U[..., i, :] - proj[..., None] * U[..., j, :]
        nrm = np.sqrt(np.sum(np.abs(U[..., i, :]) ** 2, axis=-1))
        U[..., i, :] = U[..., i, :] / nrm[..., None]
    det = np.linalg.det(U)
    U[..., N - 1, :] = U[..., N - 1, :] * det.conj()[..., None]
    return U


def two_index_basis(N: int, rep: str) -> np.ndarray:
    """Orthonormal basis e^(ab) of N x N (anti)symmetric matrices, shape [d, N, N].

    sym : pairs a <= b in lexicographic order; e^(aa) = E_aa,
          e^(ab) = (E_ab + E_ba)/sqrt(2) for a < b.
    asym: pairs a < b in lexicographic order; e^(ab) = (E_ab - E_ba)/sqrt(2).
    Orthonormal under <A, B> = tr(A^dagger B).
    """
    basis = []
    for a in range(N):
        for b in range(a, N):
            e = np.zeros((N, N), complex)
            if rep == "sym":
                if a == b:
                    e[a, a] = 1.0
                else:
                    e[a, b] = e[b, a] = 1.0 / np.sqrt(2.0)
            elif rep == "asym":
                if a == b:
                    continue
                e[a, b] = 1.0 / np.sqrt(2.0)
                e[b, a] = -1.0 / np.sqrt(2.0)
            else:
                raise ValueError(rep)
            basis.append(e)
    return np.array(basis)


def represent(U: np.ndarray, N: int, rep: str) -> np.ndarray:
    """Map fundamental links U[..., N, N] to U_R[..., d, d] (complex128 array).

    fund : U_R = U
    adj  : (U_R)_ab = 2 Re tr(T_a U T_b U^dagger)          (real matrix)
    sym, asym : (U_R)_(ab),(cd) = tr(e^(ab)^dagger U e^(cd) U^T)
    """
    U = np.asarray(U, dtype=complex)
    if rep == "fund":
        return U.copy()
    if rep == "adj":
        T = generators(N)
        # T_a U T_b U^dagger, traced
        UT = np.einsum("...ij,bjk->...bik", U, T)              # U T_b
        UTU = np.einsum("...bik,...lk->...bil", UT, U.conj())   # U T_b U^dagger
        tr = np.einsum("aji,...bij->...ab", T, UTU)             # tr(T_a X_b)
        return (2.0 * tr.real).astype(complex)
    e = two_index_basis(N, rep)
    UeUt = np.einsum("...ij,cjk,...lk->...cil", U, e, U)        # U e^(cd) U^T
    return np.einsum("aij,...cij->...ac", e.conj(), UeUt)       # tr(e^dag X) = sum conj(e)_ij X_ij
