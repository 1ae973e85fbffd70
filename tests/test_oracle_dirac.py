"""Pins of the oracle's Wilson(-clover) operator against physics and brute force.

* Clifford algebra and gamma_5 of the gamma basis;
* free field (U = 1): plane waves are exact eigenvectors of D with the
  momentum-space closed form, and of the Schur complement with its own;
* constant abelian links shift the momentum by the weight phases;
* gamma_5-hermiticity of D and Dhat, with and without clover;
* gauge covariance under random local SU(N) transformations (all reps);
* clover: Hermitian, commutes with gamma_5, traceless, vanishes on trivial
  and constant abelian fields, closed form on a constant abelian field strength;
* brute force on 2^4 / 2x4^3: dense D assembled from matrix elements, its
  adjoint, and its dense Schur complement;
* the FP16 per-site code: max maps to +-1, rounding bound.
"""
import numpy as np
import pytest

from oracle import dirac, sun
from oracle.dirac import GAMMA, GAMMA5, Geometry, WilsonOperator
from paper_2405_19294_gb300 import inputs

CASES = [(2, "fund"), (3, "fund"), (2, "adj"), (3, "sym"), (4, "asym"), (3, "adj")]


def _links(N, T, L, eps, seed):
    a = inputs.algebra_coefficients(seed, T, L, N)
    return sun.reunitarise(sun.links_from_algebra(a, eps, N))


def _spinor(T, L, d, seed):
    return inputs.gaussian_spinor(seed, T, L, d)[0]


def _ip(a, b):
    return np.vdot(a.ravel(), b.ravel())


def _g5(psi):
    return np.einsum("st,xta->xsa", GAMMA5, psi)


def test_clifford_and_gamma5():
    for mu in range(4):
        assert np.allclose(GAMMA[mu], GAMMA[mu].conj().T)
        for nu in range(4):
            ac = GAMMA[mu] @ GAMMA[nu] + GAMMA[nu] @ GAMMA[mu]
            assert np.allclose(ac, 2.0 * (mu == nu) * np.eye(4))
    assert np.allclose(GAMMA5, np.diag([1, 1, -1, -1]))
    for mu in range(4):
        assert np.allclose(GAMMA5 @ GAMMA[mu], -GAMMA[mu] @ GAMMA5)


def _plane_wave(geom, p, u):
    phase = np.exp(1j * geom.coords @ p)
    return phase[:, None, None] * u[None]


def _free_symbol(p, m0):
    # D(p) = m0 + sum_mu (1 - cos p_mu) + i sum_mu gamma_mu sin p_mu   (4x4)
    return (m0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * np.einsum("m,mst->st", np.sin(p),
                                                                        GAMMA)


@pytest.mark.parametrize("N,rep", CASES)
def test_free_field_plane_waves(N, rep):
    T, L, m0 = 6, 4, -0.3
    g = Geometry(T, L)
    d = sun.rep_dim(N, rep)
    U = np.broadcast_to(np.eye(N, dtype=complex), (g.V, 4, N, N)).copy()
    op = WilsonOperator(U, N, rep, g, m0, csw=1.3)  # clover vanishes on U = 1
    rng = np.random.default_rng(0)
    for _ in range(4):
        n = rng.integers(0, [T, L, L, L])
        p = np.array([np.pi * (2 * n[0] + 1) / T] + [2 * np.pi * n[k] / L for k in (1, 2, 3)])
        u = rng.standard_normal((4, d)) + 1j * rng.standard_normal((4, d))
        psi = _plane_wave(g, p, u)
        Dp = _free_symbol(p, m0)
        ref = _plane_wave(g, p, Dp @ u)
        assert np.max(np.abs(op.apply(psi) - ref)) < 1e-12
        # Schur complement: Dhat_e = (4+m0) - H(p)^2 / (4 (4+m0)),
        # H(p) = 2 sum cos p - 2 i sum gamma sin p
        Hp = 2 * np.sum(np.cos(p)) * np.eye(4) - 2j * np.einsum("m,mst->st", np.sin(p), GAMMA)
        c = 4 + m0
        Sp = c * np.eye(4) - Hp @ Hp / (4 * c)
        for par in (0, 1):
            out = op.apply_schur(psi, par)
            ref = np.where((g.parity == par)[:, None, None], _plane_wave(g, p, Sp @ u), 0)
            assert np.max(np.abs(out - ref)) < 1e-12


@pytest.mark.parametrize("rep", ["fund", "sym", "asym"])
def test_constant_abelian_links_shift_momentum(rep):
    N, T, L, m0 = 3, 4, 4, 0.1
    g = Geometry(T, L)
    rng = np.random.default_rng(4)
    th = rng.uniform(-np.pi, np.pi, size=(4, N))
    th[:, -1] = -th[:, :-1].sum(axis=1)      # det = 1
    U = np.zeros((g.V, 4, N, N), complex)
    for mu in range(4):
        U[:, mu] = np.diag(np.exp(1j * th[mu]))
    op = WilsonOperator(U, N, rep, g, m0)
    # weights of the basis vectors of each representation
    if rep == "fund":
        w = th
    else:
        pairs = [(a, b) for a in range(N) for b in range(a, N) if rep == "sym" or a < b]
        w = np.array([[th[mu, a] + th[mu, b] for (a, b) in pairs] for mu in range(4)])
    d = w.shape[1]
    n = np.array([1, 2, 0, 3])
    p = np.array([np.pi * (2 * n[0] + 1) / T] + [2 * np.pi * n[k] / L for k in (1, 2, 3)])
    for c in range(d):
        u = np.zeros((4, d), complex)
        u[:, c] = rng.standard_normal(4) + 1j * rng.standard_normal(4)
        psi = _plane_wave(g, p, u)
        # the antiperiodic sign on the last time slice is absorbed by p_0
        q = p + w[:, c]
        ref = _plane_wave(g, p, np.einsum("st,ta->sa", _free_symbol(q, m0), u))
        assert np.max(np.abs(op.apply(psi) - ref)) < 1e-12


@pytest.mark.parametrize("N,rep", CASES)
@pytest.mark.parametrize("csw", [0.0, 1.0])
def test_gamma5_hermiticity(N, rep, csw):
    T, L = 4, 4
    g = Geometry(T, L)
    d = sun.rep_dim(N, rep)
    op = WilsonOperator(_links(N, T, L, 0.8, 1), N, rep, g, -0.2, csw)
    chi, psi = _spinor(T, L, d, 2), _spinor(T, L, d, 3)
    lhs = _ip(chi, op.apply(psi))
    rhs = _ip(_g5(op.apply(_g5(chi))), psi)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    # the oracle's D^dagger is gamma_5 D gamma_5 and is the adjoint
    assert np.max(np.abs(op.apply(psi, dagger=True) - _g5(op.apply(_g5(psi))))) < 1e-12
    assert abs(_ip(op.apply(chi, dagger=True), psi) - lhs) < 1e-11 * abs(lhs)
    for par in (0, 1):
        lhs = _ip(chi, op.apply_schur(psi, par))
        rhs = _ip(op.apply_schur(chi, par, dagger=True), psi)
        assert abs(lhs - rhs) < 1e-11 * abs(lhs)
        assert np.max(np.abs(op.apply_schur(psi, par, dagger=True)
                             - _g5(op.apply_schur(_g5(psi), par)))) < 1e-12


@pytest.mark.parametrize("N,rep", CASES + [(5, "sym")])
def test_gauge_covariance(N, rep):
    T, L, m0, csw = 4, 4, -0.3, 1.0
    g = Geometry(T, L)
    d = sun.rep_dim(N, rep)
    U = _links(N, T, L, 1.0, 5)
    Om = sun.reunitarise(sun.links_from_algebra(
        inputs.gauge_transform_coefficients(6, T, L, N), 1.0, N))
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[:, mu] = Om @ U[:, mu] @ np.conj(np.swapaxes(Om[g.fwd[mu]], 1, 2))
    OmR = sun.represent(Om, N, rep)
    psi = _spinor(T, L, d, 7)
    psig = np.einsum("xab,xsb->xsa", OmR, psi)
    op, opg = WilsonOperator(U, N, rep, g, m0, csw), WilsonOperator(Ug, N, rep, g, m0, csw)
    lhs = opg.apply(psig)
    rhs = np.einsum("xab,xsb->xsa", OmR, op.apply(psi))
    assert np.max(np.abs(lhs - rhs)) < 1e-11
    lhs = opg.apply_schur(psig, 0)
    rhs = np.einsum("xab,xsb->xsa", OmR, op.apply_schur(psi, 0))
    assert np.max(np.abs(lhs - rhs)) < 1e-11
    # A(x) -> Omega_R(x) A(x) Omega_R(x)^dagger
    OR4 = np.einsum("st,xab->xsatb", np.eye(4), OmR).reshape(g.V, 4 * d, 4 * d)
    assert np.allclose(opg.A, OR4 @ op.A @ np.conj(np.swapaxes(OR4, 1, 2)), atol=1e-11)


@pytest.mark.parametrize("N,rep", CASES)
def test_clover_algebraic_properties(N, rep):
    T, L = 4, 4
    g = Geometry(T, L)
    d = sun.rep_dim(N, rep)
    m0, csw = -0.35, 1.0
    op = WilsonOperator(_links(N, T, L, 1.0, 8), N, rep, g, m0, csw)
    A = op.A
    assert np.allclose(A, np.conj(np.swapaxes(A, 1, 2)), atol=1e-13)
    G5 = np.kron(GAMMA5, np.eye(d))
    assert np.allclose(G5 @ A, A @ G5, atol=1e-13)
    assert np.allclose(np.trace(A, axis1=1, axis2=2), (4 + m0) * 4 * d, atol=1e-12)
    assert np.max(np.abs(A - (4 + m0) * np.eye(4 * d))) > 1e-2   # not trivially zero


def test_clover_vanishes_on_constant_abelian_links():
    N, T, L = 3, 4, 4
    g = Geometry(T, L)
    th = np.random.default_rng(9).uniform(-3, 3, size=(4, N))
    th[:, -1] = -th[:, :-1].sum(axis=1)
    U = np.zeros((g.V, 4, N, N), complex)
    for mu in range(4):
        U[:, mu] = np.diag(np.exp(1j * th[mu]))
    for rep in ("fund", "adj", "sym", "asym"):
        op = WilsonOperator(U, N, rep, g, 0.2, csw=1.7)
        assert np.allclose(op.A, 4.2 * np.eye(4 * sun.rep_dim(N, rep)), atol=1e-13)


def test_clover_closed_form_constant_field_strength():
    """U_2(x) = diag(e^{iBx}, e^{-iBx}), others 1: every 1-2 plaquette is diag(e^{iB}, e^{-iB}).

    Then Fhat_12 = diag(i sin B, -i sin B) = -Fhat_21, every other plane
    vanishes (the time-boundary sign cancels inside each plaquette), and
    A = (4+m0) + c_sw (i/2) sigma_12 (x) Fhat_12 = (4+m0) - (c_sw/2) sin B sigma_12 (x) diag(1,-1).
    """
    T, L, m0, csw = 4, 4, -0.1, 1.3
    g = Geometry(T, L)
    B = 2 * np.pi / L
    x = g.coords[:, 1]
    U = np.broadcast_to(np.eye(2, dtype=complex), (g.V, 4, 2, 2)).copy()
    U[:, 2, 0, 0] = np.exp(1j * B * x)
    U[:, 2, 1, 1] = np.exp(-1j * B * x)
    op = WilsonOperator(U, 2, "fund", g, m0, csw)
    ref = (4 + m0) * np.eye(8) - 0.5 * csw * np.sin(B) * np.kron(dirac.sigma(1, 2),
                                                                 np.diag([1.0, -1.0]))
    assert np.max(np.abs(op.A - ref[None])) < 1e-13
    sites = np.arange(g.V)
    F = dirac.field_strength(op.UR, g, 1, 2, sites)
    assert np.allclose(F, np.diag([1j * np.sin(B), -1j * np.sin(B)])[None], atol=1e-14)


def _dense_from_elements(op):
    """Dense D from its matrix elements, site block by site block (no gathers)."""
    g, d, UR = op.geom, op.d, op.UR
    n = 4 * d
    D = np.zeros((g.V * n, g.V * n), complex)
    for x in range(g.V):
        blk = slice(x * n, (x + 1) * n)
        D[blk, blk] += op.A[x] if op.A is not None else (4 + op.m0) * np.eye(n)
        for mu in range(4):
            y = g.fwd[mu][x]
            D[blk, y * n:(y + 1) * n] += -0.5 * np.kron(np.eye(4) - GAMMA[mu], UR[x, mu])
            y = g.bwd[mu][x]
            D[blk, y * n:(y + 1) * n] += -0.5 * np.kron(np.eye(4) + GAMMA[mu],
                                                        UR[y, mu].conj().T)
    return D


def _dense_by_columns(apply, V, d):
    n = V * 4 * d
    cols = []
    for j in range(n):
        e = np.zeros(n, complex)
        e[j] = 1
        cols.append(apply(e.reshape(V, 4, d)).ravel())
    return np.array(cols).T


@pytest.mark.parametrize("N,rep,T,L", [(2, "fund", 2, 2), (3, "fund", 2, 2), (2, "adj", 4, 2),
                                       (3, "sym", 2, 2)])
@pytest.mark.parametrize("csw", [0.0, 1.0])
def test_brute_force_dense(N, rep, T, L, csw):
    g = Geometry(T, L)
    d = sun.rep_dim(N, rep)
    op = WilsonOperator(_links(N, T, L, 1.0, 12), N, rep, g, -0.25, csw)
    Dm = _dense_from_elements(op)
    Dc = _dense_by_columns(op.apply, g.V, d)
    assert np.max(np.abs(Dm - Dc)) < 1e-13
    Dd = _dense_by_columns(lambda v: op.apply(v, dagger=True), g.V, d)
    assert np.max(np.abs(Dd - Dm.conj().T)) < 1e-13
    # Schur complement from dense blocks
    n = 4 * d
    ev = np.repeat(g.parity == 0, n)
    od = ~ev
    for par, (P, Q) in ((0, (ev, od)), (1, (od, ev))):
        S = Dm[np.ix_(P, P)] - Dm[np.ix_(P, Q)] @ np.linalg.solve(Dm[np.ix_(Q, Q)],
                                                                  Dm[np.ix_(Q, P)])
        Sc = _dense_by_columns(lambda v: op.apply_schur(v, par), g.V, d)[np.ix_(P, P)]
        assert np.max(np.abs(S - Sc)) < 1e-12


def test_sampled_schur_equals_full():
    N, rep, T, L = 3, "sym", 4, 4
    g = Geometry(T, L)
    d = sun.rep_dim(N, rep)
    op = WilsonOperator(_links(N, T, L, 1.0, 13), N, rep, g, -0.3, 1.0)
    psi = _spinor(T, L, d, 14)
    full = op.apply_schur(psi, 0, dagger=True)
    sites = g.sites_of_parity(0)[[0, 5, 17, 60, 127]]
    part = op.apply_schur(psi, 0, dagger=True, sites=sites)
    assert np.max(np.abs(part[sites] - full[sites])) < 1e-13


def test_fp16_code():
    v = np.random.default_rng(15).standard_normal((1000, 24)) * 10.0 ** np.random.default_rng(
        16).uniform(-3, 3, size=(1000, 1))
    v[3] = 0.0
    h, s = dirac.encode_fp16(v)
    assert h.dtype == np.float16 and s.dtype == np.float32
    assert np.all(np.max(np.abs(h.astype(np.float64)), axis=1)[np.arange(1000) != 3] == 1.0)
    dec = dirac.decode_fp16(h, s)
    assert np.all(dec[3] == 0.0) and s[3] == 0.0
    # |v - decode| <= |v| 2^-24 (to FP32) + scale 2^-11 (to FP16, half ulp at 1) + tiny
    err = np.abs(dec - v)
    assert np.all(err <= np.abs(v) * 2.0 ** -23 + s[:, None].astype(np.float64) * 2.0 ** -11)


def test_lazy_evaluation_matches_eager():
    """The lazily evaluated operator (used for full-size sampled checks) equals the eager one."""
    N, rep, T, L = 3, "sym", 4, 4
    g = Geometry(T, L)
    a = inputs.algebra_coefficients(21, T, L, N)
    U = sun.reunitarise(sun.links_from_algebra(a, 1.0, N))
    eager = WilsonOperator(U, N, rep, g, -0.35, 1.0)
    lazy = WilsonOperator(None, N, rep, g, -0.35, 1.0,
                          link_fn=lambda s: sun.reunitarise(sun.links_from_algebra(a[s], 1.0, N)))
    psi = _spinor(T, L, eager.d, 22)
    sites = g.sites_of_parity(1)[[0, 3, 50, 127]]
    for dag in (False, True):
        ref = eager.apply_schur(psi, 1, dagger=dag)
        got = lazy.apply_schur(psi, 1, dagger=dag, sites=sites)
        assert np.max(np.abs(got[sites] - ref[sites])) < 1e-13


@pytest.mark.parametrize("N,rep", [(2, "fund"), (3, "sym"), (2, "adj")])
def test_exponentiated_clover(N, rep):
    """A = (4+m0) exp(C/(4+m0)): Hermitian, commutes with gamma_5, positive, inverse by -C,
    first-order agreement with the standard clover term, gauge covariant."""
    T, L, m0 = 4, 4, -0.35
    g = Geometry(T, L)
    d = sun.rep_dim(N, rep)
    U = _links(N, T, L, 1.0, 30)
    c = 4 + m0
    op_e = WilsonOperator(U, N, rep, g, m0, 1.0, exponential=True)
    op_s = WilsonOperator(U, N, rep, g, m0, 1.0)
    A = op_e.A
    assert np.allclose(A, np.conj(np.swapaxes(A, 1, 2)), atol=1e-12)
    G5 = np.kron(GAMMA5, np.eye(d))
    assert np.allclose(G5 @ A, A @ G5, atol=1e-12)
    assert np.all(np.linalg.eigvalsh(A) > 0)                 # exp of Hermitian: positive definite
    C = op_s.A - c * np.eye(4 * d)
    import scipy.linalg
    for x in (0, 17, 100):
        Ainv = scipy.linalg.expm(-C[x] / c) / c
        assert np.allclose(A[x] @ Ainv, np.eye(4 * d), atol=1e-12)
        # eigenvalues are c exp(lambda / c) of C's eigenvalues lambda
        lam = np.linalg.eigvalsh(C[x])
        assert np.allclose(np.sort(np.linalg.eigvalsh(A[x])), np.sort(c * np.exp(lam / c)), atol=1e-11)
    # small c_sw: exponentiated and standard agree to first order, differ at second
    small_e = WilsonOperator(U, N, rep, g, m0, 1e-3, exponential=True).A
    small_s = WilsonOperator(U, N, rep, g, m0, 1e-3).A
    diff = np.max(np.abs(small_e - small_s))
    assert 0 < diff < 1e-5
    # trivial field: no clover term either way
    U1 = np.broadcast_to(np.eye(N, dtype=complex), U.shape).copy()
    assert np.allclose(WilsonOperator(U1, N, rep, g, m0, 1.0, exponential=True).A, c * np.eye(4 * d), atol=1e-13)
