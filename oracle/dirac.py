"""Wilson(-clover) Dirac operator in representation R, FP64, for the oracle.

The paper (Sec. 3.1) provides the Wilson-Dirac operator "for general higher
representations of SU(N_c)" with even-odd preconditioning and clover
(Sheikholeslami-Wohlert) improvement, and (Sec. 2.2) applies the spin
projection (1 -/+ gamma_mu) so that only half-spinors travel.  It prints no
formula; the standard definitions written out below are the reading used:

    D psi(x) = A(x) psi(x)
               - 1/2 sum_mu [ (1 - gamma_mu) U_R,mu(x) psi(x + mu)
                            + (1 + gamma_mu) U_R,mu(x - mu)^dagger psi(x - mu) ]

    A(x) = (4 + m0) + c_sw (i/4) sum_{mu,nu} sigma_mu_nu Fhat_mu_nu(x),
    sigma_mu_nu = (i/2) [gamma_mu, gamma_nu],
    Fhat_mu_nu  = (Q_mu_nu - Q_mu_nu^dagger) / 8,
    Q_mu_nu     = sum of the four counter-clockwise plaquette leaves at x,

with periodic space and antiperiodic time, the latter realised by flipping
the sign of U_R,0 on the last time slice.  Even-odd preconditioning uses the
Schur complement on parity p = (t+x+y+z) mod 2:

    Dhat_p = A_pp - D_pq A_qq^{-1} D_qp,        q = 1 - p.

Gamma matrices: the chiral, Hermitian (Euclidean) basis
    gamma_0 = [[0, -1], [-1, 0]],  gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
    gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3 = diag(1, 1, -1, -1).

Spinor fields are complex arrays psi[V][4][d] (site lexicographic
((t*L+z)*L+y)*L+x, spin, colour).  Links are U[V][4][N][N], direction 0 = t.

The oracle applies the full 4x4 gamma matrices (it never uses the
half-spinor shortcut) and full 4d x 4d clover matrices (it never uses their
chiral block structure), so that it stays a direct transcription.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np

from . import sun

# ---------------------------------------------------------------- gammas ----
_PAULI = np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=complex)
_I2 = np.eye(2, dtype=complex)
_Z2 = np.zeros((2, 2), dtype=complex)


def _block(a, b, c, d):
    return np.block([[a, b], [c, d]])


GAMMA = np.array(
    [_block(_Z2, -_I2, -_I2, _Z2)]
    + [_block(_Z2, -1j * _PAULI[k], 1j * _PAULI[k], _Z2) for k in range(3)]
)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
I4 = np.eye(4, dtype=complex)


def sigma(mu: int, nu: int) -> np.ndarray:
    """sigma_mu_nu = (i/2) [gamma_mu, gamma_nu]."""
    return 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])


# -------------------------------------------------------------- geometry ----
class Geometry:
    """Periodic T x L^3 lattice with lexicographic site order.

    ``coords[x] = (t, x, y, z)`` in direction order mu = 0..3; ``fwd[mu][x]``
    and ``bwd[mu][x]`` are the neighbours x + mu and x - mu (periodic wrap);
    ``parity[x] = (t + x + y + z) mod 2``.
    """

    def __init__(self, T: int, L: int):
        self.T, self.L = T, L
        self.V = T * L ** 3
        idx = np.arange(self.V)
        x = idx % L
        y = (idx // L) % L
        z = (idx // (L * L)) % L
        t = idx // (L ** 3)
        self.coords = np.stack([t, x, y, z], axis=1)
        self.extent = np.array([T, L, L, L])
        self.parity = (t + x + y + z) % 2
        self.fwd = np.empty((4, self.V), dtype=np.int64)
        self.bwd = np.empty((4, self.V), dtype=np.int64)
        for mu in range(4):
            e = np.zeros(4, dtype=np.int64)
            e[mu] = 1
            self.fwd[mu] = self.lex((self.coords + e) % self.extent)
            self.bwd[mu] = self.lex((self.coords - e) % self.extent)

    def lex(self, c: np.ndarray) -> np.ndarray:
        """Lexicographic index of coordinates c[..., 4] = (t, x, y, z)."""
        L = self.L
        return ((c[..., 0] * L + c[..., 3]) * L + c[..., 2]) * L + c[..., 1]

    def sites_of_parity(self, p: int) -> np.ndarray:
        return np.nonzero(self.parity == p)[0]


# ------------------------------------------------------ represented links ----
def represented_field(U: np.ndarray, N: int, rep: str, geom: Geometry) -> np.ndarray:
    """U_R[V][4][d][d] from fundamental links, with the antiperiodic-time sign.

    The fermion boundary condition in time is antiperiodic; it is realised by
    multiplying U_R,0 on the last time slice (t = T-1) by -1.
    """
    UR = sun.represent(U, N, rep)
    last = geom.coords[:, 0] == geom.T - 1
    UR[last, 0] *= -1.0
    return UR


# --------------------------------------------------------------- hopping ----
def hopping(UR: np.ndarray, psi: np.ndarray, geom: Geometry, sign: int = 1,
            sites: np.ndarray | None = None) -> np.ndarray:
    """H psi(x) = sum_mu [(1 - s g_mu) U_mu(x) psi(x+mu) + (1 + s g_mu) U_mu(x-mu)^dag psi(x-mu)].

    ``sign`` s = +1 gives the hopping term of D, s = -1 that of D^dagger (the
    adjoint of x -> U_mu(x) psi(x+mu) is y -> U_mu(y-mu)^dagger psi(y-mu), and
    the gammas are Hermitian, so taking the adjoint swaps the projectors).
    Evaluated at ``sites`` (default: all); returns an array over those sites.
    Both hops of every direction are accumulated, so on L = 2 where x+mu and
    x-mu coincide both terms are counted.
    """
    if sites is None:
        sites = np.arange(geom.V)
    d = UR.shape[-1]
    out = np.zeros((len(sites), 4, d), dtype=complex)
    for mu in range(4):
        f = geom.fwd[mu][sites]
        b = geom.bwd[mu][sites]
        u_psi = np.einsum("xac,xsc->xsa", UR[sites, mu], psi[f])
        out += np.einsum("st,xta->xsa", I4 - sign * GAMMA[mu], u_psi)
        ud_psi = np.einsum("xca,xsc->xsa", UR[b, mu].conj(), psi[b])
        out += np.einsum("st,xta->xsa", I4 + sign * GAMMA[mu], ud_psi)
    return out


# ---------------------------------------------------------------- clover ----
def _dag(M):
    return np.conj(np.swapaxes(M, -1, -2))


def clover_leaves(UR: np.ndarray, geom: Geometry, mu: int, nu: int,
                  sites: np.ndarray) -> np.ndarray:
    """Q_mu_nu(x): sum of the four plaquettes at x in the (mu, nu) plane.

    Each leaf starts and ends at x and circles its plaquette in the same
    sense, the one that goes from +mu to +nu:
        U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
      + U_nu(x) U_mu(x+nu-mu)^+ U_nu(x-mu)^+ U_mu(x-mu)
      + U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu)
      + U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^+
    """
    x = sites
    fw, bw = geom.fwd, geom.bwd
    xpm, xpn, xmm, xmn = fw[mu][x], fw[nu][x], bw[mu][x], bw[nu][x]
    xmm_pn = fw[nu][xmm]
    xmm_mn = bw[nu][xmm]
    xmn_pm = fw[mu][xmn]
    q = UR[x, mu] @ UR[xpm, nu] @ _dag(UR[xpn, mu]) @ _dag(UR[x, nu])
    q = q + UR[x, nu] @ _dag(UR[xmm_pn, mu]) @ _dag(UR[xmm, nu]) @ UR[xmm, mu]
    q = q + _dag(UR[xmm, mu]) @ _dag(UR[xmm_mn, nu]) @ UR[xmm_mn, mu] @ UR[xmn, nu]
    q = q + _dag(UR[xmn, nu]) @ UR[xmn, mu] @ UR[xmn_pm, nu] @ _dag(UR[x, mu])
    return q


def field_strength(UR: np.ndarray, geom: Geometry, mu: int, nu: int,
                   sites: np.ndarray) -> np.ndarray:
    """Fhat_mu_nu(x) = (Q_mu_nu(x) - Q_mu_nu(x)^dagger) / 8 (anti-Hermitian)."""
    q = clover_leaves(UR, geom, mu, nu, sites)
    return (q - _dag(q)) / 8.0


def clover_matrix(UR: np.ndarray, geom: Geometry, m0: float, csw: float,
                  sites: np.ndarray | None = None, exponential: bool = False) -> np.ndarray:
    """A(x) = (4 + m0) + c_sw (i/4) sum_{mu != nu} sigma_mu_nu (x) Fhat_mu_nu(x).

    With ``exponential`` the exponentiated clover term the paper supports
    (Sec. 3.1, after Francis, Fritzsch, Luscher and Rago): with C(x) the
    clover term above, A(x) = (4 + m0) exp(C(x) / (4 + m0)), the matrix
    exponential of the full 4d x 4d matrix (scipy's expm).
    Returned as full [n_sites][4d][4d] matrices, index = spin * d + colour.
    """
    if sites is None:
        sites = np.arange(geom.V)
    d = UR.shape[-1]
    sites = np.asarray(sites)
    A = np.zeros((len(sites), 4 * d, 4 * d), dtype=complex)
    A += (4.0 + m0) * np.eye(4 * d)
    if csw != 0.0:
        for mu in range(4):
            for nu in range(4):
                if mu == nu:
                    continue
                F = field_strength(UR, geom, mu, nu, sites)
                A += csw * 0.25j * np.einsum("st,xab->xsatb", sigma(mu, nu), F).reshape(
                    len(sites), 4 * d, 4 * d)
    if exponential:
        import scipy.linalg
        c = 4.0 + m0
        C = A - c * np.eye(4 * d)
        A = np.array([c * scipy.linalg.expm(C[k] / c) for k in range(len(sites))])
    return A


# ------------------------------------------------------------ lazy links ---
class LazyRepresentedField:
    """U_R[V][4][d][d] with the time-boundary sign, evaluated only where indexed.

    ``link_fn(sites)`` returns the fundamental links U[len(sites)][4][N][N] of
    the given sites.  Indexing with ``[sites, mu]`` computes (and caches) U_R
    exactly as ``represented_field`` does, so a full-size lattice can be
    checked at sampled sites without materialising the whole field.
    """

    def __init__(self, link_fn, N: int, rep: str, geom: Geometry):
        self.link_fn, self.N, self.rep, self.geom = link_fn, N, rep, geom
        self.d = sun.rep_dim(N, rep)
        self.shape = (geom.V, 4, self.d, self.d)
        self._cache = {}

    def _site_links(self, sites):
        todo = np.unique(np.asarray([x for x in np.unique(sites) if x not in self._cache], dtype=np.int64))
        if len(todo):
            UR = sun.represent(self.link_fn(todo), self.N, self.rep)
            last = self.geom.coords[todo, 0] == self.geom.T - 1
            UR[last, 0] *= -1.0
            for k, x in enumerate(todo):
                self._cache[int(x)] = UR[k]
        return np.array([self._cache[int(x)] for x in np.asarray(sites).ravel()]).reshape(
            np.shape(sites) + (4, self.d, self.d))

    def __getitem__(self, key):
        sites, mu = key
        return self._site_links(np.asarray(sites))[..., mu, :, :]


# --------------------------------------------------------------- D and D^ ---
class WilsonOperator:
    """D_R on one gauge background.  ``A`` is None for c_sw = 0 (then A = 4+m0).

    With ``link_fn`` instead of ``U`` the represented field is evaluated lazily
    (``LazyRepresentedField``) and the clover matrix only at the sites asked for.
    """

    def __init__(self, U, N: int, rep: str, geom: Geometry, m0: float,
                 csw: float = 0.0, link_fn=None, exponential: bool = False):
        self.N, self.rep, self.geom, self.m0, self.csw = N, rep, geom, m0, csw
        self.exponential = exponential
        self.d = sun.rep_dim(N, rep)
        self.lazy = link_fn is not None
        if self.lazy:
            self.UR = LazyRepresentedField(link_fn, N, rep, geom)
            self.A = None
            self._A_cache = {}
        else:
            self.UR = represented_field(U, N, rep, geom)
            self.A = clover_matrix(self.UR, geom, m0, csw, exponential=exponential) if csw != 0.0 else None

    # diagonal part --------------------------------------------------------
    def apply_A(self, psi, sites, dagger=False, inverse=False):
        """A(x) psi(x) (or its adjoint / inverse) at ``sites``; psi is over those sites."""
        d = self.d
        if self.A is None and not (self.lazy and self.csw != 0.0):
            c = 4.0 + self.m0
            return psi / c if inverse else psi * c
        if self.lazy:
            need = [int(x) for x in sites if int(x) not in self._A_cache]
            if need:
                An = clover_matrix(self.UR, self.geom, self.m0, self.csw, np.array(need),
                                   exponential=self.exponential)
                for k, x in enumerate(need):
                    self._A_cache[x] = An[k]
            A = np.array([self._A_cache[int(x)] for x in sites])
        else:
            A = self.A[sites]
        if dagger:
            A = _dag(A)
        v = psi.reshape(len(sites), 4 * d)
        if inverse:
            w = np.linalg.solve(A, v[..., None])[..., 0]
        else:
            w = np.einsum("xij,xj->xi", A, v)
        return w.reshape(len(sites), 4, d)

    # full lattice ---------------------------------------------------------
    def apply(self, psi: np.ndarray, dagger: bool = False) -> np.ndarray:
        """D psi (or D^dagger psi) on the full lattice."""
        sites = np.arange(self.geom.V)
        s = -1 if dagger else 1
        return self.apply_A(psi, sites, dagger=dagger) - 0.5 * hopping(self.UR, psi, self.geom, s)

    # even-odd Schur complement --------------------------------------------
    def apply_schur(self, psi: np.ndarray, parity: int, dagger: bool = False,
                    sites: np.ndarray | None = None) -> np.ndarray:
        """Dhat_p psi = A_pp psi_p - D_pq A_qq^{-1} D_qp psi_p (or its adjoint).

        ``psi`` is a full-lattice array of which only parity-p sites are read.
        Returns a full-lattice array that is nonzero only on the parity-p sites
        listed in ``sites`` (default: all parity-p sites).  With ``sites`` a
        subset, only the neighbourhoods needed for those outputs are computed.
        The adjoint of the Schur complement is the Schur complement of D^dagger,
        i.e. the same formula with the projector signs swapped and A^dagger.
        """
        g = self.geom
        s = -1 if dagger else 1
        q = 1 - parity
        if sites is None:
            sites = g.sites_of_parity(parity)
        sites = np.asarray(sites)
        assert np.all(g.parity[sites] == parity)
        # the opposite-parity sites that the outputs at `sites` depend on; the
        # hops from them read psi only on their (parity-p) neighbours, so psi's
        # values on parity q never enter
        nb = np.unique(np.concatenate([g.fwd[:, sites].ravel(), g.bwd[:, sites].ravel()]))
        assert np.all(g.parity[nb] == q)
        t = np.zeros_like(psi)
        t[nb] = -0.5 * hopping(self.UR, psi, g, s, nb)            # D_qp psi_p
        t[nb] = self.apply_A(t[nb], nb, dagger=dagger, inverse=True)  # A_qq^{-1}
        out = np.zeros_like(psi)
        u = -0.5 * hopping(self.UR, t, g, s, sites)                 # D_pq t
        out[sites] = self.apply_A(psi[sites], sites, dagger=dagger) - u
        return out


# ------------------------------------------------------- FP16 per-site code --
def encode_fp16(v: np.ndarray):
    """FP16 code of a per-site real vector v[..., n] with one FP32 scale per site.

    v is rounded to FP32, scale = max |v| over the site (FP32, exact), and each
    value is stored as FP16 of the correctly rounded FP32 quotient v / scale
    (round to nearest even both times).  A site that is all zero gets scale 0
    and zero codes.  Returns (codes float16[..., n], scale float32[...]).
    """
    vf = np.asarray(v, dtype=np.float64).astype(np.float32)
    scale = np.max(np.abs(vf), axis=-1)
    safe = np.where(scale > 0, scale, np.float32(1.0)).astype(np.float32)
    q = (vf / safe[..., None]).astype(np.float32)
    h = q.astype(np.float16)
    h = np.where(scale[..., None] > 0, h, np.float16(0.0))
    return h, scale.astype(np.float32)


def decode_fp16(h: np.ndarray, scale: np.ndarray) -> np.ndarray:
    """v = code * scale, evaluated exactly in FP64."""
    return h.astype(np.float64) * scale.astype(np.float64)[..., None]


def spinor_site_reals(psi: np.ndarray) -> np.ndarray:
    """psi[..., 4, d] complex -> [..., 8d] reals (re, im interleaved), for the FP16 code."""
    sh = psi.shape[:-2]
    return np.stack([psi.real, psi.imag], axis=-1).reshape(*sh, -1)


def spinor_from_site_reals(r: np.ndarray, d: int) -> np.ndarray:
    sh = r.shape[:-1]
    r = r.reshape(*sh, 4, d, 2)
    return r[..., 0] + 1j * r[..., 1]
