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
    Um, Un = UR[:, mu], UR[:, nu]
    q = Um[x] @ Un[xpm] @ _dag(Um[xpn]) @ _dag(Un[x])
    q = q + Un[x] @ _dag(Um[xmm_pn]) @ _dag(Un[xmm]) @ Um[xmm]
    q = q + _dag(Um[xmm]) @ _dag(Un[xmm_mn]) @ Um[xmm_mn] @ Un[xmn]
    q = q + _dag(Un[xmn]) @ Um[xmn] @ Un[xmn_pm] @ _dag(Um[x])
    return q


def field_strength(UR: np.ndarray, geom: Geometry, mu: int, nu: int,
                   sites: np.ndarray) -> np.ndarray:
    """Fhat_mu_nu(x) = (Q_mu_nu(x) - Q_mu_nu(x)^dagger) / 8 (anti-Hermitian)."""
    q = clover_leaves(UR, geom, mu, nu, sites)
    return (q - _dag(q)) / 8.0


def clover_matrix(UR: np.ndarray, geom: Geometry, m0: float, csw: float,
                  sites: np.ndarray | None = None) -> np.ndarray:
    """A(x) = (4 + m0) + c_sw (i/4) sum_{mu != nu} sigma_mu_nu (x) Fhat_mu_nu(x).

    Returned as full [n_sites][4d][4d] matrices, index = spin * d + colour.
    """
    if sites is None:
        sites = np.arange(geom.V)
    d = UR.shape[-1]
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
    return A


# --------------------------------------------------------------- D and D^ ---
class WilsonOperator:
    """D_R on one gauge background.  ``A`` is None for c_sw = 0 (then A = 4+m0)."""

    def __init__(self, U: np.ndarray, N: int, rep: str, geom: Geometry, m0: float,
                 csw: float = 0.0):
        self.N, self.rep, self.geom, self.m0, self.csw = N, rep, geom, m0, csw
        self.d = sun.rep_dim(N, rep)
        self.UR = represented_field(U, N, rep, geom)
        self.A = clover_matrix(self.UR, geom, m0, csw) if csw != 0.0 else None

    # diagonal part --------------------------------------------------------
    def apply_A(self, psi, sites, dagger=False, inverse=False):
        """A(x) psi(x) (or its adjoint / inverse) at ``sites``; psi is over those sites."""
        d = self.d
        if self.A is None:
            c = 4.0 + self.m0
            return psi / c if inverse else psi * c
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
        psi_p = np.where((g.parity == parity)[:, None, None], psi, 0.0)
        if sites is None:
            sites = g.sites_of_parity(parity)
        # the opposite-parity sites that the outputs at `sites` depend on
        nb = np.unique(np.concatenate([g.fwd[:, sites].ravel(), g.bwd[:, sites].ravel()]))
        assert np.all(g.parity[nb] == q)
        t = np.zeros_like(psi)
        t[nb] = -0.5 * hopping(self.UR, psi_p, g, s, nb)          # D_qp psi_p
        t[nb] = self.apply_A(t[nb], nb, dagger=dagger, inverse=True)  # A_qq^{-1}
        out = np.zeros_like(psi)
        u = -0.5 * hopping(self.UR, t, g, s, sites)                 # D_pq t
        out[sites] = self.apply_A(psi_p[sites], sites, dagger=dagger) - u
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
