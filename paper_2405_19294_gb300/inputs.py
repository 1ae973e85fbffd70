"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module only draws random numbers and shapes.  It holds none of the
method's arithmetic: the Lie-algebra coefficients it returns are turned into
SU(N) links by the library (``hr_links_from_algebra``) and, independently, by
the oracle.

Conventions (the paper gives none; the choices below are the ones both sides
read):

* lattice sites are lexicographic, ``idx = ((t*L + z)*L + y)*L + x``;
  direction 0 is time (extent T), 1..3 are x, y, z (extent L);
* gauge input: ``a[site][mu][k]`` with ``k = 0..N*N-2``, i.i.d. N(0,1), drawn
  from one PCG64 stream in exactly that order;
* spinors: ``psi[rhs][site][spin][colour]`` complex, real and imaginary
  parts i.i.d. N(0,1) (real part drawn first for each component); right-hand
  side r comes from its own stream PCG64([seed, r]).
"""
from __future__ import annotations

import numpy as np

REPS = ("fund", "adj", "sym", "asym")


def rep_dim(N: int, rep: str) -> int:
    """Dimension of the representation (fund N, adj N^2-1, sym N(N+1)/2, asym N(N-1)/2)."""
    return {"fund": N, "adj": N * N - 1, "sym": N * (N + 1) // 2, "asym": N * (N - 1) // 2}[rep]


def algebra_coefficients(seed: int, T: int, L: int, N: int) -> np.ndarray:
    """Gaussian coefficients a[V][4][N^2-1] (float64) for ``U = exp(i eps sum_k a_k T_k)``."""
    V = T * L * L * L
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((V, 4, N * N - 1))


def gaussian_spinor_rhs(seed: int, T: int, L: int, d: int, r: int) -> np.ndarray:
    """Right-hand side r of ``gaussian_spinor``: psi[V][4][d] (complex128)."""
    V = T * L * L * L
    rng = np.random.Generator(np.random.PCG64([seed, r]))
    re_im = rng.standard_normal((V, 4, d, 2))
    return re_im[..., 0] + 1j * re_im[..., 1]


def gaussian_spinor(seed: int, T: int, L: int, d: int, nrhs: int = 1) -> np.ndarray:
    """Complex Gaussian spinor fields psi[nrhs][V][4][d] (complex128)."""
    return np.stack([gaussian_spinor_rhs(seed, T, L, d, r) for r in range(nrhs)])


def gauge_transform_coefficients(seed: int, T: int, L: int, N: int) -> np.ndarray:
    """Gaussian coefficients g[V][N^2-1] for a random local gauge transformation."""
    V = T * L * L * L
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((V, N * N - 1))


def batch_shapes(seed: int, count: int = 64):
    """Shapes of the many-small-lattices workload: (T, L, N, rep) per lattice.

    L uniform in {8,10,12,14,16}; T uniform in {L, 2L} restricted to T <= 32;
    N uniform in {2..6}; rep uniform in {fund, adj, sym, asym}, redrawing the
    one-dimensional SU(2) antisymmetric case.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    while len(out) < count:
        L = int(rng.choice([8, 10, 12, 14, 16]))
        Ts = [t for t in (L, 2 * L) if t <= 32]
        T = int(rng.choice(Ts))
        N = int(rng.integers(2, 7))
        rep = REPS[int(rng.integers(0, 4))]
        if N == 2 and rep == "asym":
            continue
        out.append((T, L, N, rep))
    return out
