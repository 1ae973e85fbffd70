"""Write oracle_dhat_4x4.txt: checksums of the oracle's Wilson(-clover) operator.

The paper prints no worked example of the operator (Sec. 3.1 names it and
cites its definitions), so this fixture is not a value from the paper.  It is
a regression record of the oracle itself, written by this script from
``oracle/`` and the seeded input generators only.  The CPU test
``tests/test_oracle_golden.py`` recomputes every line; a change of the
oracle's arithmetic that moves a value must be justified by the passage (or
the reading of it) that requires it, and this script re-run.

Run from the repository root:  python tests/golden/make_golden.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import sun  # noqa: E402
from oracle.dirac import Geometry, WilsonOperator  # noqa: E402
from paper_2405_19294_gb300 import inputs  # noqa: E402

T, L, EPS, M0 = 4, 4, 1.0, -0.3
LINK_SEED, SOURCE_SEED = 0, 1
# (N, representation, c_sw, exponentiated clover)
CASES = [(2, "fund", 0.0, False), (3, "fund", 0.0, False), (2, "adj", 0.0, False), (3, "sym", 0.0, False),
         (4, "asym", 0.0, False), (3, "adj", 0.0, False), (3, "fund", 1.0, False), (2, "adj", 1.0, True)]
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_dhat_4x4.txt")


def case_values(N: int, rep: str, csw: float, expo: bool) -> list[tuple[str, float]]:
    """The recorded quantities of one case, in a fixed order."""
    a = inputs.algebra_coefficients(LINK_SEED, T, L, N)
    U = sun.reunitarise(sun.links_from_algebra(a, EPS, N))
    geom = Geometry(T, L)
    op = WilsonOperator(U, N, rep, geom, M0, csw, exponential=expo)
    psi = inputs.gaussian_spinor(SOURCE_SEED, T, L, op.d)[0]
    even = geom.parity == 0
    psi_e = np.where(even[:, None, None], psi, 0)
    y = op.apply_schur(psi_e, 0)
    z = op.apply(psi)
    ip = np.vdot(psi_e.ravel(), y.ravel())
    x0 = int(np.flatnonzero(even)[0])
    vals = [("dhat_even_norm2", float(np.vdot(y[even].ravel(), y[even].ravel()).real)),
            ("psi_dhat_psi_re", float(ip.real)), ("psi_dhat_psi_im", float(ip.imag)),
            ("d_full_norm2", float(np.vdot(z.ravel(), z.ravel()).real))]
    for s in range(4):
        vals.append((f"dhat_x{x0}_s{s}_c0_re", float(y[x0, s, 0].real)))
        vals.append((f"dhat_x{x0}_s{s}_c0_im", float(y[x0, s, 0].imag)))
    return vals


def main() -> None:
    lines = ["# Oracle regression fixture (see make_golden.py): Wilson(-clover) operator of Sec. 3.1,",
             "# even-odd Schur complement Dhat_even (Sec. 3.1, even-odd preconditioning) and full D,",
             f"# on {T}x{L}^3, links exp(i eps sum a_k T_k) eps={EPS} reunitarised (seed {LINK_SEED}),",
             f"# Gaussian source (seed {SOURCE_SEED}), m0={M0}.  Columns: N rep csw expo quantity value.",
             "# Not a value printed by the paper, which gives no worked example."]
    for N, rep, csw, expo in CASES:
        for name, v in case_values(N, rep, csw, expo):
            lines.append(f"{N} {rep} {csw} {int(expo)} {name} {v!r}")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(OUT, len(lines) - 5, "values")


if __name__ == "__main__":
    main()
