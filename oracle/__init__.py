"""FP64 CPU oracle for the Wilson(-clover) Dirac operator in representation R of SU(N).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library under
``paper_2405_19294_gb300/`` never imports it and shares no code with it; the
two meet only in the seeded random draws of ``paper_2405_19294_gb300.inputs``,
which the callers pass in as plain arrays.

The paper (Sec. 3.1 "Wilson-Dirac Operator", Sec. 3.3 "Inverters") names the
operators -- Wilson-Dirac in a general representation of SU(N_c), even-odd
preconditioning, clover improvement, conjugate gradient -- but prints no
formula.  Every function here therefore writes out the standard lattice
definition, with the conventions fixed once:

* ``sun``      generators, links from the algebra, reunitarisation, the maps
               U -> U_R for the fundamental, adjoint, 2-index symmetric and
               2-index antisymmetric representations;
* ``dirac``    gamma matrices, the Wilson operator with antiperiodic time,
               the Sheikholeslami-Wohlert clover term, the even-odd Schur
               complement, FP16 per-site encoding;
* ``solvers``  textbook conjugate gradient on the normal equations.

Everything is plain numpy in float64/complex128: no blocking, no fusion, no
reordering beyond the definitions.  The pins that tie it to mathematics
rather than to itself live in ``tests/test_oracle_*.py``.
"""
from . import sun, dirac, solvers  # noqa: F401
