"""GB300-native Wilson(-clover) Dirac operator in higher representations of SU(N).

The compute path lives in ``libhr.so`` (CUDA, sm_103a), reached through the C
ABI declared in ``include/hr.h``; ``paper_2405_19294_gb300.hr`` is its thin
ctypes binding.  ``paper_2405_19294_gb300.inputs`` draws the seeded synthetic
inputs.  Importing the package itself loads nothing: import ``hr`` to load
the library (it raises if the library has not been built).
"""
