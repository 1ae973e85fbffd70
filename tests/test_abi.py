"""The C-ABI library builds, loads without a GPU and exports every function
that include/hr.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def _declared():
    names = set()
    for h in HEADERS:
        txt = open(h).read()
        names |= set(re.findall(r"^\s*(?:int|const char \*)\s*(hr_\w+)\s*\(", txt, re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("hr_lattice_create", "hr_represent_links", "hr_dphi", "hr_cg_solve"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2405_19294_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    from paper_2405_19294_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.hr_status_string.restype = ctypes.c_char_p
    assert lib.hr_status_string(0) == b"ok"
    assert b"argument" in lib.hr_status_string(-1)


def test_create_rejects_bad_shapes_before_touching_the_device():
    from paper_2405_19294_gb300 import build
    lib = ctypes.CDLL(build.build())
    h = ctypes.c_void_p()
    for args in [(3, 4, 3, 0), (4, 3, 3, 0), (4, 4, 1, 0), (4, 4, 13, 0), (4, 4, 7, 1), (4, 4, 2, 3), (4, 4, 3, 9)]:
        assert lib.hr_lattice_create(*args, ctypes.byref(h)) == -1


def test_shape_code_round_trip():
    """The binding's launch-shape code (rows, mrhs, regs, G, block packed in
    decimal fields, as hr.h documents) decodes back to the same tuple."""
    from paper_2405_19294_gb300 import hr
    for shape in [(0, 32, 1, 0, 0), (0, 256, 0, 0, 0), (16, 128, 0, 0, 0), (0, 0, 0, 16, 0), (0, 0, 0, 8, 0),
                  (0, 576, 0, 0, 2), (0, 64, 2, 0, 0), (4, 128, 0, 0, 0), (0, 96, 0, 0, 5)]:
        code = hr._shape_code(shape)
        assert hr.Lattice._decode(code) == shape
    assert hr._shape_code((0, 32, 1)) == hr._shape_code((0, 32, 1, 0, 0)) == 100032
