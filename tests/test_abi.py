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


def test_binding_structs_match_the_header_layout(tmp_path):
    """hr.py's ctypes mirrors of hr_info, hr_cg_params and hr_cg_stats have the size and
    field offsets that a C compiler gives the structs of include/hr.h (a field added on
    one side only would shift every later field)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    from paper_2405_19294_gb300 import hr
    structs = {"hr_info": hr.hr_info, "hr_cg_params": hr.hr_cg_params, "hr_cg_stats": hr.hr_cg_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hr.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def test_binding_enums_match_the_header():
    """The precision, parity and representation codes of hr.py are the header's."""
    from paper_2405_19294_gb300 import hr
    txt = open(os.path.join(ROOT, "include", "hr.h")).read()

    def enum(tname):
        body = re.search(r"typedef enum \{([^}]*)\}\s*" + tname + ";", txt).group(1)
        return {k: int(v) for k, v in re.findall(r"(HR_\w+)\s*=\s*(-?\d+)", body)}

    prec = enum("hr_prec")
    assert prec == {"HR_F64": hr.F64, "HR_F32": hr.F32, "HR_F16": hr.F16, "HR_FF": hr.FF}
    assert sorted(hr.PREC.values()) == sorted(prec.values())
    par = enum("hr_parity")
    assert par == {"HR_EVEN": hr.EVEN, "HR_ODD": hr.ODD, "HR_FULL": hr.FULL}
    rep = enum("hr_rep")
    assert sorted(rep.values()) == sorted(hr.REP.values())
