"""The oracle against its committed regression fixture (tests/golden/).

The fixture holds checksums of the Wilson(-clover) operator of Sec. 3.1 (even-odd
Schur complement and full D) for eight representation / clover cases on a
4x4^3 lattice, written by tests/golden/make_golden.py from the oracle alone.
The paper prints no worked example, so these are not the paper's numbers: the
test guards the oracle against unintended changes of its arithmetic, while the
physics pins (test_oracle_dirac.py) fix what the values must be.
"""
import importlib.util
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "oracle_dhat_4x4.txt")


def _maker():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _records():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            N, rep, csw, expo, name, value = line.split()
            out.setdefault((int(N), rep, float(csw), bool(int(expo))), []).append((name, float(value)))
    return out


RECORDS = _records()


def test_fixture_covers_every_case():
    mk = _maker()
    assert sorted(RECORDS) == sorted(mk.CASES)
    assert all(len(v) == 12 for v in RECORDS.values())


@pytest.mark.parametrize("case", sorted(RECORDS), ids=lambda c: "%d%s_csw%g%s" % (c[0], c[1], c[2], "_exp" if c[3] else ""))
def test_oracle_matches_fixture(case):
    got = _maker().case_values(*case)
    want = RECORDS[case]
    assert [n for n, _ in got] == [n for n, _ in want]
    for (name, g), (_, w) in zip(got, want):
        assert abs(g - w) <= 1e-10 * max(1.0, abs(w)), (case, name, g, w)
