"""Shared pytest set-up: the ``gpu`` marker and the repository root on sys.path."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libhr")


@pytest.fixture(scope="session")
def hr():
    """The C-ABI binding; a GPU test that gets here without the library fails loudly."""
    from paper_2405_19294_gb300 import hr as _hr
    return _hr
