"""hr_norm2_static: the norm reduction for callers that cannot allocate.

Some callers cannot call cudaMalloc/cudaFree: code whose device memory all
comes from a framework's pool allocator, code under a fixed memory budget,
real-time callers that forbid allocation after start-up.  hr_norm2_static
keeps its reduction scratch in a fixed device array inside the library
instead of allocating it.  This test calls it through the C ABI twice in a
row and checks both results against hr_norm2 (the entry point that allocates
its scratch) within the FP64 parity tolerance, and against a NumPy sum over the
unpacked field, which shares no code with either reduction (to 1e-13 for FP64
fields, 1e-6 for FP32 / FP16 fields, whose per-site squares are FP32).

The file name makes pytest collect it last, so a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from gpu_helpers import from_complex, gpu_lattice, to_complex
from oracle.dirac import Geometry
from paper_2405_19294_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("parity,prec,nrhs", [(0, 0, 1), (2, 1, 3), (1, 2, 16)])
def test_norm2_static_matches_allocating_entry_point(hr, parity, prec, nrhs):
    T, L, N, rep = 6, 6, 3, "sym"
    lat, _ = gpu_lattice(hr, T, L, N, rep, 1.0, 0.0)
    psi = inputs.gaussian_spinor(11, T, L, lat.d, nrhs)
    f = lat.new_field(parity, prec, nrhs)
    lat.pack(f, from_complex(psi), parity, prec, nrhs)
    ref = np.array(lat.norm2(f, parity, prec, nrhs))
    # the stored field read back to FP64 on the host, summed by NumPy
    back = torch.zeros((nrhs, lat.V, 4, lat.d, 2), dtype=torch.float64, device="cuda")
    lat.unpack(back, f, parity, prec, nrhs)
    lat.synchronize()
    g = Geometry(T, L)
    mask = np.ones(g.V, bool) if parity == 2 else g.parity == parity
    host = np.array([np.sum(np.abs(to_complex(back)[r, mask]) ** 2) for r in range(nrhs)])
    lib = hr.lib_handle()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        out = torch.full((nrhs,), -1.0, dtype=torch.float64, device="cuda")
        rc = lib.hr_norm2_static(ctypes.c_void_p(f.data_ptr()), lat.Vh, lat.d, parity, prec, nrhs,
                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.hr_status_string(rc)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-13 * ref), (got, ref)
        # FP32 / FP16 fields: each site's |x|^2 is formed in FP32 before the FP64 sum
        assert np.all(np.abs(got - host) <= (1e-13 if prec == 0 else 1e-6) * host), (got, host)


def test_norm2_static_rejects_too_many_rhs(hr):
    lib = hr.lib_handle()
    out = torch.zeros(17, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    rc = lib.hr_norm2_static(ctypes.c_void_p(dummy.data_ptr()), 8, 3, 0, 1, 17,
                             ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -1
