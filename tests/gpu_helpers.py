"""Helpers shared by the GPU parity tests: build a lattice through the C ABI
and the matching oracle operator from the same seeded random draws."""
import numpy as np

from oracle import sun
from oracle.dirac import Geometry, WilsonOperator
from paper_2405_19294_gb300 import inputs

TOL = {0: 1e-13, 1: 2e-6, 2: 5e-3}   # relative L2 parity per precision (FP64, FP32, FP16)


def gpu_lattice(hr, T, L, N, rep, eps, csw, seed=0, reunitarise=True):
    """Lattice with links generated on the GPU from the seeded algebra draws."""
    import torch
    lat = hr.Lattice(T, L, N, rep)
    a = inputs.algebra_coefficients(seed, T, L, N)
    a_d = torch.from_numpy(a).cuda()
    U = torch.empty((lat.V, 4, N, N, 2), dtype=torch.float64, device="cuda")
    lat.links_from_algebra(U, a_d, eps, reunitarise)
    lat.represent_links(U, reunitarise, csw)
    return lat, U


def oracle_links(T, L, N, eps, seed=0, reunitarise=True):
    a = inputs.algebra_coefficients(seed, T, L, N)
    U = sun.links_from_algebra(a, eps, N)
    return sun.reunitarise(U) if reunitarise else U


def oracle_operator(T, L, N, rep, eps, m0, csw, seed=0, exponential=False):
    g = Geometry(T, L)
    return WilsonOperator(oracle_links(T, L, N, eps, seed), N, rep, g, m0, csw,
                          exponential=exponential)


def to_complex(t):
    """torch float64 [..., 2] (device or host) -> numpy complex128 [...]."""
    a = t.detach().cpu().numpy()
    return a[..., 0] + 1j * a[..., 1]


def from_complex(z):
    import torch
    z = np.ascontiguousarray(z)
    return torch.from_numpy(np.stack([z.real, z.imag], axis=-1)).cuda()


def rel_err(a, b, mask=None):
    if mask is not None:
        a, b = a[mask], b[mask]
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())
