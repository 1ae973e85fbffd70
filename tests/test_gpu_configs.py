"""Full-size workloads, checked on the GPU against the oracle at sampled sites.

The oracle evaluates the represented links and the clover term lazily, only
in the neighbourhoods of the sampled sites, so the full lattices
(32^3 x 64 and 24^3 x 48) stay affordable.  Sampled sites always include the
lattice corners and the time boundary (where the antiperiodic sign sits).

* SU(3) fund, 32^3 x 64, eps 1.0, m0 -0.4: Dhat in FP64 and FP32;
  CG plain FP64, mixed FP32, mixed FP16 to 1e-10
* SU(2) adj and SU(4) asym, 24^3 x 48, m0 -0.3: Dhat in FP32 and FP16;
  mixed FP16 / FP32 CG to 1e-10
* SU(3) sym with clover csw 1.0, 32^3 x 64, m0 -0.35, 12 rhs: Dhat on all
  right-hand sides at once in FP32; mixed FP32 CG on all 12 to 1e-10
"""
import numpy as np
import pytest

from gpu_helpers import TOL, from_complex, to_complex
from oracle import sun
from oracle.dirac import Geometry, WilsonOperator
from paper_2405_19294_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

WORKLOADS = {
    "su3_fund_32c64": dict(N=3, rep="fund", T=64, L=32, eps=1.0, m0=-0.4, csw=0.0, nrhs=1, precs=(0, 1, 2), inner=(0, 1, 2)),
    "su2_adj_24c48": dict(N=2, rep="adj", T=48, L=24, eps=1.0, m0=-0.3, csw=0.0, nrhs=1, precs=(1, 2), inner=(2, 1)),
    "su4_asym_24c48": dict(N=4, rep="asym", T=48, L=24, eps=1.0, m0=-0.3, csw=0.0, nrhs=1, precs=(1, 2), inner=(2, 1)),
    "su3_sym_clover_12rhs_32c64": dict(N=3, rep="sym", T=64, L=32, eps=1.0, m0=-0.35, csw=1.0, nrhs=12, precs=(0, 1, 2), inner=(1,)),
}

_cache = {}


def _setup(hr, name):
    if name in _cache:
        return _cache[name]
    c = WORKLOADS[name]
    T, L, N, rep = c["T"], c["L"], c["N"], c["rep"]
    lat = hr.Lattice(T, L, N, rep)
    a = inputs.algebra_coefficients(0, T, L, N)
    a_d = torch.from_numpy(a).cuda()
    U = torch.empty((lat.V, 4, N, N, 2), dtype=torch.float64, device="cuda")
    lat.links_from_algebra(U, a_d, c["eps"], True)
    lat.represent_links(U, True, c["csw"])
    del a_d, U
    g = Geometry(T, L)
    op = WilsonOperator(None, N, rep, g, c["m0"], c["csw"],
                        link_fn=lambda s: sun.reunitarise(sun.links_from_algebra(a[s], c["eps"], N)))
    # samples: corners / time boundary plus random even sites
    rng = np.random.default_rng(123)
    even = g.sites_of_parity(0)
    picks = [g.lex(np.array([t, x, y, z])) for (t, x, y, z) in
             [(0, 0, 0, 0), (T - 1, L - 1, 0, 0), (T - 1, 0, L - 1, 0), (0, L - 2, L - 1, L - 1),
              (T - 2, 1, 1, 0), (T // 2, L - 1, L - 1, 0)]]
    picks = [int(p) for p in picks if g.parity[p] == 0]
    sites = np.unique(np.concatenate([np.array(picks, dtype=np.int64), rng.choice(even, 10, replace=False)]))
    _cache[name] = (lat, op, g, sites)
    return _cache[name]


def _load_sources(lat, c, parity, prec):
    """Pack the Gaussian sources rhs by rhs (host memory: one rhs at a time)."""
    nrhs = c["nrhs"]
    f = lat.new_field(parity, prec, nrhs)
    fb = lat.field_bytes(parity, prec, 1)
    for r in range(nrhs):
        psi = inputs.gaussian_spinor_rhs(1, c["T"], c["L"], lat.d, r)
        lat.pack(f[r * fb:(r + 1) * fb], from_complex(psi), parity, prec, 1)
    return f


def _unpack_rhs(lat, f, parity, prec, r):
    fb = lat.field_bytes(parity, prec, 1)
    out = torch.zeros((1, lat.V, 4, lat.d, 2), dtype=torch.float64, device="cuda")
    lat.unpack(out, f[r * fb:(r + 1) * fb], parity, prec, 1)
    return to_complex(out)[0]


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_full_size_dhat_sampled(hr, name):
    c = WORKLOADS[name]
    lat, op, g, sites = _setup(hr, name)
    check_rhs = [0] if c["nrhs"] == 1 else [0, c["nrhs"] - 1]
    for prec in c["precs"]:
        fin = _load_sources(lat, c, 0, prec)
        fout = lat.new_field(0, prec, c["nrhs"])
        lat.dphi(fout, fin, 0, c["m0"], c["csw"], prec, c["nrhs"])
        lat.synchronize()
        for r in check_rhs:
            psi = inputs.gaussian_spinor_rhs(1, c["T"], c["L"], lat.d, r)
            got = _unpack_rhs(lat, fout, 0, prec, r)
            ref = op.apply_schur(psi, 0, sites=sites)
            err = np.linalg.norm(got[sites] - ref[sites]) / np.linalg.norm(ref[sites])
            assert err < TOL[prec], (name, prec, r, err)
        del fin, fout


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_full_size_cg_to_1e10(hr, name):
    c = WORKLOADS[name]
    lat, op, g, sites = _setup(hr, name)
    nrhs = c["nrhs"]
    fb_ = _load_sources(lat, c, 0, 0)
    for inner in c["inner"]:
        fx = lat.new_field(0, 0, nrhs)
        st = lat.cg_solve(fx, fb_, 0, c["m0"], c["csw"], 1e-10, inner_prec=inner, nrhs=nrhs, check_every=10)
        assert st["true_residual"] <= 1e-10, (name, inner, st)
        # oracle residual at the sampled sites of rhs 0: b - Dhat^+ Dhat x
        x = _unpack_rhs(lat, fx, 0, 0, 0)
        b = inputs.gaussian_spinor_rhs(1, c["T"], c["L"], lat.d, 0)
        s2 = np.unique(np.concatenate([sites] + [g.fwd[m][g.fwd[n][sites]] for m in range(4) for n in range(4)]
                                      + [g.bwd[m][g.bwd[n][sites]] for m in range(4) for n in range(4)]
                                      + [g.fwd[m][g.bwd[n][sites]] for m in range(4) for n in range(4)]))
        s2 = s2[g.parity[s2] == 0]
        y = op.apply_schur(x, 0, sites=s2)
        Mx = op.apply_schur(y, 0, dagger=True, sites=sites)
        res = np.linalg.norm(b[sites] - Mx[sites]) / np.linalg.norm(b[sites])
        assert res < 1e-9, (name, inner, res)
        del fx


@pytest.mark.parametrize("inner", [0, 1, 2])
def test_cg_global_oracle_residual_16c32(hr, inner):
    """The SU(3) fund operator (eps 1.0, m0 -0.4) on 16^3 x 32 (V/2 = 65536 sites: hundreds of blocks per
    launch): the oracle's residual |b - Dhat^+ Dhat x| / |b| over the whole lattice,
    not only at sampled sites, meets the 1e-10 target the library reports."""
    from gpu_helpers import gpu_lattice, oracle_operator
    T, L, N, rep, m0 = 32, 16, 3, "fund", -0.4
    lat, _ = gpu_lattice(hr, T, L, N, rep, 1.0, 0.0)
    op = oracle_operator(T, L, N, rep, 1.0, m0, 0.0)
    ev = op.geom.parity == 0
    b = np.where(ev[:, None, None], inputs.gaussian_spinor(21, T, L, lat.d)[0], 0)
    fb = lat.new_field(0, 0)
    lat.pack(fb, from_complex(b[None]), 0, 0)
    fx = lat.new_field(0, 0)
    st = lat.cg_solve(fx, fb, 0, m0, 0.0, 1e-10, inner_prec=inner)
    assert st["true_residual"] <= 1e-10, st
    out = torch.zeros((1, lat.V, 4, lat.d, 2), dtype=torch.float64, device="cuda")
    lat.unpack(out, fx, 0, 0)
    lat.synchronize()
    x = to_complex(out)[0]
    r = b - op.apply_schur(op.apply_schur(x, 0), 0, dagger=True)
    # the library stops on its own FP64 true residual; the oracle's evaluation differs by rounding
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.05e-10, st


@pytest.mark.parametrize("inner", [1, 2])
def test_multi_rhs_cg_global_oracle_residual(hr, inner):
    """The SU(3) sextet operator with clover (csw = 1, m0 -0.35) on 8^3 x 16 with 12 right-hand
    sides in one solve (FP32 or FP16 inner operator, whichever multi-rhs kernel the
    autotuner picks), checked rhs by rhs against the oracle over the whole lattice."""
    from gpu_helpers import gpu_lattice, oracle_operator
    T, L, N, rep, m0, csw, nr = 16, 8, 3, "sym", -0.35, 1.0, 12
    lat, _ = gpu_lattice(hr, T, L, N, rep, 1.0, csw)
    op = oracle_operator(T, L, N, rep, 1.0, m0, csw)
    ev = op.geom.parity == 0
    b = inputs.gaussian_spinor(22, T, L, lat.d, nr)
    b = np.where(ev[None, :, None, None], b, 0)
    fb = lat.new_field(0, 0, nr)
    lat.pack(fb, from_complex(b), 0, 0, nr)
    fx = lat.new_field(0, 0, nr)
    st = lat.cg_solve(fx, fb, 0, m0, csw, 1e-10, inner_prec=inner, nrhs=nr)
    assert st["true_residual"] <= 1e-10, st
    out = torch.zeros((nr, lat.V, 4, lat.d, 2), dtype=torch.float64, device="cuda")
    lat.unpack(out, fx, 0, 0, nr)
    lat.synchronize()
    x = to_complex(out)
    for k in range(nr):
        r = b[k] - op.apply_schur(op.apply_schur(x[k], 0), 0, dagger=True)
        assert np.linalg.norm(r) / np.linalg.norm(b[k]) <= 1.05e-10, (k, st)
