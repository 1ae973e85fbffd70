"""Many lattices at once: the batched operator (one persistent launch per
representation class and hopping stage) and the batched CG, against the
oracle and against the single-lattice entry points."""
import numpy as np
import pytest

from gpu_helpers import TOL, from_complex, gpu_lattice, oracle_operator, rel_err, to_complex
from oracle import sun
from oracle.dirac import Geometry, WilsonOperator
from paper_2405_19294_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# mixed shapes, N and representations; two lattices share a class (d=3 complex)
SMALL_BATCH = [(4, 4, 3, "fund"), (6, 4, 2, "adj"), (4, 6, 3, "asym"), (8, 4, 4, "sym"), (4, 4, 6, "adj"),
               (6, 6, 2, "fund"), (4, 2, 5, "sym")]


def _tol(prec):
    return TOL[0] if prec == 3 else TOL[prec]  # 3: float-float, held to the FP64 tolerance


def _fields(lat, psi, prec):
    f = lat.new_field(0, prec)
    lat.pack(f, from_complex(psi), 0, prec)
    return f


def _unpack(lat, f, prec):
    out = torch.zeros((1, lat.V, 4, lat.d, 2), dtype=torch.float64, device="cuda")
    lat.unpack(out, f, 0, prec)
    return to_complex(out)[0]


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("dagger", [0, 1])
def test_batch_dphi_matches_oracle(hr, prec, dagger):
    eps, m0s = 0.5, [-0.3, -0.2, -0.35, -0.3, -0.25, -0.4, -0.3]
    lats, ops, psis, ins, outs = [], [], [], [], []
    for k, (T, L, N, rep) in enumerate(SMALL_BATCH):
        lat, _ = gpu_lattice(hr, T, L, N, rep, eps, 0.0, seed=k)
        op = oracle_operator(T, L, N, rep, eps, m0s[k], 0.0, seed=k)
        psi = inputs.gaussian_spinor(10 + k, T, L, lat.d)[0]
        lats.append(lat)
        ops.append(op)
        psis.append(psi)
        ins.append(_fields(lat, psi, prec))
        outs.append(lat.new_field(0, prec))
    batch = hr.Batch(lats)
    batch.dphi(outs, ins, 0, m0s, prec, dagger)
    torch.cuda.synchronize()
    for k, lat in enumerate(lats):
        got = _unpack(lat, outs[k], prec)
        ref = ops[k].apply_schur(psis[k], 0, dagger=bool(dagger))
        mask = ops[k].geom.parity == 0
        assert rel_err(got, ref, mask) < _tol(prec), (k, SMALL_BATCH[k])
        # and the single-lattice entry point agrees
        one = lat.new_field(0, prec)
        lat.dphi(one, ins[k], 0, m0s[k], 0.0, prec, 1, dagger)
        assert rel_err(_unpack(lat, one, prec), got, mask) < _tol(prec)
    batch.close()


@pytest.mark.parametrize("inner,outer", [(1, 3), (2, 3), (1, 0), (2, 0)])  # outer 3: float-float, 0: FP64
def test_batch_cg_small(hr, inner, outer):
    eps, m0 = 0.5, -0.3
    lats, ops, bs, xs, bsrc = [], [], [], [], []
    for k, (T, L, N, rep) in enumerate(SMALL_BATCH):
        lat, _ = gpu_lattice(hr, T, L, N, rep, eps, 0.0, seed=k)
        lats.append(lat)
        ops.append(oracle_operator(T, L, N, rep, eps, m0, 0.0, seed=k))
        b = inputs.gaussian_spinor(20 + k, T, L, lat.d)[0]
        b[ops[-1].geom.parity == 1] = 0
        bsrc.append(b)
        bs.append(_fields(lat, b, 0))
        xs.append(lat.new_field(0, 0))
    batch = hr.Batch(lats)
    rc, st = batch.cg_solve(xs, bs, 0, [m0] * len(lats), 1e-8, inner_prec=inner, check_every=10,
                            outer_prec=outer)
    assert rc == 0
    for k, lat in enumerate(lats):
        x = _unpack(lat, xs[k], 0)
        op = ops[k]
        Mx = op.apply_schur(op.apply_schur(x, 0), 0, dagger=True)
        res = np.linalg.norm(bsrc[k] - Mx) / np.linalg.norm(bsrc[k])
        assert res <= 1.05e-8 and 0.0 < st[k]["true_residual"] <= 1e-8, (k, res, st[k])
        assert abs(st[k]["true_residual"] - res) <= 0.05 * res, (k, res, st[k])
        assert st[k]["iterations"] > 0
    batch.close()


def test_batch_64_lattices_to_1e8(hr):
    """The 64-lattice workload: shapes from seed 2, eps 0.5, m0 -0.3, csw 0, each solved to 1e-8."""
    shapes = inputs.batch_shapes(2, 64)
    eps, m0 = 0.5, -0.3
    lats, xs, bs = [], [], []
    for k, (T, L, N, rep) in enumerate(shapes):
        lat, _ = gpu_lattice(hr, T, L, N, rep, eps, 0.0, seed=100 + k)
        b = inputs.gaussian_spinor_rhs(200 + k, T, L, lat.d, 0)
        fb = lat.new_field(0, 0)
        lat.pack(fb, from_complex(b), 0, 0)
        del b
        lats.append(lat)
        bs.append(fb)
        xs.append(lat.new_field(0, 0))
    batch = hr.Batch(lats)
    rc, st = batch.cg_solve(xs, bs, 0, [m0] * 64, 1e-8, inner_prec=1, check_every=10)
    assert rc == 0
    assert all(s["true_residual"] <= 1e-8 for s in st)
    # oracle check of two lattices at sampled sites
    for k in (0, 37):
        T, L, N, rep = shapes[k]
        lat = lats[k]
        x = _unpack(lat, xs[k], 0)
        b = inputs.gaussian_spinor_rhs(200 + k, T, L, lat.d, 0)
        a = inputs.algebra_coefficients(100 + k, T, L, N)
        g = Geometry(T, L)
        op = WilsonOperator(None, N, rep, g, m0, 0.0,
                            link_fn=lambda s, a=a, N=N: sun.reunitarise(sun.links_from_algebra(a[s], eps, N)))
        sites = g.sites_of_parity(0)[:: max(1, (g.V // 2) // 8)][:8]
        s2 = np.unique(np.concatenate([sites] + [g.fwd[m][g.fwd[n][sites]] for m in range(4) for n in range(4)]
                                      + [g.bwd[m][g.bwd[n][sites]] for m in range(4) for n in range(4)]
                                      + [g.fwd[m][g.bwd[n][sites]] for m in range(4) for n in range(4)]))
        s2 = s2[g.parity[s2] == 0]
        y = op.apply_schur(x, 0, sites=s2)
        Mx = op.apply_schur(y, 0, dagger=True, sites=sites)
        be = np.where((g.parity == 0)[:, None, None], b, 0)
        res = np.linalg.norm(be[sites] - Mx[sites]) / np.linalg.norm(be[sites])
        assert res < 1e-7, (k, res)
    batch.close()


# one lattice per large-d_R class: complex 10, 12, 15, 21 and real 15, 24, 35
LARGE_BATCH = [(4, 4, 4, "sym"), (4, 2, 12, "fund"), (4, 4, 6, "asym"), (4, 2, 6, "sym"), (4, 4, 4, "adj"),
               (4, 2, 5, "adj"), (4, 2, 6, "adj")]


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_batch_every_class_shape(hr, prec):
    """Each candidate shape of each class, pinned in turn, in the persistent multi-lattice launch."""
    eps, m0 = 0.5, -0.3
    lats, ops, psis, ins, outs = [], [], [], [], []
    for k, (T, L, N, rep) in enumerate(LARGE_BATCH):
        lat, _ = gpu_lattice(hr, T, L, N, rep, eps, 0.0, seed=20 + k)
        ops.append(oracle_operator(T, L, N, rep, eps, m0, 0.0, seed=20 + k))
        psi = inputs.gaussian_spinor(30 + k, T, L, lat.d)[0]
        lats.append(lat)
        psis.append(psi)
        ins.append(_fields(lat, psi, prec))
        outs.append(lat.new_field(0, prec))
    batch = hr.Batch(lats)
    refs = [ops[k].apply_schur(psis[k], 0) for k in range(len(lats))]
    nshape = max(len(l.shape_candidates(prec)) for l in lats)
    for s in range(nshape):
        for lat in lats:
            cands = lat.shape_candidates(prec)
            batch.set_shape(lat.d, lat.is_real, prec, cands[min(s, len(cands) - 1)])
        batch.dphi(outs, ins, 0, [m0] * len(lats), prec, False)
        torch.cuda.synchronize()
        for k, lat in enumerate(lats):
            got = _unpack(lat, outs[k], prec)
            assert rel_err(got, refs[k], ops[k].geom.parity == 0) < _tol(prec), (s, LARGE_BATCH[k])
    batch.close()
