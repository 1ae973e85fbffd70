"""A host-side stand-in for one time slab of libhr (test infrastructure): the
same begin / end contract as ``hr.Lattice.domain_hop_begin`` / ``_end`` (and
the ``norm2`` / ``axpby`` of ``hr.Lattice``, over this slab's sites),
computed with numpy on full 4-spinors from the oracle's conventions, so that
``paper_2405_19294_gb300.slabs`` (buffer routing, stage order, exchange over
a process group) can run on gloo ranks without a GPU.  Its face buffers hold
full spinors per spatial site rather than libhr's half-spinors; only the
slab itself reads what it wrote, so the layout is private to it."""
import numpy as np
import torch

from oracle.dirac import GAMMA, Geometry

I4 = np.eye(4)


class FakeSlab:
    def __init__(self, UR_global: np.ndarray, T_global: int, L: int, t0: int, T_loc: int):
        self.L, self.t0, self.T = L, t0, T_loc
        self.geom = Geometry(T_loc, L)                    # periodic on its own; faces masked below
        V3 = L ** 3
        self.UR = UR_global[t0 * V3:(t0 + T_loc) * V3]    # lexicographic: the slab is contiguous
        self.d = UR_global.shape[-1]
        t = self.geom.coords[:, 0]
        self.top = t == T_loc - 1
        self.bottom = t == 0
        self.spatial = np.arange(self.geom.V) % V3         # face index: spatial lexicographic site

    # fields: complex128 [nrhs, V_loc, 4, d] CPU tensors; only sites of their parity are used
    def new_field(self, parity, prec, nrhs=1):
        return torch.zeros((nrhs, self.geom.V, 4, self.d), dtype=torch.complex128)

    def norm2(self, x, parity, prec, nrhs=1):
        m = self.geom.parity == parity
        return [float(np.sum(np.abs(x[r].numpy()[m]) ** 2)) for r in range(nrhs)]

    def axpby(self, x, y, a, b, parity, prec, nrhs=1):
        m = torch.from_numpy(self.geom.parity == parity)
        for r in range(nrhs):
            y[r][m] = a[r] * x[r][m] + b[r] * y[r][m]

    def new_halo(self, prec, nrhs=1):
        return torch.zeros((nrhs, self.L ** 3, 4, self.d), dtype=torch.complex128)

    def _masked_hop(self, psi, s, sites):
        g = self.geom
        out = np.zeros((len(sites), 4, self.d), complex)
        for mu in range(4):
            f, b = g.fwd[mu][sites], g.bwd[mu][sites]
            fwd = np.einsum("st,xta->xsa", I4 - s * GAMMA[mu], np.einsum("xac,xsc->xsa", self.UR[sites, mu], psi[f]))
            bwd = np.einsum("st,xta->xsa", I4 + s * GAMMA[mu],
                            np.einsum("xca,xsc->xsa", self.UR[b, mu].conj(), psi[b]))
            if mu == 0:
                fwd[self.top[sites]] = 0      # needs the slab above
                bwd[self.bottom[sites]] = 0   # needs the slab below
            out += fwd + bwd
        return out

    def domain_hop_begin(self, out, in_hop, self_field, out_parity, m0, prec, stage, send_up, send_down,
                         nrhs=1, dagger=False):
        s = -1 if dagger else 1
        g = self.geom
        q = 1 - out_parity
        diag = 4.0 + m0
        for r in range(nrhs):
            psi = in_hop[r].numpy()
            send_down[r].zero_()
            send_up[r].zero_()
            y = np.nonzero(self.bottom & (g.parity == q))[0]
            send_down[r][self.spatial[y]] = torch.from_numpy(np.einsum("st,xta->xsa", I4 - s * GAMMA[0], psi[y]))
            y = np.nonzero(self.top & (g.parity == q))[0]
            u = np.einsum("xca,xsc->xsa", self.UR[y, 0].conj(), psi[y])
            send_up[r][self.spatial[y]] = torch.from_numpy(np.einsum("st,xta->xsa", I4 + s * GAMMA[0], u))
            x = np.nonzero(g.parity == out_parity)[0]
            h = self._masked_hop(psi, s, x)
            o = np.zeros((g.V, 4, self.d), complex)
            o[x] = (-0.5 / diag) * h if stage == 0 else diag * self_field[r].numpy()[x] + 0.5 * h
            out[r].copy_(torch.from_numpy(o))

    def domain_hop_end(self, out, out_parity, m0, prec, stage, recv_up, recv_down, nrhs=1, dagger=False):
        g = self.geom
        coef = 0.5 if stage else -0.5 / (4.0 + m0)
        for r in range(nrhs):
            o = out[r].numpy().copy()
            x = np.nonzero(self.top & (g.parity == out_parity))[0]
            o[x] += coef * np.einsum("xac,xsc->xsa", self.UR[x, 0], recv_up[r].numpy()[self.spatial[x]])
            x = np.nonzero(self.bottom & (g.parity == out_parity))[0]
            o[x] += coef * recv_down[r].numpy()[self.spatial[x]]
            out[r].copy_(torch.from_numpy(o))
