"""ctypes binding of libhr (include/hr.h): argument marshalling only.

Every computation runs inside libhr's CUDA kernels; this module turns torch
tensors into device pointers and the current torch stream into the
library's stream, and raises ``HrError`` on a non-zero status.  Importing it
fails loudly if ``libhr.so`` has not been built (``__graft_entry__.build()``
or ``python -m paper_2405_19294_gb300.build``).
"""
from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("HR_LIBRARY") or os.path.join(HERE, "libhr.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "hr.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libhr.so is not built ({LIB_PATH}); run __graft_entry__.build()")
_lib = C.CDLL(LIB_PATH)

FUND, ADJ, SYM, ASYM = 0, 1, 2, 3
REP = {"fund": FUND, "adj": ADJ, "sym": SYM, "asym": ASYM}
EVEN, ODD, FULL = 0, 1, 2
F64, F32, F16, FF = 0, 1, 2, 3  # FF: float-float (hi + lo FP32 pairs in the FP64 field layout)
PREC = {"f64": F64, "f32": F32, "f16": F16, "ff": FF}


class hr_info(C.Structure):
    _fields_ = [("T", C.c_int), ("L", C.c_int), ("N", C.c_int), ("rep", C.c_int), ("d", C.c_int),
                ("is_real", C.c_int), ("volume", C.c_int64), ("half_volume", C.c_int64),
                ("flops_hop_site", C.c_double), ("bytes_hop_site", C.c_double * 3)]


class hr_cg_params(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int), ("inner_prec", C.c_int),
                ("inner_tol", C.c_double), ("nrhs", C.c_int), ("check_every", C.c_int),
                ("outer_prec", C.c_int)]


class hr_cg_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("outer_steps", C.c_int), ("true_residual", C.c_double),
                ("seconds", C.c_double), ("hop_launches", C.c_double)]


_P = C.c_void_p
_SIGS = {
    "hr_lattice_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(_P)]),
    "hr_lattice_destroy": (C.c_int, [_P]),
    "hr_set_stream": (C.c_int, [_P, _P]),
    "hr_lattice_info": (C.c_int, [_P, C.POINTER(hr_info)]),
    "hr_field_bytes": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_size_t)]),
    "hr_synchronize": (C.c_int, [_P]),
    "hr_links_from_algebra": (C.c_int, [_P, _P, _P, C.c_double, C.c_int]),
    "hr_represent_links": (C.c_int, [_P, _P, C.c_int, C.c_double]),
    "hr_export_represented_links": (C.c_int, [_P, _P]),
    "hr_export_clover": (C.c_int, [_P, _P, C.c_double, C.c_int]),
    "hr_set_clover_exponential": (C.c_int, [_P, C.c_int]),
    "hr_pack_spinor": (C.c_int, [_P, _P, _P, C.c_int, C.c_int, C.c_int]),
    "hr_unpack_spinor": (C.c_int, [_P, _P, _P, C.c_int, C.c_int, C.c_int]),
    "hr_dphi": (C.c_int, [_P, _P, _P, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int]),
    "hr_norm2": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "hr_cg_solve": (C.c_int, [_P, _P, _P, C.c_int, C.c_double, C.c_double, C.POINTER(hr_cg_params),
                              C.POINTER(hr_cg_stats)]),
    "hr_axpby": (C.c_int, [_P, _P, _P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int, C.c_int, C.c_int]),
    "hr_norm2_static": (C.c_int, [_P, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P]),
    "hr_tuned_shape": (C.c_int, [_P, C.c_int, C.c_int, C.c_int]),
    "hr_hop_shape_candidates": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int]),
    "hr_set_tuned_shape": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int]),
    "hr_batch_create": (C.c_int, [C.c_int, C.POINTER(_P), C.POINTER(_P)]),
    "hr_batch_destroy": (C.c_int, [_P]),
    "hr_batch_set_stream": (C.c_int, [_P, _P]),
    "hr_batch_set_shape": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int]),
    "hr_batch_dphi": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_P), C.c_int, C.POINTER(C.c_double), C.c_int, C.c_int]),
    "hr_batch_cg_solve": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_P), C.c_int, C.POINTER(C.c_double),
                                    C.POINTER(hr_cg_params), C.POINTER(hr_cg_stats)]),
    "hr_bicgstab_solve": (C.c_int, [_P, _P, _P, C.c_int, C.c_double, C.c_double, C.POINTER(hr_cg_params),
                                    C.POINTER(hr_cg_stats)]),
    "hr_lattice_create_domain": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(_P)]),
    "hr_domain_halo_bytes": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(C.c_size_t)]),
    "hr_domain_hop_begin": (C.c_int, [_P, _P, _P, _P, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int,
                                      _P, _P]),
    "hr_domain_hop_end": (C.c_int, [_P, _P, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P]),
    "hr_domains_dphi": (C.c_int, [C.c_int, C.POINTER(_P), C.POINTER(_P), C.POINTER(_P), C.c_int, C.c_double,
                                  C.c_int, C.c_int, C.c_int]),
    "hr_set_allocator": (C.c_int, [_P, _P, _P]),
    "hr_status_string": (C.c_char_p, [C.c_int]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def declared_symbols() -> list[str]:
    """Function names declared in include/hr.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(hr_\w+)\s*\(", txt, re.M)))


class HrError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {_lib.hr_status_string(status).decode()} ({status})")


def _check(rc: int, what: str):
    if rc != 0:
        raise HrError(rc, what)


def _ptr(t) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA torch tensor")
    return t.data_ptr()


def _ptr_or_pinned(t) -> int:
    """Device tensor, or page-locked host tensor (read/written by the kernel in place)."""
    import torch
    if isinstance(t, torch.Tensor) and (t.is_cuda or t.is_pinned()):
        return t.data_ptr()
    raise TypeError("expected a CUDA tensor or a pinned host tensor")


class Lattice:
    """One T x L^3 lattice of SU(N) fermions in representation ``rep`` (owns a libhr handle)."""

    def __init__(self, T: int, L: int, N: int, rep: str, t0: int | None = None, T_global: int | None = None):
        """With t0 and T_global: the time slab [t0, t0 + T) of a T_global x L^3 lattice."""
        import torch
        h = _P()
        if t0 is None:
            _check(_lib.hr_lattice_create(T, L, N, REP[rep], C.byref(h)), "hr_lattice_create")
        else:
            _check(_lib.hr_lattice_create_domain(T, L, N, REP[rep], t0, T_global, C.byref(h)),
                   "hr_lattice_create_domain")
        self._h = h
        self.T, self.L, self.N, self.rep = T, L, N, rep
        self.t0, self.T_global = (0, T) if t0 is None else (t0, T_global)
        info = hr_info()
        _check(_lib.hr_lattice_info(h, C.byref(info)), "hr_lattice_info")
        self.d = info.d
        self.is_real = bool(info.is_real)
        self.V = info.volume
        self.Vh = info.half_volume
        self.flops_hop_site = info.flops_hop_site
        self.bytes_hop_site = list(info.bytes_hop_site)
        self.use_stream(torch.cuda.current_stream())

    def close(self):
        if getattr(self, "_h", None):
            _lib.hr_lattice_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def use_stream(self, stream):
        _check(_lib.hr_set_stream(self._h, C.c_void_p(stream.cuda_stream)), "hr_set_stream")

    def synchronize(self):
        _check(_lib.hr_synchronize(self._h), "hr_synchronize")

    # -- fields ----------------------------------------------------------
    def field_bytes(self, parity: int, prec: int, nrhs: int = 1) -> int:
        n = C.c_size_t()
        _check(_lib.hr_field_bytes(self._h, parity, prec, nrhs, C.byref(n)), "hr_field_bytes")
        return n.value

    def new_field(self, parity: int, prec: int, nrhs: int = 1):
        """A zeroed internal field (uint8 device tensor of field_bytes bytes)."""
        import torch
        return torch.zeros(self.field_bytes(parity, prec, nrhs), dtype=torch.uint8, device="cuda")

    def pack(self, internal, canonical, parity: int, prec: int, nrhs: int = 1):
        """Canonical FP64 spinors psi[nrhs][V][4][d][2] (device or page-locked host tensor) ->
        internal field of the given parity and precision (hr_pack_spinor)."""
        _check(_lib.hr_pack_spinor(self._h, _ptr(internal), _ptr_or_pinned(canonical), parity, prec, nrhs),
               "hr_pack_spinor")

    def unpack(self, canonical, internal, parity: int, prec: int, nrhs: int = 1):
        """Internal field -> canonical FP64 spinors; other-parity sites untouched (hr_unpack_spinor)."""
        _check(_lib.hr_unpack_spinor(self._h, _ptr_or_pinned(canonical), _ptr(internal), parity, prec, nrhs),
               "hr_unpack_spinor")

    # -- gauge -----------------------------------------------------------
    def links_from_algebra(self, U, a, eps: float, reunitarise: bool = True):
        """U[V][4][N][N][2] = exp(i eps sum_k a_k T_k) from a[V][4][N^2-1] (both FP64 device tensors)."""
        _check(_lib.hr_links_from_algebra(self._h, _ptr(U), _ptr(a), eps, int(reunitarise)),
               "hr_links_from_algebra")

    def represent_links(self, U, reunitarise: bool = True, csw: float = 0.0):
        """Build U_R (with the antiperiodic time sign) in every precision, and the clover term if csw != 0."""
        _check(_lib.hr_represent_links(self._h, _ptr(U), int(reunitarise), csw), "hr_represent_links")

    def export_represented_links(self, out):
        _check(_lib.hr_export_represented_links(self._h, _ptr(out)), "hr_export_represented_links")

    def export_clover(self, out, m0: float, inverse: bool = False):
        _check(_lib.hr_export_clover(self._h, _ptr(out), m0, int(inverse)), "hr_export_clover")

    def set_clover_exponential(self, on: bool = True):
        """A = (4 + m0) exp(C / (4 + m0)) instead of (4 + m0) + C for later calls."""
        _check(_lib.hr_set_clover_exponential(self._h, int(bool(on))), "hr_set_clover_exponential")

    # -- operator and solver ---------------------------------------------
    def dphi(self, out, inp, parity: int, m0: float, csw: float, prec: int, nrhs: int = 1,
             dagger: bool = False):
        """out = Dhat_parity inp (EVEN/ODD) or D inp (FULL), or the adjoint; internal fields of
        precision prec, nrhs back to back; queued on the lattice's stream (hr_dphi)."""
        _check(_lib.hr_dphi(self._h, _ptr(out), _ptr(inp), parity, m0, csw, prec, nrhs, int(dagger)),
               "hr_dphi")

    @staticmethod
    def _decode(v):
        return ((v % 100000) // 1000, v % 1000, (v % 1000000) // 100000, (v % 100000000) // 1000000,
                v // 100000000)

    def tuned_shape(self, prec: int, nrhs: int = 1, clover: bool = False):
        """(G threads per site or 0, threads per block, register budget, multi-rhs sites per block,
        rows per warp of the rows kernel or 0) chosen by the autotuner, or None."""
        v = _lib.hr_tuned_shape(self._h, prec, nrhs, int(clover))
        return None if v < 0 else self._decode(v)

    def shape_candidates(self, prec: int, nrhs: int = 1, clover: bool = False):
        buf = (C.c_int * 32)()
        n = _lib.hr_hop_shape_candidates(self._h, prec, nrhs, int(clover), buf, 32)
        if n < 0:
            raise HrError(n, "hr_hop_shape_candidates")
        return [self._decode(v) for v in buf[:min(n, 32)]]

    def set_shape(self, prec: int, shape, nrhs: int = 1, clover: bool = False):
        _check(_lib.hr_set_tuned_shape(self._h, prec, nrhs, int(clover), _shape_code(shape)),
               "hr_set_tuned_shape")

    # -- time-slab sub-domain -------------------------------------------
    def halo_bytes(self, prec: int, nrhs: int = 1) -> int:
        n = C.c_size_t()
        _check(_lib.hr_domain_halo_bytes(self._h, prec, nrhs, C.byref(n)), "hr_domain_halo_bytes")
        return n.value

    def new_halo(self, prec: int, nrhs: int = 1):
        import torch
        return torch.empty(self.halo_bytes(prec, nrhs), dtype=torch.uint8, device="cuda")

    def domain_hop_begin(self, out, in_hop, self_field, out_parity: int, m0: float, prec: int, stage: int,
                         send_up, send_down, nrhs: int = 1, dagger: bool = False):
        sp = _ptr(self_field) if self_field is not None else None
        _check(_lib.hr_domain_hop_begin(self._h, _ptr(out), _ptr(in_hop), sp, out_parity, m0, prec, nrhs,
                                        int(dagger), stage, _ptr(send_up), _ptr(send_down)), "hr_domain_hop_begin")

    def domain_hop_end(self, out, out_parity: int, m0: float, prec: int, stage: int, recv_up, recv_down,
                       nrhs: int = 1, dagger: bool = False):
        _check(_lib.hr_domain_hop_end(self._h, _ptr(out), out_parity, m0, prec, nrhs, int(dagger), stage,
                                      _ptr(recv_up), _ptr(recv_down)), "hr_domain_hop_end")

    def norm2(self, x, parity: int, prec: int, nrhs: int = 1):
        """|x_r|^2 per right-hand side, accumulated in FP64 (synchronous)."""
        out = (C.c_double * nrhs)()
        _check(_lib.hr_norm2(self._h, _ptr(x), parity, prec, nrhs, out), "hr_norm2")
        return list(out)

    def axpby(self, x, y, a, b, parity: int, prec: int, nrhs: int = 1):
        """y_r = a_r x_r + b_r y_r per rhs (a, b: scalars or sequences of nrhs floats)."""
        av = a if hasattr(a, "__len__") else [a] * nrhs
        bv = b if hasattr(b, "__len__") else [b] * nrhs
        A = (C.c_double * nrhs)(*[float(v) for v in av])
        B = (C.c_double * nrhs)(*[float(v) for v in bv])
        _check(_lib.hr_axpby(self._h, _ptr(x), _ptr(y), A, B, parity, prec, nrhs), "hr_axpby")

    def cg_solve(self, x, b, parity: int, m0: float, csw: float, tol: float, inner_prec: int = F64,
                 inner_tol: float = 0.0, nrhs: int = 1, maxit: int = 100000, check_every: int = 10,
                 raise_on_error: bool = True, outer_prec: int = FF):
        """Solve Dhat^+ Dhat x = b (D^+ D for FULL) to a true relative residual tol: plain FP64
        CG, or defect correction around an FP32 / FP16 inner CG whose outer residuals run in
        outer_prec (F64, or FF: float-float) (hr_cg_solve).  Returns the status and statistics;
        raises HrError on failure unless raise_on_error is False."""
        prm = hr_cg_params(tol, maxit, inner_prec, inner_tol, nrhs, check_every, outer_prec)
        st = hr_cg_stats()
        rc = _lib.hr_cg_solve(self._h, _ptr(x), _ptr(b), parity, m0, csw, C.byref(prm), C.byref(st))
        if rc != 0 and raise_on_error:
            raise HrError(rc, "hr_cg_solve")
        return {"status": rc, "iterations": st.iterations, "outer_steps": st.outer_steps,
                "true_residual": st.true_residual, "seconds": st.seconds,
                "hop_launches": st.hop_launches}


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)
_allocator_refs = []


def use_torch_allocator(on: bool = True):
    """Back libhr's large device buffers by PyTorch's caching allocator (on the
    current device and stream), so they show in torch.cuda.memory_allocated()
    and share its pool; on=False returns to cudaMalloc."""
    import torch
    if not on:
        _check(_lib.hr_set_allocator(None, None, None), "hr_set_allocator")
        return

    def alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(nbytes)
        except Exception:
            return None

    def release(ptr, nbytes, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    fa, ff = _ALLOC_FN(alloc), _FREE_FN(release)
    _allocator_refs.append((fa, ff))   # the C side keeps the pointers: keep the thunks alive
    _check(_lib.hr_set_allocator(C.cast(fa, _P), C.cast(ff, _P), None), "hr_set_allocator")


def domains_dphi(lats, outs, ins, parity: int, m0: float, prec: int, nrhs: int = 1, dagger: bool = False):
    """Dhat_p on all time slabs of one lattice held in this process (exchange by device copies)."""
    n = len(lats)
    arr = lambda xs: (_P * n)(*[_P(_ptr(x)) for x in xs])
    hs = (_P * n)(*[l._h for l in lats])
    _check(_lib.hr_domains_dphi(n, hs, arr(outs), arr(ins), parity, m0, prec, nrhs, int(dagger)), "hr_domains_dphi")


def _shape_code(shape):
    """(G, block, regs[, mrhs[, rows]]) -> the integer code of the C ABI."""
    g, bs, regs = shape[0], shape[1], shape[2]
    mr = shape[3] if len(shape) > 3 else 0
    rows = shape[4] if len(shape) > 4 else 0
    return rows * 100000000 + mr * 1000000 + regs * 100000 + g * 1000 + bs


class Batch:
    """Many lattices solved together (one launch per representation class and stage)."""

    def __init__(self, lattices):
        import torch
        self.lattices = list(lattices)
        arr = (_P * len(self.lattices))(*[l._h for l in self.lattices])
        h = _P()
        _check(_lib.hr_batch_create(len(self.lattices), arr, C.byref(h)), "hr_batch_create")
        self._h = h
        _check(_lib.hr_batch_set_stream(h, C.c_void_p(torch.cuda.current_stream().cuda_stream)),
               "hr_batch_set_stream")

    def close(self):
        if getattr(self, "_h", None):
            _lib.hr_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ptrs(self, ts):
        return (_P * len(ts))(*[_ptr(t) for t in ts])

    def set_shape(self, d: int, is_real: bool, prec: int, shape):
        """Pin the launch shape (a tuple as Lattice.shape_candidates lists them) of class (d, is_real)."""
        _check(_lib.hr_batch_set_shape(self._h, d, int(is_real), prec, _shape_code(shape)), "hr_batch_set_shape")

    def dphi(self, outs, ins, parity: int, m0s, prec: int, dagger: bool = False):
        m = (C.c_double * len(m0s))(*m0s)
        _check(_lib.hr_batch_dphi(self._h, self._ptrs(outs), self._ptrs(ins), parity, m, prec, int(dagger)),
               "hr_batch_dphi")

    def cg_solve(self, xs, bs, parity: int, m0s, tol: float, inner_prec: int = F32, inner_tol: float = 0.0,
                 maxit: int = 100000, check_every: int = 10, raise_on_error: bool = True, outer_prec: int = FF):
        """Lock-step mixed CG on every lattice of the batch; outer residuals in outer_prec
        (FF: float-float, F64) (hr_batch_cg_solve)."""
        m = (C.c_double * len(m0s))(*m0s)
        prm = hr_cg_params(tol, maxit, inner_prec, inner_tol, 1, check_every, outer_prec)
        st = (hr_cg_stats * len(xs))()
        rc = _lib.hr_batch_cg_solve(self._h, self._ptrs(xs), self._ptrs(bs), parity, m, C.byref(prm), st)
        if rc != 0 and raise_on_error:
            raise HrError(rc, "hr_batch_cg_solve")
        return rc, [{"iterations": s.iterations, "outer_steps": s.outer_steps, "true_residual": s.true_residual,
                     "seconds": s.seconds} for s in st]


def _bicgstab(self, x, b, parity: int, m0: float, csw: float, tol: float, inner_prec: int = F64,
              inner_tol: float = 0.0, nrhs: int = 1, maxit: int = 100000, check_every: int = 10,
              raise_on_error: bool = True, outer_prec: int = FF):
    """BiCGstab on Dhat (D for FULL) to a true relative residual tol: plain FP64, or defect
    correction around an FP32 inner BiCGstab with outer residuals in outer_prec (hr_bicgstab_solve)."""
    prm = hr_cg_params(tol, maxit, inner_prec, inner_tol, nrhs, check_every, outer_prec)
    st = hr_cg_stats()
    rc = _lib.hr_bicgstab_solve(self._h, _ptr(x), _ptr(b), parity, m0, csw, C.byref(prm), C.byref(st))
    if rc != 0 and raise_on_error:
        raise HrError(rc, "hr_bicgstab_solve")
    return {"status": rc, "iterations": st.iterations, "outer_steps": st.outer_steps,
            "true_residual": st.true_residual, "seconds": st.seconds}


Lattice.bicgstab_solve = _bicgstab


def lib_handle():
    """The loaded ctypes library (for tests of the exported symbols)."""
    return _lib
