"""Benchmark: even-odd Wilson-Dirac operator GB/s and CG time-to-1e-10.

Workload (default): SU(3) fundamental fermions on a 32^3 x 64 lattice, links
exp(i eps sum a_k T_k) with eps = 1.0 (seeded Gaussian a_k, reunitarised),
m0 = -0.4, the Schur complement Dhat on the even sites.  One step = one
FP32 application of Dhat (two hopping launches) on a Gaussian source, with L2
flushed between steps by reading a 512 MiB buffer (a read leaves no dirty
lines to be written back inside the next timed step); value = algorithmic bytes / time,
where the bytes are the ideal-reuse model 16*l*w + 5*s*w per even site
(l = link reals, s = spinor reals, w = bytes per real).  The same line reports
the FP64 Dhat, the end-to-end number through the C ABI with host buffers, and
CG on Dhat^+ Dhat to a true FP64 relative residual of 1e-10 (plain FP64,
FP32-inner and FP16-inner mixed precision).

--impl reference times the FP64 CPU oracle on all host cores instead (bounded
sample: the same operator on a 32 x 16^3 lattice per step, its even sites
split over one process per core) in the same unit.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Dphi GB/s (% of HBM peak) + CG time-to-1e-10, mixed/multi-RHS vs FP64"
WORKLOAD = dict(T=64, L=32, N=3, rep="fund", eps=1.0, m0=-0.4, csw=0.0)
SAMPLE = dict(T=32, L=16)  # bounded CPU sample for the oracle legs


def bytes_per_even_site(N, rep, w):
    """Ideal-reuse bytes of one Dhat application per even site: 16 l w + 5 s w."""
    d = {"fund": N, "adj": N * N - 1, "sym": N * (N + 1) // 2, "asym": N * (N - 1) // 2}[rep]
    l = d * d if rep == "adj" else 2 * d * d
    s = 8 * d
    extra = 5 * 4 if w == 2 else 0   # FP16 site scales: 5 spinor passes
    return 16 * l * w + 5 * s * w + extra


def flops_per_even_site(N, rep):
    d = {"fund": N, "adj": N * N - 1, "sym": N * (N + 1) // 2, "asym": N * (N - 1) // 2}[rep]
    hop = (64 if rep == "adj" else 128) * d * d + 56 * d
    return 2 * hop


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ----------------------------------------------------------------- clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[5 + k]
                          and "Not" not in r[5 + k]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------- reference arm --
# The FP64 oracle on the host cores: the even Schur operator on a bounded
# sample lattice, its even sites split into one contiguous block per worker
# process (spawned, so that no worker inherits a CUDA context).  Every worker
# builds the same seeded operator once; a step hands each worker its block.
_ORACLE = {}


def _oracle_init(T, L):
    from oracle import sun
    from oracle.dirac import Geometry, WilsonOperator
    from paper_2405_19294_gb300 import inputs
    wl = WORKLOAD
    g = Geometry(T, L)
    a = inputs.algebra_coefficients(0, T, L, wl["N"])
    U = sun.reunitarise(sun.links_from_algebra(a, wl["eps"], wl["N"]))
    op = WilsonOperator(U, wl["N"], wl["rep"], g, wl["m0"], wl["csw"])
    _ORACLE["op"] = op
    _ORACLE["psi"] = inputs.gaussian_spinor(1, T, L, op.d)[0]


def _oracle_block(sites):
    op, psi = _ORACLE["op"], _ORACLE["psi"]
    return op.apply_schur(psi, 0, sites=sites)[sites]


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


class OraclePool:
    """One spawned worker per host core, each holding the sample operator."""

    def __init__(self, T, L, cores=None):
        import multiprocessing as mp
        from oracle.dirac import Geometry
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"     # one thread per worker process
        self.cores = cores or os.cpu_count() or 1
        self.T, self.L = T, L
        ev = Geometry(T, L).sites_of_parity(0)
        self.sites = len(ev)
        self.blocks = [b for b in np.array_split(ev, self.cores) if len(b)]
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_init, initargs=(T, L))
        self.pool.map(_oracle_block, self.blocks)    # every worker has built its operator

    def dhat(self):
        """One even Schur operator application over all blocks; wall seconds."""
        t0 = time.perf_counter()
        self.pool.map(_oracle_block, self.blocks, chunksize=1)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()

    def describe(self, reps, sec):
        return (f"Dhat even on {self.T}x{self.L}^3 ({self.sites} even sites) per step, split over "
                f"{self.cores} worker processes (one per host core, {cpu_model()}); {reps} reps, "
                f"{sec * 1e3:.1f} ms each")


def run_reference(args):
    """The FP64 oracle on the host cores: Dhat on the bounded sample lattice per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    T, L = SAMPLE["T"], SAMPLE["L"]
    pool = OraclePool(T, L)
    for _ in range(args.warmup):
        pool.dhat()
    t = [pool.dhat() for _ in range(args.steps)]
    pool.close()
    ms = 1e3 * float(np.mean(t))
    gbs = bytes_per_even_site(WORKLOAD["N"], WORKLOAD["rep"], 4) * pool.sites / (ms * 1e-3) / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(gbs, 4), "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"SU(3) fund 32^3x64 Dhat even (sampled: {T}x{L}^3 per step)",
                       "T": WORKLOAD["T"], "L": WORKLOAD["L"], "seeds": {"links": 0, "source": 1}},
            "cpu_baseline": {"value": round(gbs, 4), "unit": "GB/s (FP32-equivalent bytes of the same Dhat)",
                             "cores": pool.cores, "cpu": cpu_model(), "kind": "oracle",
                             "sample": pool.describe(args.steps, ms * 1e-3)},
            "e2e": {"value": round(gbs, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def cpu_baseline_leg(seconds=10.0):
    """Time the oracle's Dhat on the bounded sample over all host cores (about 10 s)."""
    T, L = SAMPLE["T"], SAMPLE["L"]
    pool = OraclePool(T, L)
    pool.dhat()
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < seconds:
        pool.dhat()
        n += 1
    dt = (time.perf_counter() - t0) / n
    pool.close()
    gbs = bytes_per_even_site(WORKLOAD["N"], WORKLOAD["rep"], 4) * pool.sites / dt / 1e9
    return {"value": round(gbs, 4), "unit": "GB/s (FP32-equivalent bytes of the same Dhat)",
            "cores": pool.cores, "cpu": cpu_model(), "kind": "oracle", "sample": pool.describe(n, dt)}


# ------------------------------------------------------- multi-process --
def job_timing(ms_step, world, dist, device=None):
    """Whole-job step time: the maximum over ranks (replicas run independent
    lattices, so the job finishes when the slowest rank does).  A host-side
    reduction of one scalar; no data of the operator crosses ranks."""
    if dist is None or world == 1:
        return float(ms_step)
    import torch
    t = torch.tensor([float(ms_step)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(bytes_per_step_per_rank, world, ms_job):
    """Aggregate GB/s over all ranks: every rank moves its own replica's bytes."""
    return world * bytes_per_step_per_rank / (ms_job * 1e-3) / 1e9


# ------------------------------------------------------------------ main --
def hop_source_digest():
    h = hashlib.sha256()
    for f in ("hop.cuh", "cplx.cuh"):
        with open(os.path.join(ROOT, "paper_2405_19294_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(key):
    """DRAM bytes per even site from the committed ncu capture, if the kernel is unchanged."""
    p = os.path.join(ROOT, "profiles", "hop_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    if rec.get("source_digest") != hop_source_digest():
        return None
    return rec.get(key)


# ------------------------------------------------------------ suite mode --
def _lattice(hr, inputs, torch, T, L, N, rep, eps, csw, seed=0):
    lat = hr.Lattice(T, L, N, rep)
    a = torch.from_numpy(inputs.algebra_coefficients(seed, T, L, N)).cuda()
    U = torch.empty((lat.V, 4, N, N, 2), dtype=torch.float64, device="cuda")
    lat.links_from_algebra(U, a, eps, True)
    lat.represent_links(U, True, csw)
    del a, U
    return lat


def _pack_rhs(lat, inputs, torch, seed, T, L, nrhs, prec, parity=0):
    f = lat.new_field(parity, prec, nrhs)
    fb = lat.field_bytes(parity, prec, 1)
    for r in range(nrhs):
        psi = inputs.gaussian_spinor_rhs(seed, T, L, lat.d, r)
        lat.pack(f[r * fb:(r + 1) * fb], torch.from_numpy(np.stack([psi.real, psi.imag], -1)).cuda(), parity, prec)
    return f


def _timed_cg(lat, fx, fb, m0, csw, inner, nrhs=1, inner_tol=0.0, reps=2, outer=3):
    """Wall time of a CG solve to 1e-10 (mixed: outer residuals in float-float, outer=3, or FP64, 0)."""
    import torch
    res = None
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = lat.cg_solve(fx, fb, 0, m0, csw, 1e-10, inner_prec=inner, inner_tol=inner_tol, nrhs=nrhs,
                           check_every=20, raise_on_error=False, outer_prec=outer)
        res["wall_s"] = round(time.perf_counter() - t0, 4)
    res["outer"] = None if inner == 0 else ("ff" if outer == 3 else "fp64")
    return res


def _warm(lat, prec, nrhs, m0, csw):
    """One operator application per key so the autotuner runs outside the timed solves."""
    fi = lat.new_field(0, prec, nrhs)
    fo = lat.new_field(0, prec, nrhs)
    lat.dphi(fo, fi, 0, m0, csw, prec, nrhs)
    lat.dphi(fi, fo, 0, m0, csw, prec, nrhs, True)
    lat.synchronize()


def run_suite(args):
    """Measurements of the other workloads (one JSON line each; not the bench line)."""
    import torch
    from paper_2405_19294_gb300 import hr, inputs
    out = []
    which = set(args.suite.split(","))
    # SU(2) adjoint and SU(4) antisymmetric on 24^3 x 48: mixed-precision CG
    for N, rep in ((2, "adj"), (4, "asym")) if "c2" in which else ():
        T, L, m0 = 48, 24, -0.3
        lat = _lattice(hr, inputs, torch, T, L, N, rep, 1.0, 0.0)
        fb = _pack_rhs(lat, inputs, torch, 1, T, L, 1, hr.F64)
        fx = lat.new_field(0, hr.F64)
        line = {"suite": "SU(%d) %s 24^3x48 CG to 1e-10" % (N, rep), "m0": m0}
        for name, inner, itol in (("fp64", hr.F64, 0.0), ("mixed_fp32", hr.F32, 0.0),
                                  ("mixed_fp16", hr.F16, 0.0), ("mixed_fp16_itol3e-3", hr.F16, 3e-3)):
            r = _timed_cg(lat, fx, fb, m0, 0.0, inner, inner_tol=itol)
            line[name] = {k: r[k] for k in ("wall_s", "iterations", "outer_steps", "true_residual", "status")}
        for k in list(line):
            if k.startswith("mixed") and line["fp64"]["wall_s"] > 0:
                line[k]["speedup_vs_fp64"] = round(line["fp64"]["wall_s"] / line[k]["wall_s"], 2)
        # Dhat GB/s per precision (L2 flushed between steps)
        flush = torch.ones(128 << 20, dtype=torch.float32, device="cuda")
        gb = {}
        for prec in (hr.F32, hr.F16):
            fi = _pack_rhs(lat, inputs, torch, 1, T, L, 1, prec)
            fo = lat.new_field(0, prec)
            for _ in range(3):
                lat.dphi(fo, fi, 0, m0, 0.0, prec)
            ts = []
            st = torch.cuda.current_stream()
            for _ in range(20):
                flush.sum()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                lat.dphi(fo, fi, 0, m0, 0.0, prec)
                e1.record(st)
                ts.append((e0, e1))
            torch.cuda.synchronize()
            ms = float(np.median([a_.elapsed_time(b_) for a_, b_ in ts]))
            w = 4 if prec == hr.F32 else 2
            gb[("fp32", "fp32", "fp16")[prec]] = round(bytes_per_even_site(N, rep, w) * lat.Vh / ms / 1e6, 1)
        line["dhat_gbs"] = gb
        out.append(line)
        print(json.dumps(line), flush=True)
        lat.close()
        del fb, fx
        torch.cuda.empty_cache()
    if "bicg" in which:
        out.append(_suite_bicgstab(hr, inputs, torch))
    if "c3" in which:
        out.append(_suite_c3(hr, inputs, torch))
    if "c4" in which:
        out.append(_suite_c4(hr, inputs, torch))
    if "largen" in which:
        out.extend(_suite_large_nc(hr, inputs, torch))
    if "larged" in which:
        out.extend(_suite_large_d(hr, inputs, torch))
    if "blas" in which:
        out.append(_suite_blas(hr, inputs, torch))
    return out


def _suite_blas(hr, inputs, torch):
    """Reduction bandwidth (Sec. 3.2): hr_norm2 over 12 even-parity SU(3) fields of 32^3 x 64
    per precision, wall time per call (it returns the sums to the host), cold L2."""
    T, L, N, rep, nr = 64, 32, 3, "fund", 12
    lat = _lattice(hr, inputs, torch, T, L, N, rep, 1.0, 0.0)
    flush = torch.ones(128 << 20, dtype=torch.float32, device="cuda")
    peak = measured_peaks()[0]["hbm_gbs"]
    line = {"suite": "norm2 of 12 even-parity SU(3) fund fields, 32^3x64, FP64 accumulation", "fields": nr}
    for name, prec in (("fp64", hr.F64), ("fp32", hr.F32), ("fp16", hr.F16)):
        f = lat.new_field(0, prec, nr)
        f.zero_()                  # contents do not matter for the timing
        nbytes = lat.field_bytes(0, prec, nr)
        for _ in range(3):
            lat.norm2(f, 0, prec, nr)
        ts = []
        for _ in range(10):
            flush.sum()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lat.norm2(f, 0, prec, nr)
            ts.append(time.perf_counter() - t0)
        dt = float(np.median(ts))
        line[name] = {"bytes": nbytes, "ms": round(dt * 1e3, 4), "GBs": round(nbytes / dt / 1e9, 1),
                      "frac_of_measured_copy": round(nbytes / dt / 1e9 / peak, 3)}
        del f
    print(json.dumps(line), flush=True)
    lat.close()
    return line


def _suite_large_d(hr, inputs, torch):
    """Every launch shape of the large representations (d_R = 8 ... 35), FP32 Dhat
    at 32 x 16^3 (and FP16 / FP64 for SU(6) adjoint), cold L2 between steps."""
    m0 = -0.4
    flush = torch.ones(128 << 20, dtype=torch.float32, device="cuda")
    lines = []
    for N, rep, prec in ((3, "adj", hr.F32), (4, "sym", hr.F32), (6, "asym", hr.F32), (4, "adj", hr.F32),
                         (6, "sym", hr.F32), (5, "adj", hr.F32), (6, "adj", hr.F32), (6, "adj", hr.F16),
                         (6, "sym", hr.F16), (6, "adj", hr.F64)):
        T, L = 32, 16
        lat = _lattice(hr, inputs, torch, T, L, N, rep, 1.0, 0.0)
        fi = _pack_rhs(lat, inputs, torch, 1, T, L, 1, prec)
        fo = lat.new_field(0, prec)
        w = {hr.F64: 8, hr.F32: 4, hr.F16: 2}[prec]
        bytes_ = bytes_per_even_site(N, rep, w) * lat.Vh
        shapes = {}
        for sh in lat.shape_candidates(prec):
            lat.set_shape(prec, sh)
            ms = _time_dhat(lat, fi, fo, m0, prec, torch, flush)
            fam = "site" if (sh[0] == 0 and sh[4] == 0) else ("rows" if sh[4] else "split")
            shapes[str(tuple(sh))] = {"family": fam, "ms": round(ms, 4), "GBs": round(bytes_ / ms / 1e6, 1)}
        best = {}
        for k, v in shapes.items():
            if v["family"] not in best or v["ms"] < best[v["family"]]["ms"]:
                best[v["family"]] = dict(v, shape=k)
        line = {"suite": "large d_R, Dhat at 16^3x32, every launch shape", "N": N, "rep": rep, "d": lat.d,
                "prec": ("fp64", "fp32", "fp16")[prec], "best_per_family": best, "shapes": shapes}
        print(json.dumps(line), flush=True)
        lines.append(line)
        lat.close()
        del fi, fo
        torch.cuda.empty_cache()
    return lines


def run_one_dhat(spec):
    """A single pinned-shape Dhat case for ncu captures: three applications, no timing.

    spec = N,REP,T,L,PREC,SHAPE[,CSW[,NRHS]] (defaults csw 0, one right-hand side)."""
    import torch
    from paper_2405_19294_gb300 import hr, inputs
    parts = spec.split(",")
    N, rep, T, L, prec, shape = parts[:6]
    csw = float(parts[6]) if len(parts) > 6 else 0.0
    nrhs = int(parts[7]) if len(parts) > 7 else 1
    N, T, L = int(N), int(T), int(L)
    prec = hr.PREC[prec]
    lat = _lattice(hr, inputs, torch, T, L, N, rep, 1.0, csw)
    fi = _pack_rhs(lat, inputs, torch, 1, T, L, nrhs, prec)
    fo = lat.new_field(0, prec, nrhs)
    lat.set_shape(prec, tuple(int(v) for v in shape.split(":")), nrhs=nrhs, clover=csw != 0)
    m0 = -0.35 if csw else -0.4
    for _ in range(3):
        lat.dphi(fo, fi, 0, m0, csw, prec, nrhs)
    torch.cuda.synchronize()
    print(json.dumps({"one_dhat": spec, "d": lat.d, "shape": lat.tuned_shape(prec, nrhs=nrhs, clover=csw != 0)}))


def _large_nc_geometry(N, target_bytes):
    """L^3 x T, T in {L, 3L/2, 2L} (both even), whose FP32 Dhat moves closest to target_bytes."""
    bps = bytes_per_even_site(N, "fund", 4)
    want = target_bytes / bps * 2          # sites of the full lattice
    best = None
    for L in range(4, 130, 2):
        for T in (L, 3 * L // 2, 2 * L):
            if T % 2:
                continue
            err = abs(T * L ** 3 - want) / want
            if best is None or err < best[0]:
                best = (err, T, L)
    return best[1], best[2]


def _time_dhat(lat, fi, fo, m0, prec, torch, flush, reps=10):
    for _ in range(2):
        lat.dphi(fo, fi, 0, m0, 0.0, prec)
    st = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        flush.sum()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        lat.dphi(fo, fi, 0, m0, 0.0, prec)
        e1.record(st)
        ts.append((e0, e1))
    torch.cuda.synchronize()
    return float(np.median([a.elapsed_time(b) for a, b in ts]))


def _suite_large_nc(hr, inputs, torch):
    """Large-N_c scaling (Sec. 3.1.2): SU(N_c) fundamental, N_c = 2 ... 12, FP32
    Dhat, the lattice shrunk as N_c grows so that every point moves about the
    same bytes; every launch shape timed, grouped into the one-site-per-thread
    kernel (the paper's default) and the kernels split over the colour rows
    (its LARGE_N kernel: here the rows and colour-split kernels)."""
    m0, prec = -0.3, hr.F32
    flush = torch.ones(128 << 20, dtype=torch.float32, device="cuda")
    lines = []
    for N in range(2, 13):
        T, L = _large_nc_geometry(N, 2.0e9)
        lat = _lattice(hr, inputs, torch, T, L, N, "fund", 1.0, 0.0)
        fi = _pack_rhs(lat, inputs, torch, 1, T, L, 1, prec)
        fo = lat.new_field(0, prec)
        bytes_ = bytes_per_even_site(N, "fund", 4) * lat.Vh
        flops = flops_per_even_site(N, "fund") * lat.Vh
        shapes = {}
        for sh in lat.shape_candidates(prec):
            lat.set_shape(prec, sh)
            ms = _time_dhat(lat, fi, fo, m0, prec, torch, flush)
            fam = "site" if (sh[0] == 0 and sh[4] == 0) else ("rows" if sh[4] else "split")
            shapes[str(tuple(sh))] = {"family": fam, "ms": round(ms, 4),
                                      "GBs": round(bytes_ / ms / 1e6, 1), "GFLOPs": round(flops / ms / 1e6, 1)}
        best = {}
        for k, v in shapes.items():
            if v["family"] not in best or v["ms"] < best[v["family"]]["ms"]:
                best[v["family"]] = dict(v, shape=k)
        line = {"suite": "large-N_c scaling, SU(N_c) fund, FP32 Dhat, ~2 GB moved per application",
                "N_c": N, "lattice": f"{L}^3x{T}", "even_sites": lat.Vh, "model_bytes": int(bytes_),
                "model_flops": int(flops), "best_per_family": best, "shapes": shapes}
        print(json.dumps(line), flush=True)
        lines.append(line)
        lat.close()
        del fi, fo
        torch.cuda.empty_cache()
    return lines


def _suite_bicgstab(hr, inputs, torch):
    """BiCGstab on Dhat directly vs CG on the normal equations, SU(3) fund 32^3 x 64, to 1e-10."""
    T, L, N, rep, m0 = 64, 32, 3, "fund", -0.4
    lat = _lattice(hr, inputs, torch, T, L, N, rep, 1.0, 0.0)
    fb = _pack_rhs(lat, inputs, torch, 1, T, L, 1, hr.F64)
    fx = lat.new_field(0, hr.F64)
    line = {"suite": "SU(3) fund 32^3x64: BiCGstab on Dhat vs CG on Dhat^+Dhat, to 1e-10", "m0": m0,
            "note": "BiCGstab residual is |b - Dhat x|/|b|; CG residual is that of the normal system"}
    # mixed solves: outer residuals in float-float, and in FP64 (_fp64_outer)
    for name, fn, inner, outer in (("cg_fp64", lat.cg_solve, hr.F64, hr.F64),
                                   ("cg_mixed_fp32", lat.cg_solve, hr.F32, hr.FF),
                                   ("cg_mixed_fp32_fp64_outer", lat.cg_solve, hr.F32, hr.F64),
                                   ("bicgstab_fp64", lat.bicgstab_solve, hr.F64, hr.F64),
                                   ("bicgstab_mixed_fp32", lat.bicgstab_solve, hr.F32, hr.FF),
                                   ("bicgstab_mixed_fp32_fp64_outer", lat.bicgstab_solve, hr.F32, hr.F64)):
        r = None
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = fn(fx, fb, 0, m0, 0.0, 1e-10, inner_prec=inner, check_every=10, raise_on_error=False,
                   outer_prec=outer)
            r["wall_s"] = round(time.perf_counter() - t0, 4)
        line[name] = {k: r[k] for k in ("wall_s", "iterations", "outer_steps", "true_residual", "status")}
    print(json.dumps(line), flush=True)
    lat.close()
    return line


def _suite_c3(hr, inputs, torch):
    """SU(3) sextet with clover, 32^3 x 64, 12 right-hand sides in one solve."""
    T, L, N, rep, m0, csw, nr = 64, 32, 3, "sym", -0.35, 1.0, 12
    lat = _lattice(hr, inputs, torch, T, L, N, rep, 1.0, csw)
    for prec, k in ((hr.F32, nr), (hr.F32, 1), (hr.F64, nr), (hr.F64, 1)):
        _warm(lat, prec, k, m0, csw)
    fb = _pack_rhs(lat, inputs, torch, 1, T, L, nr, hr.F64)
    fx = lat.new_field(0, hr.F64, nr)
    line = {"suite": "SU(3) sym csw=1 32^3x64 12 rhs CG to 1e-10", "m0": m0}
    r = _timed_cg(lat, fx, fb, m0, csw, hr.F32, nrhs=nr, reps=1)
    line["mixed_fp32_12rhs"] = {k: r[k] for k in ("wall_s", "iterations", "outer_steps", "true_residual", "status")}
    line["mixed_fp32_12rhs"]["seconds_per_rhs"] = round(r["wall_s"] / nr, 4)
    fb1 = lat.new_field(0, hr.F64)
    fx1 = lat.new_field(0, hr.F64)
    fbytes = lat.field_bytes(0, hr.F64, 1)
    fb1.copy_(fb[:fbytes])
    r1 = _timed_cg(lat, fx1, fb1, m0, csw, hr.F32, reps=1)
    line["mixed_fp32_1rhs"] = {k: r1[k] for k in ("wall_s", "iterations", "outer_steps", "true_residual", "status")}
    r64 = _timed_cg(lat, fx1, fb1, m0, csw, hr.F64, reps=1)
    line["fp64_1rhs"] = {k: r64[k] for k in ("wall_s", "iterations", "outer_steps", "true_residual", "status")}
    line["per_rhs_speedup_vs_single_mixed"] = round(r1["wall_s"] / (r["wall_s"] / nr), 2)
    line["per_rhs_speedup_vs_fp64"] = round(r64["wall_s"] / (r["wall_s"] / nr), 2)
    # the operator alone: 12-rhs Dhat vs 12 single-rhs Dhat, FP32
    fi = lat.new_field(0, hr.F32, nr)
    fo = lat.new_field(0, hr.F32, nr)
    st = torch.cuda.current_stream()
    fbytes32 = lat.field_bytes(0, hr.F32, 1)
    def _ev(fn, reps=5):
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            ts.append((e0, e1))
        torch.cuda.synchronize()
        return float(np.median([a_.elapsed_time(b_) for a_, b_ in ts]))
    t_multi = _ev(lambda: lat.dphi(fo, fi, 0, m0, csw, hr.F32, nr))
    t_single = _ev(lambda: [lat.dphi(fo[r * fbytes32:(r + 1) * fbytes32], fi[r * fbytes32:(r + 1) * fbytes32],
                                     0, m0, csw, hr.F32, 1) for r in range(nr)])
    line["dhat_ms_12rhs"] = round(t_multi, 3)
    line["dhat_ms_12x1rhs"] = round(t_single, 3)
    print(json.dumps(line), flush=True)
    lat.close()
    del fb, fx, fb1, fx1, fi, fo
    torch.cuda.empty_cache()
    return line


def _suite_c4(hr, inputs, torch):
    """64 lattices of mixed shape / N / representation, each solved to 1e-8."""
    shapes = inputs.batch_shapes(2, 64)
    lats, xs, bs = [], [], []
    for k, (T, L, N, rep) in enumerate(shapes):
        lt = _lattice(hr, inputs, torch, T, L, N, rep, 0.5, 0.0, seed=100 + k)
        lats.append(lt)
        bs.append(_pack_rhs(lt, inputs, torch, 200 + k, T, L, 1, hr.F64))
        xs.append(lt.new_field(0, hr.F64))
    batch = hr.Batch(lats)
    batch.cg_solve(xs, bs, 0, [-0.3] * 64, 1e-8, inner_prec=hr.F32)   # warm-up (tuning, graph)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, st = batch.cg_solve(xs, bs, 0, [-0.3] * 64, 1e-8, inner_prec=hr.F32)
    tb = time.perf_counter() - t0
    for k, lt in enumerate(lats):      # warm-up: tuning and graphs of the single-lattice path
        lt.cg_solve(xs[k], bs[k], 0, -0.3, 0.0, 1e-8, inner_prec=hr.F32, raise_on_error=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    per = []
    for k, lt in enumerate(lats):
        per.append(lt.cg_solve(xs[k], bs[k], 0, -0.3, 0.0, 1e-8, inner_prec=hr.F32, raise_on_error=False))
    tp = time.perf_counter() - t0
    vol = sum(T * L ** 3 for (T, L, N, rep) in shapes)
    its = sum(s_["iterations"] for s_ in st)
    line = {"suite": "64 lattices (8^4 .. 16^3x32, N 2..6, mixed reps) CG to 1e-8", "status": rc,
            "sites": vol, "batched_s": round(tb, 4), "per_lattice_s": round(tp, 4),
            "batched_speedup": round(tp / tb, 2),
            "max_true_residual": max(s_["true_residual"] for s_ in st),
            "iterations_sum": its, "site_iterations_per_s_batched": round(sum(
                (T * L ** 3 // 2) * s_["iterations"] for (T, L, N, rep), s_ in zip(shapes, st)) / tb, 1)}
    # model bytes of the operator applications (ideal reuse): two FP32 Dhat per inner
    # iteration, two FP64 Dhat per outer true residual; their rate against the batched time
    b_in = sum(2 * s_["iterations"] * bytes_per_even_site(N, rep, 4) * (T * L ** 3 // 2)
               for (T, L, N, rep), s_ in zip(shapes, st))
    b_out = sum(2 * s_["outer_steps"] * bytes_per_even_site(N, rep, 8) * (T * L ** 3 // 2)
                for (T, L, N, rep), s_ in zip(shapes, st))
    line["operator_model_gb"] = {"fp32_inner": round(b_in / 1e9, 2), "fp64_outer": round(b_out / 1e9, 2)}
    line["operator_model_gbs_batched"] = round((b_in + b_out) / tb / 1e9, 1)
    print(json.dumps(line), flush=True)
    batch.close()
    return line


# ------------------------------------------------ the other workloads --
# Measured inside the default bench run so that they carry its clock record;
# every number is an operator or a whole solve on the GPU after a warm-up.
def _ev_ms(torch, fn, reps, flush=None):
    st = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.sum()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        ts.append((e0, e1))
    torch.cuda.synchronize()
    return float(np.median([a.elapsed_time(b) for a, b in ts]))


def _cg_rec(res):
    rec = {"seconds": round(res["wall_s"], 4), "iterations": res["iterations"], "outer_steps": res["outer_steps"],
           "true_residual": res["true_residual"], "status": res["status"]}
    if res.get("outer"):
        rec["outer_residuals"] = res["outer"]
    return rec


def _rel_diff(torch, lat, f_lo, prec, f64, nrhs=1):
    """|D_prec psi - D_64 psi| / |D_64 psi| over the even sites (the FP64 operator is
    the one held to 1e-13 of the oracle by the parity tests)."""
    a = torch.zeros((nrhs, lat.V, 4, lat.d, 2), dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    lat.unpack(a, f_lo, 0, prec, nrhs)
    lat.unpack(b, f64, 0, 0, nrhs)
    lat.synchronize()
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def bench_adj_asym_24c48(hr, inputs, torch, flush, peak):
    """SU(2) adjoint and SU(4) antisymmetric, 24^3 x 48, m0 = -0.3: Dhat GB/s per
    precision, and CG to 1e-10 (plain FP64, FP32 and FP16 inner solves)."""
    T, L, m0 = 48, 24, -0.3
    out = {}
    for N, rep in ((2, "adj"), (4, "asym")):
        lat = _lattice(hr, inputs, torch, T, L, N, rep, 1.0, 0.0)
        rec = {"lattice": "24^3x48", "d_R": lat.d, "m0": m0}
        f64 = _pack_rhs(lat, inputs, torch, 1, T, L, 1, hr.F64)
        o64 = lat.new_field(0, hr.F64)
        lat.dphi(o64, f64, 0, m0, 0.0, hr.F64)
        for prec, w in ((hr.F32, 4), (hr.F16, 2)):
            fi = _pack_rhs(lat, inputs, torch, 1, T, L, 1, prec)
            fo = lat.new_field(0, prec)
            lat.dphi(fo, fi, 0, m0, 0.0, prec)
            ms = _ev_ms(torch, lambda: lat.dphi(fo, fi, 0, m0, 0.0, prec), 20, flush)
            gbs = bytes_per_even_site(N, rep, w) * lat.Vh / ms / 1e6
            rec["dhat_" + ("fp32" if prec == hr.F32 else "fp16")] = {
                "ms": round(ms, 4), "GBs": round(gbs, 1), "frac_of_measured_hbm": round(gbs / peak, 3),
                "shape": lat.tuned_shape(prec), "rel_err_vs_fp64": _rel_diff(torch, lat, fo, prec, o64)}
        fx = lat.new_field(0, hr.F64)
        cg = {}
        for name, inner, itol in (("fp64", hr.F64, 0.0), ("mixed_fp32", hr.F32, 0.0),
                                  ("mixed_fp16", hr.F16, 3e-3)):
            cg[name] = _cg_rec(_timed_cg(lat, fx, f64, m0, 0.0, inner, inner_tol=itol))
            if name != "fp64":
                cg[name]["speedup_vs_fp64"] = round(cg["fp64"]["seconds"] / cg[name]["seconds"], 2)
        cg["mixed_fp16"]["inner_tol"] = 3e-3
        rec["cg"] = cg
        out[f"SU({N}) {rep}"] = rec
        lat.close()
        torch.cuda.empty_cache()
    return out


def bench_sextet_clover_12rhs(hr, inputs, torch, flush, peak, nr=12):
    """SU(3) sextet with clover (csw = 1), 32^3 x 64, m0 = -0.35, 12 right-hand
    sides: the 12-rhs Dhat (one link and clover read per site for all rhs) in
    FP32 and FP16, 12 single-rhs Dhat for comparison, and the 12-rhs CG per rhs
    against a plain FP64 single-rhs solve."""
    T, L, N, rep, m0, csw = 64, 32, 3, "sym", -0.35, 1.0
    lat = _lattice(hr, inputs, torch, T, L, N, rep, 1.0, csw)
    d = lat.d
    rec = {"lattice": "32^3x64", "d_R": d, "m0": m0, "csw": csw, "nrhs": nr}
    fb = _pack_rhs(lat, inputs, torch, 1, T, L, nr, hr.F64)
    o64 = lat.new_field(0, hr.F64, nr)
    lat.dphi(o64, fb, 0, m0, csw, hr.F64, nr)
    flops = nr * 2 * (128 * d * d + 56 * d + 64 * d * d - 8 * d) * lat.Vh
    for prec, w in ((hr.F32, 4), (hr.F16, 2)):
        fi = _pack_rhs(lat, inputs, torch, 1, T, L, nr, prec)
        fo = lat.new_field(0, prec, nr)
        lat.dphi(fo, fi, 0, m0, csw, prec, nr)
        ms = _ev_ms(torch, lambda: lat.dphi(fo, fi, 0, m0, csw, prec, nr), 10, flush)
        # links once per site for all rhs, A^{-1} and A once each, 5 spinor passes per rhs
        scale_b = 5 * 4 * nr if w == 2 else 0
        model = (16 * 2 * d * d * w + 2 * 8 * d * d * 4 + nr * 5 * 8 * d * w + scale_b) * lat.Vh
        gbs = model / ms / 1e6
        key = "fp32" if prec == hr.F32 else "fp16"
        rec["dhat_12rhs_" + key] = {"ms": round(ms, 3), "model_bytes": int(model), "GBs": round(gbs, 1),
                                    "frac_of_measured_hbm": round(gbs / peak, 3),
                                    "TFLOPs": round(flops / ms / 1e9, 2),
                                    "shape": lat.tuned_shape(prec, nrhs=nr, clover=True),
                                    "rel_err_vs_fp64": _rel_diff(torch, lat, fo, prec, o64, nr)}
        if prec == hr.F32:
            fb1 = lat.field_bytes(0, prec, 1)
            lat.dphi(fo[:fb1], fi[:fb1], 0, m0, csw, prec, 1)
            ms1 = _ev_ms(torch, lambda: [lat.dphi(fo[r * fb1:(r + 1) * fb1], fi[r * fb1:(r + 1) * fb1], 0, m0, csw,
                                                  prec, 1) for r in range(nr)], 5, flush)
            rec["dhat_12x1rhs_fp32_ms"] = round(ms1, 3)
        del fi, fo
    del o64
    for prec, k in ((hr.F32, nr), (hr.F16, nr), (hr.F64, 1), (hr.FF, nr), (hr.F64, nr)):
        _warm(lat, prec, k, m0, csw)
    fx = lat.new_field(0, hr.F64, nr)
    cg = {}
    r32 = _timed_cg(lat, fx, fb, m0, csw, hr.F32, nrhs=nr, reps=1)
    cg["mixed_fp32_12rhs"] = dict(_cg_rec(r32), seconds_per_rhs=round(r32["wall_s"] / nr, 4))
    r16 = _timed_cg(lat, fx, fb, m0, csw, hr.F16, nrhs=nr, inner_tol=3e-3, reps=1)
    cg["mixed_fp16_12rhs"] = dict(_cg_rec(r16), seconds_per_rhs=round(r16["wall_s"] / nr, 4), inner_tol=3e-3)
    r32d = _timed_cg(lat, fx, fb, m0, csw, hr.F32, nrhs=nr, reps=1, outer=hr.F64)
    cg["mixed_fp32_12rhs_fp64_outer"] = dict(_cg_rec(r32d), seconds_per_rhs=round(r32d["wall_s"] / nr, 4))
    fb1 = lat.new_field(0, hr.F64)
    fx1 = lat.new_field(0, hr.F64)
    fb1.copy_(fb[:lat.field_bytes(0, hr.F64, 1)])
    r64 = _timed_cg(lat, fx1, fb1, m0, csw, hr.F64, reps=1)
    cg["fp64_1rhs"] = _cg_rec(r64)
    for k_ in ("mixed_fp32_12rhs", "mixed_fp16_12rhs"):
        cg[k_]["per_rhs_speedup_vs_fp64"] = round(r64["wall_s"] / cg[k_]["seconds_per_rhs"], 2)
    rec["cg"] = cg
    lat.close()
    del fb, fx, fb1, fx1
    torch.cuda.empty_cache()
    return rec


def bench_64_lattices(hr, inputs, torch, nlat=64):
    """64 lattices (8^4 ... 16^3 x 32, N = 2..6, mixed representations), m0 = -0.3:
    one batched FP32 Dhat against 64 single-lattice launches (aggregate sites/s),
    and the batched CG to 1e-8 against 64 single-lattice solves."""
    shapes = inputs.batch_shapes(2, nlat)
    lats, xs, bs, fi, fo = [], [], [], [], []
    for k, (T, L, N, rep) in enumerate(shapes):
        lt = _lattice(hr, inputs, torch, T, L, N, rep, 0.5, 0.0, seed=100 + k)
        lats.append(lt)
        bs.append(_pack_rhs(lt, inputs, torch, 200 + k, T, L, 1, hr.F64))
        xs.append(lt.new_field(0, hr.F64))
        fi.append(_pack_rhs(lt, inputs, torch, 200 + k, T, L, 1, hr.F32))
        fo.append(lt.new_field(0, hr.F32))
    batch = hr.Batch(lats)
    m0s = [-0.3] * nlat
    sites = sum(lt.Vh for lt in lats)
    batch.dphi(fo, fi, 0, m0s, hr.F32)
    for k, lt in enumerate(lats):
        lt.dphi(fo[k], fi[k], 0, -0.3, 0.0, hr.F32)
    tb = _ev_ms(torch, lambda: batch.dphi(fo, fi, 0, m0s, hr.F32), 10)
    tp = _ev_ms(torch, lambda: [lt.dphi(fo[k], fi[k], 0, -0.3, 0.0, hr.F32) for k, lt in enumerate(lats)], 10)
    rec = {"lattices": nlat, "even_sites": int(sites),
           "dhat_fp32": {"batched_ms": round(tb, 4), "per_lattice_ms": round(tp, 4),
                         "batched_sites_per_s": round(sites / tb * 1e3, 1),
                         "per_lattice_sites_per_s": round(sites / tp * 1e3, 1),
                         "speedup": round(tp / tb, 2)}}
    batch.cg_solve(xs, bs, 0, m0s, 1e-8, inner_prec=hr.F32)     # warm-up: tuning, graph capture
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, st = batch.cg_solve(xs, bs, 0, m0s, 1e-8, inner_prec=hr.F32)
    t_b = time.perf_counter() - t0
    for k, lt in enumerate(lats):
        lt.cg_solve(xs[k], bs[k], 0, -0.3, 0.0, 1e-8, inner_prec=hr.F32, raise_on_error=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    per = [lt.cg_solve(xs[k], bs[k], 0, -0.3, 0.0, 1e-8, inner_prec=hr.F32, raise_on_error=False)
           for k, lt in enumerate(lats)]
    t_p = time.perf_counter() - t0
    rec["cg_1e-8"] = {"status": rc, "batched_s": round(t_b, 4), "per_lattice_s": round(t_p, 4),
                      "speedup": round(t_p / t_b, 2), "outer_residuals": "ff",
                      "max_true_residual_batched": max(s_["true_residual"] for s_ in st),
                      "max_true_residual_per_lattice": max(r["true_residual"] for r in per)}
    # the batched solve with FP64 outer residuals, for comparison
    batch.cg_solve(xs, bs, 0, m0s, 1e-8, inner_prec=hr.F32, outer_prec=hr.F64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc64, st64 = batch.cg_solve(xs, bs, 0, m0s, 1e-8, inner_prec=hr.F32, outer_prec=hr.F64)
    rec["cg_1e-8_fp64_outer"] = {"status": rc64, "batched_s": round(time.perf_counter() - t0, 4),
                                 "max_true_residual_batched": max(s_["true_residual"] for s_ in st64)}
    batch.close()
    for lt in lats:
        lt.close()
    torch.cuda.empty_cache()
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cg", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the adjoint / antisymmetric, 12-rhs sextet and 64-lattice measurements")
    ap.add_argument("--suite", default="", help="comma list of c2,bicg,c3,c4,largen,larged,blas: measure those workloads instead")
    ap.add_argument("--shape", default="", help="pin the hop shape 'regs,G,block' (profiling runs only)")
    ap.add_argument("--prec", default="f32", choices=["f32", "f16"], help="timed Dhat precision (profiling runs only)")
    ap.add_argument("--T", type=int, default=WORKLOAD["T"], help="time extent (profiling runs only)")
    ap.add_argument("--L", type=int, default=WORKLOAD["L"], help="space extent (profiling runs only)")
    ap.add_argument("--one-dhat", default="", metavar="N,REP,T,L,PREC,SHAPE[,CSW[,NRHS]]",
                    help="profiling case: build one lattice (PREC f64/f32/f16), pin the launch shape "
                         "SHAPE = G:block:regs:mrhs:rows and apply Dhat (clover coefficient CSW, NRHS "
                         "right-hand sides) three times, nothing else")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    if args.suite:
        run_suite(args)
        return
    if args.one_dhat:
        run_one_dhat(args.one_dhat)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_2405_19294_gb300 import hr, inputs

    wl = WORKLOAD
    T, L, N, rep = args.T, args.L, wl["N"], wl["rep"]
    lat = hr.Lattice(T, L, N, rep)
    a = torch.from_numpy(inputs.algebra_coefficients(0, T, L, N)).cuda()
    U = torch.empty((lat.V, 4, N, N, 2), dtype=torch.float64, device="cuda")
    lat.links_from_algebra(U, a, wl["eps"], True)
    lat.represent_links(U, True, wl["csw"])
    del a
    psi = inputs.gaussian_spinor(1, T, L, lat.d)
    src_host = torch.from_numpy(np.stack([psi.real, psi.imag], -1)).pin_memory()
    del psi
    src = src_host.cuda()
    stream = torch.cuda.current_stream()
    TP = hr.F32 if args.prec == "f32" else hr.F16   # timed precision
    if args.shape:
        regs, g, bs = (int(v) for v in args.shape.split(","))
        lat.set_shape(TP, (g, bs, regs))
    fin = {p: lat.new_field(hr.EVEN, p) for p in (hr.F64, hr.F32, hr.F16, hr.FF)}
    fout = {p: lat.new_field(hr.EVEN, p) for p in (hr.F64, hr.F32, hr.F16, hr.FF)}
    for p in (hr.F64, hr.F32, hr.F16, hr.FF):
        lat.pack(fin[p], src, hr.EVEN, p)
    flush = torch.ones(128 << 20, dtype=torch.float32, device="cuda")   # 512 MiB, read to evict L2
    m0, csw = wl["m0"], wl["csw"]

    def timed(prec, steps):
        ts = []
        for _ in range(steps):
            flush.sum()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.dphi(fout[prec], fin[prec], hr.EVEN, m0, csw, prec)
            e1.record(stream)
            ts.append((e0, e1))
        torch.cuda.synchronize()
        return [x.elapsed_time(y) for x, y in ts]

    clocks = ClockSampler(local)   # runs through warm-up, timed region and the FP64 leg
    for _ in range(args.warmup):
        lat.dphi(fout[TP], fin[TP], hr.EVEN, m0, csw, TP)
    lat.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    ms32 = timed(TP, args.steps)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - t_wall
    lat.synchronize()
    ms_step = job_timing(float(np.mean(ms32)), world, dist, device="cuda")
    sites = lat.Vh
    b32 = bytes_per_even_site(N, rep, 4 if TP == hr.F32 else 2) * sites
    gbs = job_value(b32, world, ms_step)

    # FP64 Dhat (FP64-ALU bound on this part)
    for _ in range(3):
        lat.dphi(fout[hr.F64], fin[hr.F64], hr.EVEN, m0, csw, hr.F64)
    ms64 = float(np.mean(timed(hr.F64, max(3, args.steps // 4))))
    # the same FP64-accurate Dhat in float-float arithmetic (the mixed solvers' outer residuals)
    for _ in range(3):
        lat.dphi(fout[hr.FF], fin[hr.FF], hr.EVEN, m0, csw, hr.FF)
    msff = float(np.mean(timed(hr.FF, max(3, args.steps // 4))))
    # FP16 Dhat (per-site scaled FP16 storage, FP32 arithmetic), unless it is the timed precision
    peaks, kind = measured_peaks()
    fp16 = None
    if TP != hr.F16:
        for _ in range(3):
            lat.dphi(fout[hr.F16], fin[hr.F16], hr.EVEN, m0, csw, hr.F16)
        ms16 = float(np.mean(timed(hr.F16, args.steps)))
        g16 = bytes_per_even_site(N, rep, 2) * sites / (ms16 * 1e-3) / 1e9
        fp16 = {"ms_per_step": round(ms16, 4), "GBs": round(g16, 2), "frac_of_measured_hbm": round(g16 / peaks["hbm_gbs"], 4),
                "shape": lat.tuned_shape(hr.F16),
                "rel_err_vs_fp64": _rel_diff(torch, lat, fout[hr.F16], hr.F16, fout[hr.F64])}
    b64 = bytes_per_even_site(N, rep, 8) * sites
    fl = flops_per_even_site(N, rep) * sites

    # end to end through the C ABI with host buffers: every step copies the
    # canonical FP64 source from page-locked host memory to the device
    # (DMA), packs it, applies Dhat, unpacks and copies the result back to
    # page-locked host memory.  Steps are pipelined the way a serving loop
    # would run them: the copies go on their own streams with double-buffered
    # device staging, so the host-to-device copy of step k+1 and the
    # device-to-host copy of step k-1 overlap step k's kernels (the host link
    # is full duplex); the kernels of successive steps stay in order on the
    # lattice's stream.  (The library can also read / write page-locked host
    # memory in place -- only the parity's sites cross the host link -- but
    # per-thread scattered reads over the host link measured slower than one
    # bulk DMA copy of the whole field for this layout.)
    s_h2d, s_d2h = torch.cuda.Stream(), torch.cuda.Stream()
    out_host = [torch.empty_like(src_host).pin_memory() for _ in range(2)]
    dev_in = [torch.empty_like(src) for _ in range(2)]
    dev_out = [torch.zeros_like(src) for _ in range(2)]
    ev = lambda: torch.cuda.Event()
    packed = [ev(), ev()]      # dev_in[b] consumed by pack
    landed = [ev(), ev()]      # dev_in[b] filled
    done = [ev(), ev()]        # dev_out[b] filled
    drained = [ev(), ev()]     # dev_out[b] copied out
    for b in range(2):
        packed[b].record(stream)
        drained[b].record(stream)

    def e2e_run(nsteps):
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        s_h2d.wait_stream(stream)
        s_d2h.wait_stream(stream)
        for k in range(nsteps):
            b = k % 2
            with torch.cuda.stream(s_h2d):
                s_h2d.wait_event(packed[b])
                dev_in[b].copy_(src_host, non_blocking=True)
                landed[b].record(s_h2d)
            stream.wait_event(landed[b])
            lat.pack(fin[hr.F32], dev_in[b], hr.EVEN, hr.F32)
            packed[b].record(stream)
            lat.dphi(fout[hr.F32], fin[hr.F32], hr.EVEN, m0, csw, hr.F32)
            stream.wait_event(drained[b])
            lat.unpack(dev_out[b], fout[hr.F32], hr.EVEN, hr.F32)
            done[b].record(stream)
            with torch.cuda.stream(s_d2h):
                s_d2h.wait_event(done[b])
                out_host[b].copy_(dev_out[b], non_blocking=True)
                drained[b].record(s_d2h)
        stream.wait_stream(s_h2d)
        stream.wait_stream(s_d2h)
        t1.record(stream)
        t1.synchronize()
        return t0.elapsed_time(t1) / nsteps

    e2e_run(args.warmup)
    e2e = e2e_run(args.steps)
    out_host = out_host[(args.steps - 1) % 2]
    h2d = src_host.numel() * 8
    d2h = out_host.numel() * 8

    # CG time-to-1e-10
    cg = None
    if not args.no_cg:
        cg = {}
        fb = lat.new_field(hr.EVEN, hr.F64)
        fx = lat.new_field(hr.EVEN, hr.F64)
        lat.pack(fb, src, hr.EVEN, hr.F64)
        # mixed solves: outer residuals in float-float (the default) and in FP64
        for name, inner, outer in (("fp64", hr.F64, hr.F64), ("mixed_fp32", hr.F32, hr.FF),
                                   ("mixed_fp16", hr.F16, hr.FF), ("mixed_fp32_fp64_outer", hr.F32, hr.F64),
                                   ("mixed_fp16_fp64_outer", hr.F16, hr.F64)):
            res = None
            for rep_ in range(2):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                res = lat.cg_solve(fx, fb, hr.EVEN, m0, csw, 1e-10, inner_prec=inner, check_every=20,
                                   raise_on_error=False, outer_prec=outer)
                res["wall_s"] = time.perf_counter() - t0
            cg[name] = {"seconds": round(res["wall_s"], 4), "iterations": res["iterations"],
                        "outer_steps": res["outer_steps"], "true_residual": res["true_residual"],
                        "status": res["status"]}
            if inner != hr.F64:
                cg[name]["outer_residuals"] = "ff" if outer == hr.FF else "fp64"
        if cg["fp64"]["seconds"] > 0:
            for k in ("mixed_fp32", "mixed_fp16", "mixed_fp32_fp64_outer", "mixed_fp16_fp64_outer"):
                cg[k]["speedup_vs_fp64"] = round(cg["fp64"]["seconds"] / cg[k]["seconds"], 2)

    # the other workloads (SU(2) adj / SU(4) asym 24^3x48, the 12-rhs sextet with clover,
    # 64 small lattices), inside the same clock record; keys c2, c3, c4
    configs = None
    if not args.no_configs:
        configs = {"c2": bench_adj_asym_24c48(hr, inputs, torch, flush, peaks["hbm_gbs"]),
                   "c3": bench_sextet_clover_12rhs(hr, inputs, torch, flush, peaks["hbm_gbs"]),
                   "c4": bench_64_lattices(hr, inputs, torch)}
    clk = clocks.stop()
    traffic = ncu_traffic(f"dram_bytes_per_even_site_{args.prec}")
    roof = {"bound": "hbm", "achieved": round(gbs / world, 2), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(gbs / world / peaks["hbm_gbs"], 4), "peak_kind": kind,
            "traffic": (round(traffic * sites / 2) if traffic else None),
            "kernel": f"hop_kernel<3,false,{TP}>, tuned shape (G, block, regs, mrhs, rows) = {lat.tuned_shape(TP)}, "
                      "2 launches per Dhat"}
    line = {"metric": METRIC, "value": round(gbs, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
            "config": {"workload": "SU(3) fund 32^3x64 Dhat even (even-odd Schur), eps=1.0 reunitarised, "
                                   "m0=-0.4", "T": T, "L": L, "N": N, "rep": rep,
                       "l2": "flushed between steps (512 MiB read)", "parallelism": f"replicas x{world}",
                       "seeds": {"links": 0, "source": 1}},
            "roofline": roof,
            "gpu_launches": 2 * args.steps,
            "e2e": {"value": round(world * b32 / (e2e * 1e-3) / 1e9, 2), "unit": "GB/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e, 3),
                    "mode": "steps pipelined: host-to-device of step k+1 and device-to-host of step k-1 "
                            "overlap step k's kernels (copy streams, double-buffered staging)"},
            "fp64": {"ms_per_step": round(ms64, 4), "gbs": round(b64 / (ms64 * 1e-3) / 1e9, 2),
                     "tflops": round(fl / (ms64 * 1e-3) / 1e12, 3), "bound": "alu (FP64)"},
            "ff": {"ms_per_step": round(msff, 4), "gbs": round(b64 / (msff * 1e-3) / 1e9, 2),
                   "frac_of_measured_hbm": round(b64 / (msff * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
                   "speedup_vs_fp64": round(ms64 / msff, 2), "shape": lat.tuned_shape(hr.FF),
                   "rel_err_vs_fp64": _rel_diff(torch, lat, fout[hr.FF], hr.FF, fout[hr.F64]),
                   "arithmetic": "float-float (FP32 pairs, 48 bits), FP64 bytes"},
            "fp16": fp16, "cg": cg, "configs": configs, "clocks": clk, "wall_timed_s": round(wall, 3)}
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline_leg()
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
