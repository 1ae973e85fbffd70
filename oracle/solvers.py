"""Krylov solvers for the oracle: conjugate gradient and BiCGstab.

The paper (Sec. 3.3) lists the conjugate gradient among the GPU-ported
inverters without spelling it out.  This is textbook Hestenes-Stiefel CG on a
Hermitian positive-definite operator M, started from x = 0, with the stopping
rule: stop when the recursively updated residual satisfies |r| <= tol |b|,
then recompute the true residual b - M x; if that is still above tol |b|,
restart from it (r = p = b - M x) and continue.

For the Wilson operator it is run on the normal equations M = D^dagger D
(full lattice) or M = Dhat^dagger Dhat (even-odd Schur complement).

The paper (Sec. 3.3) also ports the stabilised bi-conjugate gradient of van
der Vorst (1992), which solves the non-Hermitian system Dhat x = b directly.
``bicgstab`` follows that algorithm's steps (shadow residual r^ = r0, one
BiCG step with coefficient alpha, then a minimal-residual step omega), with
the same stopping rule as ``cg`` (recursive residual, then the true residual,
restart from it if needed).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np


def vdot(a: np.ndarray, b: np.ndarray) -> complex:
    """<a, b> = sum conj(a) b over all components."""
    return np.vdot(a.ravel(), b.ravel())


def cg(apply_M, b: np.ndarray, tol: float, maxit: int = 100000):
    """Solve M x = b.  Returns (x, iterations, true relative residual)."""
    bnorm = np.sqrt(vdot(b, b).real)
    x = np.zeros_like(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    r = b.copy()
    p = r.copy()
    rr = vdot(r, r).real
    it = 0
    while it < maxit:
        Ap = apply_M(p)
        pAp = vdot(p, Ap).real
        alpha = rr / pAp
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = vdot(r, r).real
        it += 1
        if np.sqrt(rr_new) <= tol * bnorm:
            r_true = b - apply_M(x)
            rt = np.sqrt(vdot(r_true, r_true).real)
            if rt <= tol * bnorm:
                return x, it, rt / bnorm
            r = r_true
            p = r.copy()
            rr = vdot(r, r).real
            continue
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
    r_true = b - apply_M(x)
    return x, it, np.sqrt(vdot(r_true, r_true).real) / bnorm


def solve_wilson_full(op, b: np.ndarray, tol: float, maxit: int = 100000):
    """x = D^{-1} b on the full lattice via CG on D^dagger D: x = (D^+D)^{-1} D^+ b."""
    rhs = op.apply(b, dagger=True)
    x, it, _ = cg(lambda v: op.apply(op.apply(v), dagger=True), rhs, tol, maxit)
    return x, it


def solve_wilson_eo(op, b: np.ndarray, tol: float, maxit: int = 100000):
    """x = D^{-1} b through the even-odd Schur complement on the even sites.

        b'_e = b_e - D_eo A_oo^{-1} b_o
        Dhat_e x_e = b'_e     solved as x_e = (Dhat^+ Dhat)^{-1} Dhat^+ b'_e
        x_o = A_oo^{-1} (b_o - D_oe x_e)
    """
    from .dirac import hopping
    g = op.geom
    ev = g.parity == 0
    od = ~ev
    even_sites, odd_sites = np.nonzero(ev)[0], np.nonzero(od)[0]
    b_o = np.where(od[:, None, None], b, 0.0)
    t = np.zeros_like(b)
    t[odd_sites] = op.apply_A(b_o[odd_sites], odd_sites, inverse=True)
    bp = np.where(ev[:, None, None], b, 0.0)
    bp[even_sites] -= -0.5 * hopping(op.UR, t, g, 1, even_sites)
    rhs = op.apply_schur(bp, 0, dagger=True)
    xe, it, _ = cg(lambda v: op.apply_schur(op.apply_schur(v, 0), 0, dagger=True), rhs, tol,
                   maxit)
    x = xe.copy()
    u = np.zeros_like(b)
    u[odd_sites] = b[odd_sites] - (-0.5 * hopping(op.UR, xe, g, 1, odd_sites))
    x[odd_sites] = op.apply_A(u[odd_sites], odd_sites, inverse=True)
    return x, it


def bicgstab(apply_A, b: np.ndarray, tol: float, maxit: int = 100000):
    """Solve A x = b (A need not be Hermitian).  Returns (x, iterations, true relative residual).

    Each iteration: rho = <r^, r>; beta = (rho / rho_old)(alpha / omega);
    p = r + beta (p - omega v); v = A p; alpha = rho / <r^, v>; s = r - alpha v;
    t = A s; omega = <t, s> / <t, t>; x += alpha p + omega s; r = s - omega t.
    """
    bnorm = np.sqrt(vdot(b, b).real)
    x = np.zeros_like(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    r = b.copy()
    it = 0
    while it < maxit:
        rhat = r.copy()
        rho_old = alpha = omega = 1.0 + 0.0j
        v = np.zeros_like(b)
        p = np.zeros_like(b)
        restart = False
        while it < maxit:
            rho = vdot(rhat, r)
            beta = (rho / rho_old) * (alpha / omega)
            p = r + beta * (p - omega * v)
            v = apply_A(p)
            alpha = rho / vdot(rhat, v)
            s = r - alpha * v
            t = apply_A(s)
            tt = vdot(t, t).real
            omega = vdot(t, s) / tt if tt > 0 else 0.0
            x = x + alpha * p + omega * s
            r = s - omega * t
            rho_old = rho
            it += 1
            if np.sqrt(vdot(r, r).real) <= tol * bnorm:
                r_true = b - apply_A(x)
                rt = np.sqrt(vdot(r_true, r_true).real)
                if rt <= tol * bnorm:
                    return x, it, rt / bnorm
                r = r_true
                restart = True
                break
        if not restart:
            break
    r_true = b - apply_A(x)
    return x, it, np.sqrt(vdot(r_true, r_true).real) / bnorm
