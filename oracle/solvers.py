"""Solver loops of the oracle, in plain numpy FP64 (test infrastructure only).

The paper's outer solver is a flexible BiCGStab in double precision with a
lower-precision solver as its preconditioner (Sec. 2); neither paper it cites
for the algorithm is part of this project, so the loop below is the standard
right-preconditioned BiCGStab of van der Vorst with a preconditioner that may
change between applications:

    r = b - M x, rhat = r, rho0 = alpha = omega = 1, v = p = 0
    repeat:
        rho = <rhat, r>;  beta = (rho / rho0) (alpha / omega)
        p = r + beta (p - omega v);  phat = K^-1 p;  v = M phat
        alpha = rho / <rhat, v>;  s = r - alpha v;  shat = K^-1 s;  t = M shat
        omega = <t, s> / <t, t>;  x += alpha phat + omega shat;  r = s - omega t
        rho0 = rho
    until |r| <= tol |b|, then recompute r = b - M x; restart if it fails.

With K = 1 this is plain BiCGStab.  <a, b> = sum conj(a) b.
"""
from __future__ import annotations

import numpy as np


class SolveResult:
    def __init__(self, x, iters, converged, true_rel_resid, status):
        self.x = x
        self.iters = iters
        self.converged = converged
        self.true_rel_resid = true_rel_resid
        self.status = status

    def __repr__(self):
        return (f"SolveResult(iters={self.iters}, converged={self.converged}, "
                f"true_rel_resid={self.true_rel_resid:.3e}, status={self.status!r})")


def _dot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def _norm(a):
    return float(np.sqrt(np.real(_dot(a, a))))


def bicgstab(M, b, x0=None, tol=1e-12, maxiter=10000, precond=None, max_restarts=5):
    """Flexible right-preconditioned BiCGStab in FP64.

    M, precond: callables on arrays shaped like b.  precond=None means K = 1.
    """
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    K = precond if precond is not None else (lambda u: u)
    bnorm = _norm(b)
    if bnorm == 0.0:
        return SolveResult(np.zeros_like(b), 0, True, 0.0, "ok")
    iters = 0
    status = "not_converged"
    for _ in range(max_restarts + 1):
        r = b - M(x)
        if _norm(r) <= tol * bnorm:
            status = "ok"
            break
        rhat = r.copy()
        rho0 = alpha = omega = 1.0 + 0j
        v = np.zeros_like(b)
        p = np.zeros_like(b)
        while iters < maxiter:
            rho = _dot(rhat, r)
            if rho == 0:
                status = "breakdown"
                break
            beta = (rho / rho0) * (alpha / omega)
            p = r + beta * (p - omega * v)
            phat = K(p)
            v = M(phat)
            rv = _dot(rhat, v)
            if rv == 0:
                status = "breakdown"
                break
            alpha = rho / rv
            s = r - alpha * v
            shat = K(s)
            t = M(shat)
            tt = np.real(_dot(t, t))
            omega = _dot(t, s) / tt if tt > 0 else 0.0
            x = x + alpha * phat + omega * shat
            r = s - omega * t
            rho0 = rho
            iters += 1
            if _norm(r) <= tol * bnorm:
                break
            if omega == 0:
                status = "breakdown"
                break
        true_r = _norm(b - M(x)) / bnorm
        if true_r <= tol:
            status = "ok"
            break
        if status == "breakdown" or iters >= maxiter:
            break
    true_r = _norm(b - M(x)) / bnorm
    return SolveResult(x, iters, true_r <= tol, true_r,
                       "ok" if true_r <= tol else status)


def action_and_force(op, phi, tol=1e-14, maxiter=20000, hop_only=False):
    """S = phi^+ (M^+ M)^-1 phi and its force F per link.

    Y solves M^+ Y = phi, X solves M X = Y, S = |Y|^2 (= phi^+ X).
    Returns (S, F, X, Y).
    """
    from . import force
    ry = bicgstab(op.Mdag, phi, tol=tol, maxiter=maxiter)
    rx = bicgstab(op.M, ry.x, tol=tol, maxiter=maxiter)
    Y, X = ry.x, rx.x
    S = float(np.real(_dot(Y, Y)))
    F = force(op.dims, op.tbc, op.kappa, op.csw, op.U, X, Y, hop_only=hop_only)
    return S, F, X, Y
