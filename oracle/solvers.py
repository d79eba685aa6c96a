"""Preconditioned Krylov solvers (oracle; test infrastructure only).

The paper (Sec. 3.1) studies three iterative solvers for the preconditioned systems:
Richardson Minimal Residual (Canuto et al. 1995), Conjugate Gradient (Press et al.
1992) and GMRES (Saad & Schultz 1986), all started from a zero initial guess unless a
warm start is given (Sec. 3.1, last paragraph: previous solution as initial guess).
The paper does not print the algorithms; these are the textbook forms, with the readings
listed below.

Common conventions (identical in the CUDA library so that iterates can be compared):

* vectors are numpy arrays of any shape; (u, v) is the plain Euclidean inner product over
  all entries and ||v|| its norm;
* relres = ||b - A x|| / ||b||; a solver stops as soon as its monitored relres <= tol, or
  after ``maxit`` operator applications inside the loop;
* CG is the preconditioned Hestenes--Stiefel recurrence;  for the pressure system both A
  and M are negative semi-definite and the recurrence is the same as on (-A, -M);
* GMRES is right-preconditioned (A M y = r0, x = x0 + M y), Arnoldi by modified
  Gram--Schmidt, Givens rotations, restarted every ``restart`` iterations; its monitored
  residual is the Givens estimate |g_{j+1}|;
* the status is decided by the monitored residual (recurrence residual for CG and RMR,
  Givens estimate for GMRES), and the true residual ||b - A x||/||b|| of the returned
  iterate is reported beside it: near the rounding floor of the operator
  (~ eps * ||A|| ||x|| / ||b||) the two differ;
* RMR: z = M r, w = A z, alpha = (r, w)/(w, w), x += alpha z, r -= alpha w (the minimal
  residual choice of the Richardson step length).

Status strings: "converged", "max_iter", "breakdown", "nonfinite", "diverged" (RMR only:
relres grew above 1e3 times the best value seen; the paper observes RMR diverging at high
density ratios, Sec. 3.1 and 3.2.  CG's residual 2-norm is not monotone -- only the energy
norm of its error is -- so a residual-growth test would misfire near the rounding floor;
GMRES's residual estimate is monotone).
"""

from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np


@dataclass
class SolveResult:
    x: np.ndarray
    iters: int
    status: str
    history: list = field(default_factory=list)
    relres_true: float = float("nan")


def _dot(u, v) -> float:
    return float(np.dot(u.ravel(), v.ravel()))


def _norm(u) -> float:
    return float(np.sqrt(_dot(u, u)))


DIVERGE_FACTOR = 1e3


def _finish(A, b, x, bnorm, it, status, hist) -> SolveResult:
    rt = _norm(b - A(x)) / bnorm if bnorm > 0 else 0.0
    return SolveResult(x=x, iters=it, status=status, history=hist, relres_true=rt)


def cg(A, M, b, x0=None, tol=1e-10, maxit=500) -> SolveResult:
    """Preconditioned conjugate gradient."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    bnorm = _norm(b)
    if bnorm == 0.0:
        return SolveResult(x=np.zeros_like(b), iters=0, status="converged", history=[0.0], relres_true=0.0)
    r = b - A(x)
    rel = _norm(r) / bnorm
    hist = [rel]
    if rel <= tol:
        return _finish(A, b, x, bnorm, 0, "converged", hist)
    z = M(r)
    p = z.copy()
    rz = _dot(r, z)
    it = 0
    status = "max_iter"
    while it < maxit:
        q = A(p)
        pq = _dot(p, q)
        it += 1
        if pq == 0.0 or rz == 0.0:
            status = "breakdown"
            break
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        rel = _norm(r) / bnorm
        hist.append(rel)
        if not np.isfinite(rel):
            status = "nonfinite"
            break
        if rel <= tol:
            status = "converged"
            break
        z = M(r)
        rz_new = _dot(r, z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return _finish(A, b, x, bnorm, it, status, hist)


def rmr(A, M, b, x0=None, tol=1e-10, maxit=500) -> SolveResult:
    """Richardson minimal residual: x += alpha M r with alpha minimising ||r - alpha A M r||."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    bnorm = _norm(b)
    if bnorm == 0.0:
        return SolveResult(x=np.zeros_like(b), iters=0, status="converged", history=[0.0], relres_true=0.0)
    r = b - A(x)
    rel = _norm(r) / bnorm
    hist = [rel]
    if rel <= tol:
        return _finish(A, b, x, bnorm, 0, "converged", hist)
    it = 0
    best = rel
    status = "max_iter"
    while it < maxit:
        z = M(r)
        w = A(z)
        it += 1
        ww = _dot(w, w)
        if ww == 0.0:
            status = "breakdown"
            break
        alpha = _dot(r, w) / ww
        x = x + alpha * z
        r = r - alpha * w
        rel = _norm(r) / bnorm
        hist.append(rel)
        if not np.isfinite(rel):
            status = "nonfinite"
            break
        if rel <= tol:
            status = "converged"
            break
        if rel > DIVERGE_FACTOR * best:
            status = "diverged"
            break
        best = min(best, rel)
    return _finish(A, b, x, bnorm, it, status, hist)


def _givens(a: float, b: float):
    """Rotation (c, s) with c*a + s*b = hypot(a, b) and -s*a + c*b = 0."""
    if b == 0.0:
        return 1.0, 0.0
    h = np.hypot(a, b)
    return a / h, b / h


def gmres(A, M, b, x0=None, tol=1e-10, maxit=500, restart=30) -> SolveResult:
    """Right-preconditioned restarted GMRES(restart) with modified Gram--Schmidt.

    Convergence is decided by the Givens estimate of the residual (like the recurrence
    residual of CG and RMR); a cycle that ends without convergence restarts from the true
    residual of the updated iterate, which is also checked against tol.
    """
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    bnorm = _norm(b)
    if bnorm == 0.0:
        return SolveResult(x=np.zeros_like(b), iters=0, status="converged", history=[0.0], relres_true=0.0)
    m = int(restart)
    it = 0
    hist = []
    status = "max_iter"
    while True:
        r = b - A(x)
        beta = _norm(r)
        rel = beta / bnorm
        if not hist:
            hist.append(rel)
        if not np.isfinite(rel):
            status = "nonfinite"
            break
        if rel <= tol:
            status = "converged"
            break
        if it >= maxit:
            status = "max_iter"
            break
        V = [r / beta]
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k = 0
        conv = False
        while k < m and it < maxit:
            w = A(M(V[k]))
            it += 1
            for i in range(k + 1):
                H[i, k] = _dot(w, V[i])
                w = w - H[i, k] * V[i]
            hn = _norm(w)
            H[k + 1, k] = hn
            # apply the previous rotations to the new column
            for i in range(k):
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            cs[k], sn[k] = _givens(H[k, k], H[k + 1, k])
            H[k, k] = cs[k] * H[k, k] + sn[k] * H[k + 1, k]
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            est = abs(g[k + 1]) / bnorm
            hist.append(est)
            k += 1
            if est <= tol or hn == 0.0:   # converged, or happy breakdown (invariant space)
                conv = True
                break
            if not np.isfinite(est):
                break
            V.append(w / hn)
        # least-squares update x += M V y with H[:k,:k] y = g[:k]
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        upd = np.zeros_like(b)
        for i in range(k):
            upd = upd + y[i] * V[i]
        x = x + M(upd)
        if not np.all(np.isfinite(y)) or not np.isfinite(hist[-1]):
            status = "nonfinite"
            break
        if conv:
            status = "converged"
            break
        # otherwise: restart (the loop head forms the true residual of the new iterate)
    return _finish(A, b, x, bnorm, it, status, hist)


SOLVERS = {"cg": cg, "gmres": gmres, "rmr": rmr}


def solve(kind: str, A, M, b, x0=None, tol=1e-10, maxit=500, restart=30) -> SolveResult:
    if kind == "gmres":
        return gmres(A, M, b, x0, tol, maxit, restart)
    return SOLVERS[kind](A, M, b, x0, tol, maxit)
