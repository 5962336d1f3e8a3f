"""FP64 Krylov solvers of the oracle (test infrastructure only).

* ``cg_normal``  -- CG on D D^dag y = b, x = D^dag y (the CG comparator of Sec. 1.1 / Fig. 1 and the
  CG solver of Sec. 1.2).  Pinned by dense LU on 2^4 / 4^4 lattices.
* ``gmres``      -- restarted GMRES with modified Gram-Schmidt and Givens rotations (the coarse
  solve D_c^-1 of Eq. 1 is approximated with it).  Pinned by dense LU.
* ``fgmres``     -- right-preconditioned flexible GMRES (Sec. 1.1: "a flexible iterative Krylov
  solver is preconditioned at every iteration step"); the true residual is recomputed at every
  restart.  Pinned by dense LU and by the full-rank-P exact-coarse-correction case.

All vectors are numpy arrays of any shape; inner products are <a, b> = sum conj(a) b.
"""
from __future__ import annotations

import numpy as np


def _dot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def _nrm(a):
    return float(np.sqrt(np.real(_dot(a, a))))


def cg_normal(apply_D, apply_Ddag, b, tol=1e-12, maxiter=100000, x0=None):
    """Solve D x = b by CG on D D^dag y = b, x = D^dag y.  Returns (x, iterations, rel_res)."""
    bn = _nrm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0
    y = np.zeros_like(b)
    r = b.copy()
    if x0 is not None:
        # warm start: only through the residual (y stays 0, correction added at the end)
        r = b - apply_D(x0)
    p = r.copy()
    rr = np.real(_dot(r, r))
    it = 0
    while it < maxiter and np.sqrt(rr) > tol * bn:
        q = apply_Ddag(p)
        ap = apply_D(q)
        alpha = rr / np.real(_dot(q, q))
        y += alpha * p
        r -= alpha * ap
        rr_new = np.real(_dot(r, r))
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    x = apply_Ddag(y)
    if x0 is not None:
        x = x + x0
    return x, it, _nrm(b - apply_D(x)) / bn


def _arnoldi_cycle(apply_A, r0, m, rtol_abs, precond=None):
    """One (F)GMRES cycle of at most m steps from residual r0.

    Returns the correction e (sum of z_j y_j, z_j = M v_j or v_j) and the number of steps taken.
    Stops early when the Givens least-squares residual estimate falls to rtol_abs.
    """
    beta = _nrm(r0)
    v = [r0 / beta]
    z = []
    h = np.zeros((m + 1, m), dtype=np.complex128)
    cs = np.zeros(m, dtype=np.complex128)
    sn = np.zeros(m, dtype=np.complex128)
    g = np.zeros(m + 1, dtype=np.complex128)
    g[0] = beta
    k = 0
    for j in range(m):
        zj = precond(v[j]) if precond is not None else v[j]
        z.append(zj)
        w = apply_A(zj)
        for i in range(j + 1):            # modified Gram-Schmidt
            h[i, j] = _dot(v[i], w)
            w = w - h[i, j] * v[i]
        hn = _nrm(w)
        h[j + 1, j] = hn
        for i in range(j):                # previous rotations [[conj c, conj s], [-s, c]]
            t = np.conj(cs[i]) * h[i, j] + np.conj(sn[i]) * h[i + 1, j]
            h[i + 1, j] = -sn[i] * h[i, j] + cs[i] * h[i + 1, j]
            h[i, j] = t
        a, bb = h[j, j], h[j + 1, j]
        den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
        cs[j] = a / den if den != 0 else 1.0
        sn[j] = bb / den if den != 0 else 0.0
        h[j, j] = den
        h[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = np.conj(cs[j]) * g[j]
        k = j + 1
        if abs(g[j + 1]) <= rtol_abs or hn == 0.0:
            break
        v.append(w / hn)
    # back substitution on the k x k upper triangle
    y = np.zeros(k, dtype=np.complex128)
    for i in range(k - 1, -1, -1):
        y[i] = (g[i] - np.dot(h[i, i + 1:k], y[i + 1:k])) / h[i, i]
    e = np.zeros_like(r0)
    for i in range(k):
        e = e + y[i] * z[i]
    return e, k


def gmres(apply_A, b, m=30, tol=1e-12, maxiter=10000, x0=None, precond=None):
    """Restarted (flexible, if precond is given) GMRES(m) with right preconditioning.

    The true residual b - A x is recomputed at every restart and the solve stops when
    ||b - A x|| <= tol ||b|| or after maxiter inner steps.  Returns (x, steps, rel_res).
    """
    bn = _nrm(b)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    if bn == 0.0:
        return x, 0, 0.0
    r = b - apply_A(x) if x0 is not None else b.copy()
    steps = 0
    while True:
        rn = _nrm(r)
        if rn <= tol * bn or steps >= maxiter:
            return x, steps, rn / bn
        e, k = _arnoldi_cycle(apply_A, r, min(m, maxiter - steps), tol * bn, precond)
        x = x + e
        steps += k
        r = b - apply_A(x)


def fgmres(apply_A, b, precond, m=10, tol=1e-10, maxiter=10000, x0=None):
    """Flexible GMRES(m), right-preconditioned by the (possibly varying) map precond."""
    return gmres(apply_A, b, m=m, tol=tol, maxiter=maxiter, x0=x0, precond=precond)


def gmres_fixed(apply_A, b, m, rtol):
    """Approximate inverse from zero: one GMRES cycle of at most m steps, stopping once the
    Givens residual estimate is <= rtol ||b||.  This is the coarse solve D_c^-1 of Eq. 1."""
    bn = _nrm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0
    return _arnoldi_cycle(apply_A, b, m, rtol * bn, None)


def mr(apply_A, b, n):
    """n minimal-residual steps from zero: e += a r, r -= a A r with a = <Ar, r>/<Ar, Ar>."""
    e = np.zeros_like(b)
    r = b.copy()
    for _ in range(n):
        p = apply_A(r)
        pp = np.real(_dot(p, p))
        if pp == 0.0:
            break
        a = _dot(p, r) / pp
        e += a * r
        r -= a * p
    return e
