"""FP64 oracle of the hopping-parameter search (test infrastructure only).

The workloads fix kappa indirectly: "kappa tuned so that sigma_min(D_W) is about a target at
mu = 0".  sigma_min(D_W) is the smallest singular value of D_W, equal to the smallest |eigenvalue|
of the Hermitian Q = G5 D_W (Eq. 3 uses Q = G5 D).  This module assembles D_W as a sparse matrix,
gets min |lambda(Q)| by shift-invert Lanczos around 0 (scipy ``eigsh``, i.e. a sparse LU of Q), and
runs the search: start at m0 = 0, step m0 down by 0.05 until sigma_min drops below the target, then
bisect the last step until sigma_min is within +-2 % of the target (the first crossing from above);
if no m0 down to -2 reaches the target, the most critical m0 (minimum of sigma_min) is used.

Pinned by tests/test_oracle_kappa.py: the sparse matrix equals the matrix-free operator of
``oracle.dirac`` on random vectors, and on the free field sigma_min equals the closed form
min_p sqrt(M(p)^2 + sum_mu sin^2 p_mu) over the allowed momenta.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import dirac


def sparse_DW(U, p: dirac.Params, clover=None):
    """Sparse FP64 matrix of D_W (twist excluded); dof index = 12 * lex_site + 3 * spin + colour."""
    lat = U.shape[:4]
    V = int(np.prod(lat))
    if clover is None:
        clover = dirac.clover_term(U, p.csw)
    site = np.arange(V).reshape(lat)
    rows, cols, vals = [], [], []

    def add_blocks(row_site, col_site, blocks):
        # blocks[V, 12, 12]
        r = (12 * row_site.reshape(V, 1, 1) + np.arange(12).reshape(1, 12, 1)) + 0 * np.arange(12).reshape(1, 1, 12)
        c = (12 * col_site.reshape(V, 1, 1) + np.arange(12).reshape(1, 1, 12)) + 0 * np.arange(12).reshape(1, 12, 1)
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(blocks.ravel())

    diag = clover.reshape(V, 12, 12) + (4.0 + p.m0) * np.eye(12)[None]
    add_blocks(site, site, diag)
    t_index = np.indices(lat)[0]
    T = lat[0]
    for mu in range(4):
        Umu = U[..., mu, :, :].reshape(V, 3, 3)
        fwd_site = dirac.shift_fwd(site[..., None, None], mu)[..., 0, 0]    # index of x + mu
        bwd_site = dirac.shift_bwd(site[..., None, None], mu)[..., 0, 0]    # index of x - mu
        sgn_f = np.ones(lat)
        sgn_b = np.ones(lat)
        if mu == 3 and p.tbc != 1:
            sgn_f[t_index == T - 1] = p.tbc
            sgn_b[t_index == 0] = p.tbc
        Pm = dirac.I4 - dirac.GAMMA[mu]
        Pp = dirac.I4 + dirac.GAMMA[mu]
        f = -0.5 * sgn_f.reshape(V, 1, 1, 1, 1) * np.einsum("st,vab->vsatb", Pm, Umu)
        Ub = dirac.dagger(U[..., mu, :, :])                                  # U_mu(x)^dag at x
        Ub = dirac.shift_bwd(Ub, mu).reshape(V, 3, 3)                        # U_mu(x - mu)^dag
        b = -0.5 * sgn_b.reshape(V, 1, 1, 1, 1) * np.einsum("st,vab->vsatb", Pp, Ub)
        add_blocks(site, fwd_site, f.reshape(V, 12, 12))
        add_blocks(site, bwd_site, b.reshape(V, 12, 12))
    n = 12 * V
    return sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def sigma_min(U, p: dirac.Params, clover=None):
    """Smallest singular value of D_W = smallest |eigenvalue| of Q = G5 D_W."""
    D = sparse_DW(U, p, clover)
    n = D.shape[0]
    g5 = np.tile(np.repeat(np.diag(dirac.GAMMA5).real, 3), n // 12)
    Q = sp.diags(g5) @ D
    Q = ((Q + Q.getH()) * 0.5).tocsc()   # exact Hermitian form (removes rounding asymmetry)
    lu = spla.splu(Q, permc_spec="MMD_AT_PLUS_A")
    inv = spla.LinearOperator(Q.shape, matvec=lu.solve, dtype=np.complex128)
    w = spla.eigsh(Q, k=1, sigma=0.0, which="LM", OPinv=inv, return_eigenvectors=False, tol=1e-10)
    return float(np.min(np.abs(w)))


def sigma_min_mg(U, p: dirac.Params, clover=None, mgp=None, seed=7, tol=1e-10):
    """sigma_min(D_W) by Lanczos (ARPACK) on Q^-1, with Q^-1 v = D_W^-1 G5 v from the oracle's own
    two-level DD-alpha-AMG solve at mu = 0; used where a sparse LU of Q is too expensive."""
    from . import mg
    from synth import fields  # noqa: F401  (seeded vectors only)
    p0 = dirac.Params(kappa=p.kappa, csw=p.csw, mu=0.0, tbc=p.tbc)
    if mgp is None:
        mgp = mg.MGParams(nv=8, n_init=3, n_iter=1)
    H = mg.Hierarchy(U, p0, mgp, clover)
    lat = U.shape[:4]
    H.setup(fields.gaussian_spinor((lat[3], lat[2], lat[1], lat[0]), seed, n=mgp.nv))
    shape = lat + (4, 3)
    n = int(np.prod(shape))

    def qinv(v):
        x, _, res = H.solve(dirac.apply_g5(v.reshape(shape)), tol=tol, mu=0.0)
        return x.ravel()

    op = spla.LinearOperator((n, n), matvec=qinv, dtype=np.complex128)
    w = spla.eigsh(op, k=2, which="LM", return_eigenvectors=False, tol=1e-6)
    return float(1.0 / np.max(np.abs(w)))


def search_m0(U, csw, tbc, target, step=0.05, rel_tol=0.02, m0_min=-2.0, log=None, method=None, progress=None):
    """kappa search on sigma_min(D_W(m0)).

    Scan m0 = 0, -step, -2 step, ... down to m0_min.  If sigma_min drops below the target, bisect
    the last step until sigma_min is within +-rel_tol of the target (the first crossing from
    above).  If it never does (a lattice too small or a field too smooth to have a mode that
    low), return the scan's minimiser refined by golden-section search: the most critical m0.
    Returns (m0, sigma_min, reached_target)."""
    clover = dirac.clover_term(U, csw)
    method = sigma_min if method is None else method
    log = [] if log is None else log

    def s(m0):
        v = method(U, dirac.Params(kappa=dirac.kappa_from_m0(m0), csw=csw, tbc=tbc), clover)
        log.append((m0, v))
        if progress is not None:
            progress(m0, v)
        return v

    hi, s_hi = 0.0, s(0.0)
    if s_hi < target:
        raise ValueError("sigma_min already below target at m0 = 0")
    n = int(round(-m0_min / step))
    for i in range(1, n + 1):
        lo = -i * step
        s_lo = s(lo)
        if s_lo < target:
            if abs(s_lo - target) <= rel_tol * target:
                return lo, s_lo, True
            for _ in range(60):
                mid = 0.5 * (lo + hi)
                s_mid = s(mid)
                if abs(s_mid - target) <= rel_tol * target:
                    return mid, s_mid, True
                if s_mid < target:
                    lo = mid
                else:
                    hi = mid
            raise ValueError("bisection did not reach the tolerance")
        hi, s_hi = lo, s_lo
    # no crossing: golden-section refinement around the scan minimum
    m_best, s_best = min(log, key=lambda t: t[1])
    a_, b_ = m_best - step, m_best + step
    g = (np.sqrt(5.0) - 1.0) / 2.0
    c_, d_ = b_ - g * (b_ - a_), a_ + g * (b_ - a_)
    fc, fd = s(c_), s(d_)
    for _ in range(12):
        if fc < fd:
            b_, d_, fd = d_, c_, fc
            c_ = b_ - g * (b_ - a_)
            fc = s(c_)
        else:
            a_, c_, fc = c_, d_, fd
            d_ = a_ + g * (b_ - a_)
            fd = s(d_)
    m_best, s_best = min(log, key=lambda t: t[1])
    return m_best, s_best, False


def mg_steps(U, m0, csw, mu, block, nv, b, v0, tol=1e-10, max_steps=50):
    """Outer FGMRES steps of the oracle's two-level DD-alpha-AMG (paper defaults: SAP k = 3, MR 4,
    coarse GMRES 30 / 5e-2, setup 5 + 3, restart 10) on D(mu) at this m0; max_steps + 1 if it does
    not reach tol within max_steps."""
    from . import mg
    p = dirac.Params(kappa=dirac.kappa_from_m0(m0), csw=csw, mu=mu, tbc=-1)
    H = mg.Hierarchy(U, p, mg.MGParams(block=block, agg=block, nv=nv, restart=10))
    H.setup(v0)
    x, steps, res = H.solve(b, tol=tol, maxiter=max_steps)
    return steps if res <= tol else max_steps + 1


def search_m0_mg(U, csw, mu, block, nv, b, v0, max_steps=50, step=0.1, n_bisect=2, log=None, progress=None):
    """The most critical m0 at which the two-level method still converges: walk m0 = 0, -step, ...
    and stop at the first m0 whose solve needs more than max_steps outer steps; then bisect n_bisect
    times between the last converging m0 and that one.  Returns the last converging m0."""
    log = [] if log is None else log

    def ok(m0):
        n = mg_steps(U, m0, csw, mu, block, nv, b, v0, max_steps=max_steps)
        log.append((m0, n))
        if progress is not None:
            progress(m0, n)
        return n <= max_steps

    if not ok(0.0):
        raise ValueError("the method does not converge at m0 = 0")
    good, bad = 0.0, None
    k = 1
    while bad is None:
        m0 = -k * step
        if m0 < -4.0:
            raise ValueError("no divergence edge above m0 = -4")
        if ok(m0):
            good = m0
        else:
            bad = m0
        k += 1
    for _ in range(n_bisect):
        mid = 0.5 * (good + bad)
        if ok(mid):
            good = mid
        else:
            bad = mid
    return good


def select_m0(mg_log, ratio=2.0):
    """From a convergence-edge walk [(m0, steps), ...]: the most critical m0 whose outer step count
    is at most ratio times the count at m0 = 0 (a margin below the edge, where the step count on the
    small search lattice still carries over to the workload's lattice)."""
    base = dict(mg_log)[0.0]
    ok = [m for m, n in mg_log if n <= ratio * base]
    return min(ok)
