"""FP64 oracle of the multigrid for the non-degenerate doublet (test infrastructure only).

Eq. 2: D_ND = D x I2 + i mubar G5 x tau3 - epsbar I x tau1, i.e. [[D(mubar), -epsbar],
[-epsbar, D(-mubar)]] on a flavour pair psi2[2, ...].  Sec. 1.2 coarsens it with the prolongation P
of the single-flavour operator used flavour-diagonally, P_ND = P x I2, so
D_ND,c = P_ND^dag D_ND P_ND = D_c x I2 + i mubar G5_c x tau3 - epsbar I x tau1 (P^dag P = I and
G5 P = P G5_c); the third level repeats this with P2_ND = P2 x I2.

The shifted doublet systems of the rational approximation (Sec. 3, Q_ND^2 + delta^2 =
(Q_ND - i delta)(Q_ND + i delta) with Q_ND + i delta = (G5 x tau1)(D_ND + i delta G5 x tau1)) add the
site-local term i delta G5 x tau1 (p.ndshift), which P_ND maps to i delta G5_c x tau1.

Readings (the paper gives only the coarse operator): the smoother is SAP on D_ND, whose block
solves are MR steps on the flavour-coupled block operator (inner products over both flavours);
the cycle, the coarse GMRES, the level-1 K-cycle and the outer FGMRES are those of the single-flavour
method with D, D_c, D_cc replaced by their doublet forms; P and P2 come from the single-flavour
setup of D(mubar) (the flavour-diagonal part of D_ND).

Pinned by tests/test_oracle_nd.py: the block operator against the full operator on block-local
vectors, SAP at epsbar = 0 against two independent single-flavour SAPs with +-mubar, both coarse
operators against their definitions, and the two- and three-level solves against dense LU and
against CG on the normal equations of D_ND.
"""
from __future__ import annotations

import numpy as np

from . import dirac, krylov, mg


def apply_DND_blocks(U, psi2, p: dirac.Params, clover, bdims):
    """Block-diagonal Dirichlet form of D_ND (hops across block faces dropped; the flavour mixing
    is site-local)."""
    u = mg.apply_D_blocks(U, psi2[0], p, clover, bdims, p.mubar) - p.epsbar * psi2[1]
    d = mg.apply_D_blocks(U, psi2[1], p, clover, bdims, -p.mubar) - p.epsbar * psi2[0]
    if p.ndshift:
        u = u + 1j * p.ndshift * dirac.apply_g5(psi2[1])
        d = d + 1j * p.ndshift * dirac.apply_g5(psi2[0])
    return np.stack([u, d])


def block_inner_nd(a2, b2, bdims):
    return mg.block_inner(a2[0], b2[0], bdims) + mg.block_inner(a2[1], b2[1], bdims)


def block_mr_nd(U, p, clover, r2, bdims, n_mr):
    """n_mr MR steps on every block of D_ND at once, step lengths from both flavours."""
    e = np.zeros_like(r2)
    r = r2.copy()
    for _ in range(n_mr):
        q = apply_DND_blocks(U, r, p, clover, bdims)
        qq = np.real(block_inner_nd(q, q, bdims))
        qr = block_inner_nd(q, r, bdims)
        a = np.where(qq > 0, qr / np.where(qq > 0, qq, 1.0), 0.0)
        ab = mg.block_broadcast(a, bdims)
        e += ab * r
        r -= ab * q
    return e


def sap_nd(U, p, clover, b2, bdims, n_sweeps, n_mr, x0=None):
    """Multiplicative SAP on D_ND: n_sweeps x (colour 0, colour 1) block-MR updates."""
    lat = U.shape[:4]
    col = mg.block_colour(lat, bdims)
    x = np.zeros_like(b2) if x0 is None else x0.copy()
    for _ in range(n_sweeps):
        for c in (0, 1):
            r = b2 - dirac.apply_DND(U, x, p, clover)
            rc = r * (col == c)[..., None, None]
            x = x + block_mr_nd(U, p, clover, rc, bdims, n_mr)
    return x


def restrict_nd(P, r2):
    return np.stack([mg.restrict(P, r2[0]), mg.restrict(P, r2[1])])


def prolong_nd(P, c2):
    return np.stack([mg.prolong(P, c2[0]), mg.prolong(P, c2[1])])


def restrict_c_nd(P2, r2):
    return np.stack([mg.restrict_c(P2, r2[0]), mg.restrict_c(P2, r2[1])])


def prolong_c_nd(P2, c2):
    return np.stack([mg.prolong_c(P2, c2[0]), mg.prolong_c(P2, c2[1])])


class Level1ND:
    """Level-1 K-cycle of the doublet on top of a single-flavour Level1 (its P2 and D_cc)."""

    def __init__(self, L1: mg.Level1, mubar, epsbar, delta=0.0):
        self.L1, self.mubar, self.epsbar, self.delta = L1, mubar, epsbar, delta

    def A(self, x2):
        return mg.coarse_apply_nd(self.L1.Dc, x2, self.mubar, self.epsbar, self.delta)

    def A2(self, x2):
        return mg.coarse_apply_nd(self.L1.Dcc, x2, self.mubar, self.epsbar, self.delta)

    def smooth(self, b2, x2):
        r = b2 - self.A(x2)
        e, _ = krylov.gmres_fixed(self.A, r, self.L1.prm.smooth_m, 0.0)
        return x2 + e

    def cycle(self, r2):
        prm = self.L1.prm
        e2, _ = krylov.gmres_fixed(self.A2, restrict_c_nd(self.L1.P2, r2), prm.coarse_m, prm.coarse_rtol)
        return self.smooth(r2, prolong_c_nd(self.L1.P2, e2))

    def solve(self, b2):
        prm = self.L1.prm
        x, _, _ = krylov.fgmres(self.A, b2, self.cycle, m=prm.k_restart, tol=prm.k_rtol, maxiter=prm.k_maxiter)
        return x


class HierarchyND:
    """DD-alpha-AMG for D_ND from a single-flavour hierarchy H (its P, D_c and optional Level1)."""

    def __init__(self, H: mg.Hierarchy, L1: mg.Level1 = None):
        self.H, self.p = H, H.p
        self.L1 = None if L1 is None else Level1ND(L1, H.p.mubar, H.p.epsbar, H.p.ndshift)

    def D(self, x2):
        return dirac.apply_DND(self.H.U, x2, self.p, self.H.clover)

    def smooth(self, b2, x0):
        m = self.H.mg
        return sap_nd(self.H.U, self.p, self.H.clover, b2, m.block, m.sap_sweeps, m.sap_mr, x0)

    def coarse_apply(self, c2):
        return mg.coarse_apply_nd(self.H.Dc, c2, self.p.mubar, self.p.epsbar, self.p.ndshift)

    def coarse_solve(self, c2):
        if self.L1 is not None:
            return self.L1.solve(c2)
        e, _ = krylov.gmres_fixed(self.coarse_apply, c2, self.H.mg.coarse_m, self.H.mg.coarse_rtol)
        return e

    def cycle(self, r2):
        z = prolong_nd(self.H.P, self.coarse_solve(restrict_nd(self.H.P, r2)))
        return self.smooth(r2, z)

    def solve(self, b2, tol=1e-10, maxiter=2000):
        return krylov.fgmres(self.D, b2, self.cycle, m=self.H.mg.restart, tol=tol, maxiter=maxiter)
