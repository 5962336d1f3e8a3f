"""FP64 oracle of the even-odd reduced twisted-mass operator (test infrastructure only).

The paper's simulations run on the even-odd reduced operator (Sec. 1.2, simulation
characteristics) and its CG comparator is an odd-even CG (Fig. 1 caption).  The reduction is the
Schur complement of D(mu) with respect to the even sites:

* site parity p(x) = (x + y + z + t) mod 2; the hopping term connects only opposite parities, so
  D(mu) = M(mu) + H with the site-local M(mu) = (4 + m0) + C(x) + i mu g5 and the hopping part
  H = -1/2 sum_mu [...] of ``oracle.dirac.hopping``;
* in even/odd blocks D = [[M_e, H_eo], [H_oe, M_o]] and the operator on the odd sites is
      Dhat(mu) = M_o - H_oe M_e^-1 H_eo;
* D x = b is solved by Dhat x_o = b_o - H_oe M_e^-1 b_e, then x_e = M_e^-1 (b_e - H_eo x_o).

Fields here are full-lattice arrays ([..., T, Z, Y, X, 4, 3]) that vanish on the parity they do
not live on, so every step reads as the block formula it implements.

Pinned by tests/test_oracle_eo.py: the even-odd solve equals the dense LU solution of the full D
(brute force on 4^4), det D = det M_e det Dhat (Schur determinant identity, dense 2^4),
gamma5-hermiticity g5 Dhat(mu) g5 = Dhat(-mu)^dag, and the odd-even CG against the full CG.
"""
from __future__ import annotations

import numpy as np

from . import dirac, krylov


def parity(lat_shape):
    """0 on even sites, 1 on odd sites of a (T, Z, Y, X) lattice."""
    t, z, y, x = np.indices(lat_shape)
    return (x + y + z + t) % 2


def site_mass(U, p: dirac.Params, mu=None, clover=None):
    """Per-site 12 x 12 matrices M(x) = (4 + m0) + C(x) + i mu g5, as [T, Z, Y, X, 12, 12]."""
    mu = p.mu if mu is None else mu
    if clover is None:
        clover = dirac.clover_term(U, p.csw)
    lat = U.shape[:4]
    M = clover.reshape(lat + (12, 12)).copy()
    M += (4.0 + p.m0) * np.eye(12)
    M += 1j * mu * np.kron(dirac.GAMMA5, np.eye(3))
    return M


def apply_site(M, psi):
    """(M psi)(x) with per-site 12 x 12 matrices."""
    v = psi.reshape(psi.shape[:-2] + (12, 1))
    return np.matmul(M, v).reshape(psi.shape)


def restrict_parity(psi, par, which):
    """psi on the sites of parity `which`, zero elsewhere."""
    return psi * (par == which)[..., None, None]


def schur_apply(U, x, p: dirac.Params, mu=None, clover=None):
    """Dhat(mu) x_o = M_o x_o - H_oe M_e^-1 H_eo x_o for x supported on the odd sites."""
    mu = p.mu if mu is None else mu
    if clover is None:
        clover = dirac.clover_term(U, p.csw)
    lat = U.shape[:4]
    par = parity(lat)
    M = site_mass(U, p, mu, clover)
    Minv = np.linalg.inv(M)
    xo = restrict_parity(x, par, 1)
    h_e = restrict_parity(dirac.hopping(U, xo, p.tbc), par, 0)        # H_eo x_o
    t_e = apply_site(Minv, h_e)                                        # M_e^-1 H_eo x_o
    y = apply_site(M, xo) - dirac.hopping(U, t_e, p.tbc)               # M_o x_o - H_oe t_e
    return restrict_parity(y, par, 1)


def schur_apply_dag(U, x, p: dirac.Params, mu=None, clover=None):
    """Dhat(mu)^dag = g5 Dhat(-mu) g5 (gamma5-hermiticity of every block)."""
    mu = p.mu if mu is None else mu
    return dirac.apply_g5(schur_apply(U, dirac.apply_g5(x), p, -mu, clover))


def eo_rhs(U, b, p: dirac.Params, mu=None, clover=None):
    """b_o - H_oe M_e^-1 b_e: the right-hand side of the odd-site system."""
    mu = p.mu if mu is None else mu
    if clover is None:
        clover = dirac.clover_term(U, p.csw)
    par = parity(U.shape[:4])
    Minv = np.linalg.inv(site_mass(U, p, mu, clover))
    t_e = apply_site(Minv, restrict_parity(b, par, 0))
    return restrict_parity(b - dirac.hopping(U, t_e, p.tbc), par, 1)


def eo_reconstruct(U, b, x_o, p: dirac.Params, mu=None, clover=None):
    """x = x_o + M_e^-1 (b_e - H_eo x_o): the full solution from the odd-site one."""
    mu = p.mu if mu is None else mu
    if clover is None:
        clover = dirac.clover_term(U, p.csw)
    par = parity(U.shape[:4])
    Minv = np.linalg.inv(site_mass(U, p, mu, clover))
    xo = restrict_parity(x_o, par, 1)
    x_e = apply_site(Minv, restrict_parity(b - dirac.hopping(U, xo, p.tbc), par, 0))
    return xo + restrict_parity(x_e, par, 0)


def cg_eo(U, b, p: dirac.Params, mu=None, clover=None, tol=1e-12, maxiter=100000):
    """The odd-even CG of Fig. 1: CG on Dhat Dhat^dag for the odd-site system, then the even sites
    by reconstruction.  Returns (x, iterations, relative residual of the full system)."""
    mu = p.mu if mu is None else mu
    if clover is None:
        clover = dirac.clover_term(U, p.csw)
    rhs = eo_rhs(U, b, p, mu, clover)
    A = lambda v: schur_apply(U, v, p, mu, clover)
    Ad = lambda v: schur_apply_dag(U, v, p, mu, clover)
    xo, it, _ = krylov.cg_normal(A, Ad, rhs, tol=tol, maxiter=maxiter)
    x = eo_reconstruct(U, b, xo, p, mu, clover)
    r = b - dirac.apply_D(U, x, p, mu, clover)
    return x, it, float(np.linalg.norm(r) / np.linalg.norm(b))
