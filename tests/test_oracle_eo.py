"""Pins of the oracle's even-odd reduced operator (Sec. 1.2 uses the even-odd reduced operator;
Fig. 1's comparator is an odd-even CG):

* brute force on 4^4: the even-odd solve (Schur system solved by dense LU on the odd sites, then
  the even sites reconstructed) equals the dense LU solution of the full D;
* the Schur determinant identity det D = det M_e * det Dhat on 2^4 (log-determinants);
* gamma5-hermiticity g5 Dhat(mu) g5 = Dhat(-mu)^dag with random vectors;
* the odd-even CG reaches the full CG's solution.
"""
import numpy as np

from oracle import dirac, eo, krylov
from synth import fields
from tests.conftest import rel


def _case(dims, seed, m0=-0.3, csw=1.3, mu=0.07):
    U = fields.gauge_field(dims, 0.45, seed)
    p = dirac.Params(kappa=dirac.kappa_from_m0(m0), csw=csw, mu=mu, tbc=-1)
    return U, p, dirac.clover_term(U, p.csw)


def _odd_dense(U, p, C, dims, mu):
    """Dense Dhat on the odd sites (columns from odd unit vectors) and the odd dof indices."""
    shape = fields.lattice_shape(dims) + (4, 3)
    par = np.repeat(eo.parity(fields.lattice_shape(dims)).ravel(), 12)
    odd = np.where(par == 1)[0]
    cols = []
    for k in odd:
        e = np.zeros(int(np.prod(shape)), dtype=np.complex128)
        e[k] = 1.0
        cols.append(eo.schur_apply(U, e.reshape(shape), p, mu, C).ravel()[odd])
    return np.stack(cols, axis=1), odd, par


def test_even_odd_solve_equals_dense_lu():
    dims = (4, 4, 4, 4)
    U, p, C = _case(dims, 300)
    shape = fields.lattice_shape(dims) + (4, 3)
    b = fields.gaussian_spinor(dims, 301)
    D = dirac.dense_matrix(lambda v: dirac.apply_D(U, v, p, clover=C), shape)
    x_lu = np.linalg.solve(D, b.ravel())
    Dh, odd, par = _odd_dense(U, p, C, dims, p.mu)
    rhs = eo.eo_rhs(U, b, p, clover=C).ravel()
    assert np.abs(rhs[par == 0]).max() == 0.0
    xo = np.zeros(D.shape[0], dtype=np.complex128)
    xo[odd] = np.linalg.solve(Dh, rhs[odd])
    x = eo.eo_reconstruct(U, b, xo.reshape(shape), p, clover=C)
    assert rel(x.ravel(), x_lu) < 1e-12


def test_schur_determinant_identity():
    dims = (2, 2, 2, 2)
    U, p, C = _case(dims, 302)
    shape = fields.lattice_shape(dims) + (4, 3)
    D = dirac.dense_matrix(lambda v: dirac.apply_D(U, v, p, clover=C), shape)
    Dh, odd, par = _odd_dense(U, p, C, dims, p.mu)
    M = eo.site_mass(U, p, clover=C)
    ev = eo.parity(fields.lattice_shape(dims)) == 0
    s_full, l_full = np.linalg.slogdet(D)
    s_h, l_h = np.linalg.slogdet(Dh)
    s_e, l_e = np.linalg.slogdet(M[ev])
    assert abs(l_full - (l_h + np.sum(l_e))) < 1e-10 * abs(l_full)
    assert abs(s_full - s_h * np.prod(s_e)) < 1e-9


def test_schur_gamma5_hermiticity():
    dims = (4, 4, 2, 4)
    U, p, C = _case(dims, 303)
    par = eo.parity(fields.lattice_shape(dims))
    x = eo.restrict_parity(fields.gaussian_spinor(dims, 304), par, 1)
    y = eo.restrict_parity(fields.gaussian_spinor(dims, 305), par, 1)
    lhs = np.vdot(y.ravel(), dirac.apply_g5(eo.schur_apply(U, dirac.apply_g5(x), p, p.mu, C)).ravel())
    rhs = np.vdot(eo.schur_apply(U, y, p, -p.mu, C).ravel(), x.ravel())
    assert abs(lhs - rhs) < 1e-13 * abs(rhs)


def test_odd_even_cg_equals_full_cg():
    dims = (4, 4, 4, 4)
    U, p, C = _case(dims, 306)
    b = fields.gaussian_spinor(dims, 307)
    x_eo, it_eo, res = eo.cg_eo(U, b, p, clover=C, tol=1e-12)
    x_cg, it_cg, _ = krylov.cg_normal(lambda v: dirac.apply_D(U, v, p, clover=C),
                                      lambda v: dirac.apply_Ddag(U, v, p, clover=C), b, tol=1e-13)
    assert res < 1e-11
    assert rel(x_eo, x_cg) < 1e-10
    assert it_eo < it_cg
