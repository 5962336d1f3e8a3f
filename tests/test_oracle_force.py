"""Pins of the oracle's pseudofermion force against central finite differences of
S = ||D^-1 phi||^2 (dense LU solves, exact up to rounding) and against gauge covariance."""
import numpy as np
import pytest

from oracle import dirac, force
from synth import fields


def _solver(U, p):
    shape = U.shape[:4] + (4, 3)
    C = dirac.clover_term(U, p.csw)
    D = dirac.dense_matrix(lambda v: dirac.apply_D(U, v, p, clover=C), shape)
    lu_solve = lambda A, b: np.linalg.solve(A, b.ravel()).reshape(shape)
    return lambda b, dag: lu_solve(D.conj().T if dag else D, b)


def _rotate(U, H, t):
    return np.einsum("...ab,...bc->...ac", fields.exp_i_hermitian(H, t), U)


@pytest.mark.parametrize("csw,mu,tbc", [(1.3, 0.05, -1), (0.0, 0.2, 1), (1.0, -0.1, -1)])
def test_force_matches_finite_differences(csw, mu, tbc):
    dims = (4, 4, 2, 2)
    U = fields.gauge_field(dims, 0.5, 61)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.1), csw=csw, mu=mu, tbc=tbc)
    phi = fields.gaussian_spinor(dims, 62)
    F = force.force(U, phi, p, _solver(U, p))
    # F is traceless Hermitian
    assert np.abs(F - dirac.dagger(F)).max() < 1e-13
    assert np.abs(np.trace(F, axis1=-2, axis2=-1)).max() < 1e-13
    omegas = fields.su3_algebra_directions(dims, 63, 3)
    h = 1e-4
    for om in omegas:
        H = force.algebra_to_matrix(om)
        sp = force.action(_rotate(U, H, h), phi, p, _solver(_rotate(U, H, h), p))
        sm = force.action(_rotate(U, H, -h), phi, p, _solver(_rotate(U, H, -h), p))
        fd = (sp - sm) / (2 * h)
        an = float(np.real(np.einsum("...ab,...ba->...", H, F).sum()))
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
        # the su(3) coefficients reproduce the same directional derivative
        assert abs(np.sum(om * force.matrix_to_algebra(F)) - an) < 1e-10 * abs(an)


def test_force_gauge_covariance():
    dims = (4, 2, 2, 4)
    U = fields.gauge_field(dims, 0.6, 64)
    g = fields.gauge_transform(dims, 65)
    p = dirac.Params(kappa=dirac.kappa_from_m0(0.0), csw=1.4, mu=0.1, tbc=-1)
    phi = fields.gaussian_spinor(dims, 66)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ dirac.dagger(dirac.shift_fwd(g, mu))
    F = force.force(U, phi, p, _solver(U, p))
    Fg = force.force(Ug, dirac.colour_mul(g, phi), p, _solver(Ug, p))
    want = np.einsum("...ab,...mbc,...dc->...mad", g, F, np.conj(g))
    assert np.abs(Fg - want).max() < 1e-11 * np.abs(F).max()
