"""Pins of the oracle's HMC pieces (Sec. 2: Hasenbusch-split monomials on nested minimal-norm time
scales): gauge and ratio-monomial forces against central finite differences, the integrator's
second order, and reversibility."""
import dataclasses

import numpy as np
import pytest

from oracle import dirac, force, hmc
from synth import fields

DIMS = (4, 4, 4, 4)


def _rot(U, om, t):
    return np.einsum("...ab,...bc->...ac", fields.exp_i_hermitian(force.algebra_to_matrix(om), t), U)


def test_gauge_force_finite_differences():
    U = fields.gauge_field(DIMS, 0.3, 200)
    beta = 5.6
    F = hmc.gauge_force(U, beta)
    for om in fields.su3_algebra_directions(DIMS, 201, 3):
        H = force.algebra_to_matrix(om)
        h = 1e-5
        fd = (hmc.gauge_action(_rot(U, om, h), beta) - hmc.gauge_action(_rot(U, om, -h), beta)) / (2 * h)
        an = float(np.real(np.einsum("...ab,...ba->...", H, F).sum()))
        assert abs(fd - an) <= 1e-7 * abs(an)


def test_ratio_monomial_force_finite_differences():
    U = fields.gauge_field(DIMS, 0.3, 202)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.2), csw=1.0, tbc=-1)
    m = hmc.Monomial("ratio", mu=0.05, mu2=0.2)
    T = hmc.Trajectory(U, p, [m], [([m], 1)], tol=1e-14)
    T.heatbath([fields.gaussian_spinor(DIMS, 203)])
    F = T.force(m)
    for om in fields.su3_algebra_directions(DIMS, 204, 2):
        H = force.algebra_to_matrix(om)
        h = 1e-5
        S = []
        for t in (h, -h):
            T.U = _rot(U, om, t)
            S.append(T.action(m))
        T.U = U
        fd = (S[0] - S[1]) / (2 * h)
        an = float(np.real(np.einsum("...ab,...ba->...", H, F).sum()))
        assert abs(fd - an) <= 1e-6 * abs(an)


def _trajectory(n_outer, seed=205):
    U = fields.gauge_field(DIMS, 0.3, seed)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.2), csw=1.0, tbc=-1)
    mons = [hmc.Monomial("gauge", beta=5.6), hmc.Monomial("ratio", mu=0.05, mu2=0.3), hmc.Monomial("det", mu=0.3)]
    levels = [([mons[1]], n_outer), ([mons[2]], 1), ([mons[0]], 2)]
    T = hmc.Trajectory(U, p, mons, levels, tol=1e-13)
    T.heatbath([fields.gaussian_spinor(DIMS, seed + 1), fields.gaussian_spinor(DIMS, seed + 2)])
    P0 = np.random.default_rng(seed + 3).standard_normal(fields.lattice_shape(DIMS) + (4, 8))
    return T, P0, U


@pytest.mark.slow
def test_integrator_second_order_and_reversibility():
    tau = 0.25
    dh = []
    for n in (2, 4):
        T, P0, U0 = _trajectory(n)
        P, d = T.run(P0, tau)
        dh.append(abs(d))
    assert 2.5 < dh[0] / dh[1] < 6.5, dh          # dH ~ e^2
    T, P0, U0 = _trajectory(2)
    P, _ = T.run(P0, tau)
    P2, _ = T.run(-P, tau)                         # flipped momenta: back to the start
    assert np.abs(T.U - U0).max() < 1e-9
    assert np.abs(P2 + P0).max() < 1e-9
