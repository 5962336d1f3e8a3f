"""GPU HMC (Sec. 2: Hasenbusch-split monomials on nested minimal-norm time scales, solves by the
mixed-precision DD-alpha-AMG) against the oracle's trajectory (oracle/hmc.py) from the same links,
momenta and heat-bath Gaussians: the Wilson gauge action and force, the final links, momenta and
dH; and reversibility of the GPU trajectory (momenta flipped, pseudofermions kept)."""
import numpy as np
import pytest

from oracle import dirac, force, hmc
from synth import fields
from tests.conftest import rel

tmg = pytest.importorskip("paper_1710_06198_gb300")
pytestmark = pytest.mark.gpu

DIMS, BLOCK = (8, 4, 4, 4), (4, 2, 2, 2)


def _ctx(U, p, nv=4):
    ctx = tmg.Context(DIMS, BLOCK)
    ctx.set_params(p.kappa, p.csw, 0.05)
    ctx.load_gauge(U, -1)
    prm = tmg.Context.mg_defaults()
    prm.nv, prm.n_init, prm.n_iter = nv, 3, 1
    ctx.setup(fields.gaussian_spinor(DIMS, 210, n=nv), prm)
    return ctx


def test_gauge_action_and_force():
    U = fields.gauge_field(DIMS, 0.3, 211)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.2), csw=1.0, tbc=-1)
    ctx = tmg.Context(DIMS, BLOCK)
    ctx.set_params(p.kappa, p.csw, 0.05)
    ctx.load_gauge(U, -1)
    assert abs(ctx.gauge_action(5.6) - hmc.gauge_action(U, 5.6)) < 1e-12 * hmc.gauge_action(U, 5.6)
    want = force.matrix_to_algebra(hmc.gauge_force(U, 5.6))
    assert rel(ctx.gauge_force(5.6), want) < 1e-12


def _inputs(seed):
    U = fields.gauge_field(DIMS, 0.3, seed)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.2), csw=1.0, tbc=-1)
    eta = np.stack([fields.gaussian_spinor(DIMS, seed + 1), fields.gaussian_spinor(DIMS, seed + 2)])
    P0 = np.random.default_rng(seed + 3).standard_normal(fields.lattice_shape(DIMS) + (4, 8))
    return U, p, eta, P0


def test_trajectory_matches_oracle():
    U, p, eta, P0 = _inputs(212)
    beta, tau = 5.6, 0.2
    mons = [hmc.Monomial("gauge", beta=beta), hmc.Monomial("ratio", mu=0.05, mu2=0.3), hmc.Monomial("det", mu=0.3)]
    T = hmc.Trajectory(U, p, mons, [([mons[1]], 2), ([mons[2]], 1), ([mons[0]], 2)], tol=1e-13)
    T.heatbath(list(eta))
    P_want, dH_want = T.run(P0, tau)
    ctx = _ctx(U, p)
    hp = tmg.Context.hmc_params(beta, tau, [(0.05, 0.3, 0), (0.3, 0.0, 1)], [2, 1, 2], tol_action=1e-13,
                                tol_force=1e-13, setup_iters_start=0, setup_iters_force=0)
    P = P0.copy()
    dH, st = ctx.hmc_trajectory(hp, P, eta)
    assert rel(ctx.get_gauge(), T.U) < 1e-10
    assert rel(P, P_want) < 1e-9
    assert abs(dH - dH_want) < 1e-7 * max(1.0, abs(dH_want)), (dH, dH_want)
    # time scales of 2, 1 and 2 steps: 2 x 3 ratio forces, 4 x 3 det forces, 8 x 2 x 3 gauge forces
    # and 8 x 2 x 2 link updates
    assert st["fermion_forces"] == 6 + 12 and st["gauge_forces"] == 48 and st["link_updates"] == 32


def test_trajectory_reversibility_and_setup_updates():
    """Default solver tolerances of Sec. 2 (1e-11 action, 1e-9 force) and setup updates (3 at the
    start, 1 per lightest force): flipping the momenta retraces the trajectory."""
    U, p, eta, P0 = _inputs(213)
    ctx = _ctx(U, p)
    hp = tmg.Context.hmc_params(5.6, 0.2, [(0.05, 0.3, 0), (0.3, 0.0, 1)], [2, 1, 2], tol_action=1e-12, tol_force=1e-11)
    P = P0.copy()
    dH1, _ = ctx.hmc_trajectory(hp, P, eta)
    P = -P
    hp.keep_phi = 1
    dH2, _ = ctx.hmc_trajectory(hp, P, eta)
    assert rel(ctx.get_gauge(), U) < 1e-8
    assert rel(P, -P0) < 1e-8
    assert abs(dH1 + dH2) < 1e-6 * max(1.0, abs(dH1))
