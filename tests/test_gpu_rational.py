"""GPU multi-shift CG (tmg_mms_cg, the MMS-CG of Sec. 3) and rational-function application
(tmg_rational_apply, R of Eq. 5) against the oracle's multi-shift CG on the same operators:
A = D^dag D (one flavour) and A = Q_ND^2 (the non-degenerate doublet, Eqs. 2 and 4), FP64."""
import numpy as np
import pytest

from oracle import dirac, rational
from synth import fields
from tests.conftest import rel

tmg = pytest.importorskip("paper_1710_06198_gb300")
pytestmark = pytest.mark.gpu

DIMS, BLOCK = (8, 4, 4, 4), (4, 2, 2, 2)


def _ctx(U, p):
    ctx = tmg.Context(DIMS, BLOCK)
    ctx.set_params(p.kappa, p.csw, p.mu, p.mubar, p.epsbar)
    ctx.load_gauge(U, p.tbc)
    return ctx


@pytest.mark.parametrize("flavours", [1, 2])
def test_mms_cg_matches_oracle(flavours):
    U = fields.gauge_field(DIMS, 0.4, 170)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.2), csw=1.2, mu=0.05, mubar=0.12, epsbar=0.13, tbc=-1)
    C = dirac.clover_term(U, p.csw)
    if flavours == 1:
        A = lambda v: dirac.apply_Ddag(U, dirac.apply_D(U, v, p, clover=C), p, clover=C)
        b = fields.gaussian_spinor(DIMS, 171)
    else:
        A = lambda v: dirac.apply_QND(U, dirac.apply_QND(U, v, p, clover=C), p, clover=C)
        b = fields.gaussian_spinor(DIMS, 171, flavours=2)
    sig = [0.002, 0.01, 0.1, 1.0]
    want, _ = rational.mms_cg(A, b, sig, tol=1e-13)
    ctx = _ctx(U, p)
    x, st = ctx.mms_cg(b, sig, tol=1e-12, flavours=flavours)
    assert st["true_residual"] <= 1e-11
    for s in range(len(sig)):
        assert rel(x[s], want[s]) < 1e-9, s


def test_rational_apply_matches_oracle():
    U = fields.gauge_field(DIMS, 0.4, 172)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.2), csw=1.2, mubar=0.12, epsbar=0.13, tbc=-1)
    C = dirac.clover_term(U, p.csw)
    A = lambda v: dirac.apply_QND(U, dirac.apply_QND(U, v, p, clover=C), p, clover=C)
    phi = fields.gaussian_spinor(DIMS, 173, flavours=2)
    a, num, den, delta = rational.zolotarev(8, 1e-3, 60.0)
    want, _ = rational.rational_apply(A, phi, a, num, den, tol=1e-13)
    ctx = _ctx(U, p)
    got, st = ctx.rational_apply(phi, a, num, den, tol=1e-12, flavours=2)
    assert rel(got, want) < 1e-9


@pytest.mark.parametrize("flavours", [1, 2])
def test_rational_apply_with_multigrid_shifts(flavours):
    """Sec. 3's split: the smallest shifts by the multigrid (two solves each; for the doublet
    through D_ND +- i sqrt(q) (G5 x tau1)), the rest by the multi-shift CG; the result equals the
    oracle's all-MMS-CG evaluation of the same rational function."""
    U = fields.gauge_field(DIMS, 0.4, 174)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.2), csw=1.2, mu=0.05, mubar=0.12, epsbar=0.13, tbc=-1)
    C = dirac.clover_term(U, p.csw)
    if flavours == 1:
        A = lambda v: dirac.apply_Ddag(U, dirac.apply_D(U, v, p, clover=C), p, clover=C)
        phi = fields.gaussian_spinor(DIMS, 175)
    else:
        A = lambda v: dirac.apply_QND(U, dirac.apply_QND(U, v, p, clover=C), p, clover=C)
        phi = fields.gaussian_spinor(DIMS, 175, flavours=2)
    a, num, den, delta = rational.zolotarev(6, 1e-3, 60.0)
    want, _ = rational.rational_apply(A, phi, a, num, den, tol=1e-13)
    ctx = _ctx(U, p)
    if flavours == 2:
        ctx.set_params(p.kappa, p.csw, p.mubar, p.mubar, p.epsbar)    # setup on D(mubar)
    prm = tmg.Context.mg_defaults()
    prm.nv, prm.n_init, prm.n_iter = 4, 3, 1
    ctx.setup(fields.gaussian_spinor(DIMS, 176, n=4), prm)
    if flavours == 2:
        ctx.set_params(p.kappa, p.csw, p.mu, p.mubar, p.epsbar)
    got, st = ctx.rational_apply(phi, a, num, den, tol=1e-12, flavours=flavours, mg_below=float(np.sort(den)[3]))
    assert rel(got, want) < 1e-9
