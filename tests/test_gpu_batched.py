"""Multi-right-hand-side path: the multi-column dslash (tmg_apply with n_rhs > 1) and the
lock-step batched mixed-precision solve (TMG_SOLVE_MG_BATCHED, batched SAP / P / P^dag / coarse
GMRES), checked against the FP64 oracle and against one-at-a-time solves."""
import numpy as np
import pytest

from oracle import dirac
from synth import fields
from tests.conftest import rel

tmg = pytest.importorskip("paper_1710_06198_gb300")
pytestmark = pytest.mark.gpu

DIMS, BLOCK = (8, 8, 4, 4), (4, 4, 2, 2)


@pytest.fixture(scope="module")
def case():
    U = fields.gauge_field(DIMS, 0.4, 95)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.3), csw=1.1, mu=0.02, tbc=-1)
    ctx = tmg.Context(DIMS, BLOCK)
    ctx.set_params(p.kappa, p.csw, p.mu)
    ctx.load_gauge(U, -1)
    prm = tmg.Context.mg_defaults()
    prm.nv, prm.n_init, prm.n_iter = 4, 3, 1
    ctx.setup(fields.gaussian_spinor(DIMS, 96, n=4), prm)
    return ctx, U, p, dirac.clover_term(U, p.csw)


@pytest.mark.parametrize("prec", [tmg.PREC_F32, tmg.PREC_F16])
def test_multi_column_dslash(case, prec):
    ctx, U, p, C = case
    xs = fields.gaussian_spinor(DIMS, 97, n=5)
    mus = [0.02, -0.02, 0.1, 0.0, -0.3]
    y = ctx.apply(xs, tmg.OP_D, prec, mu_per_col=mus)
    tol = 1e-6 if prec == tmg.PREC_F32 else 5e-3
    for j, m in enumerate(mus):
        assert rel(y[j], dirac.apply_D(U, xs[j], p, mu=m, clover=C)) < tol


def test_batched_solve_multi_shift(case):
    """Point sources and twisted masses mu_k = sqrt(mu^2 + sigma_k) (shifted normal equations map
    to twists, Sec. 1.1) in one lock-step solve."""
    ctx, U, p, C = case
    b = np.concatenate([fields.point_sources(DIMS)[:3], fields.gaussian_spinor(DIMS, 98, n=3)])
    sig = [1e-5, 1e-3, 1e-1]
    mus = [p.mu, -p.mu, p.mu] + [float(np.sqrt(p.mu ** 2 + s)) for s in sig]
    x, st = ctx.solve(b, tol=1e-10, method=tmg.SOLVE_MG_BATCHED, mu_per_col=mus)
    assert st["true_residual"] <= 1e-10
    for j, m in enumerate(mus):
        assert rel(dirac.apply_D(U, x[j], p, mu=m, clover=C), b[j]) <= 1e-10
    x1, _ = ctx.solve(b[4], tol=1e-12, method=tmg.SOLVE_MG_MIXED, mu_per_col=[mus[4]])
    assert rel(x[4], x1) < 1e-8


def test_batched_solve_fp16_links():
    """The lock-step solve with the FP16-link fine level (multi-column dslash and SAP with FP16
    links and clover, FP32 spinors) still reaches 1e-10."""
    U = fields.gauge_field(DIMS, 0.4, 99)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.3), csw=1.0, mu=0.02, tbc=-1)
    ctx = tmg.Context(DIMS, BLOCK)
    ctx.set_params(p.kappa, p.csw, p.mu)
    ctx.load_gauge(U, -1)
    prm = tmg.Context.mg_defaults()
    prm.nv, prm.n_init, prm.n_iter, prm.prec_fine = 4, 3, 1, tmg.PREC_F16
    ctx.setup(fields.gaussian_spinor(DIMS, 96, n=4), prm)
    b = fields.gaussian_spinor(DIMS, 100, n=3)
    x, st = ctx.solve(b, tol=1e-10, method=tmg.SOLVE_MG_BATCHED, mu_per_col=[p.mu, -p.mu, 0.05])
    C = dirac.clover_term(U, p.csw)
    for j, m in enumerate([p.mu, -p.mu, 0.05]):
        assert rel(dirac.apply_D(U, x[j], p, mu=m, clover=C), b[j]) <= 1e-10


def test_shifted_solves_with_taylor_guesses(case):
    """tmg_solve_shifts: D(mu_k) x_k = b for twists mu_k = sqrt(mu^2 + sigma_k) (shifted normal
    equations, Sec. 1.1), with zero, previous-solution and first-order Taylor (Sec. 3) initial
    guesses.  Every system reaches 1e-10 measured with the oracle's operator; the three guesses
    give the same solutions; the Taylor guess leaves the systems after the first no more outer
    iterations than the zero guess."""
    ctx, U, p, C = case
    b = fields.gaussian_spinor(DIMS, 101)
    sig = np.logspace(-4, -3, 4)
    mus = [float(np.sqrt(p.mu ** 2 + s)) for s in sig]
    out = {}
    for guess in (0, 1, 2):
        x, its, st = ctx.solve_shifts(b, mus, tol=1e-10, guess=guess, taylor_tol=1e-2)
        for k, m in enumerate(mus):
            assert rel(dirac.apply_D(U, x[k], p, mu=m, clover=C), b) <= 1e-10, (guess, k)
        out[guess] = (x, its)
    for guess in (1, 2):
        assert rel(out[guess][0], out[0][0]) < 1e-8
    assert sum(out[2][1][1:]) <= sum(out[0][1][1:]), (out[0][1], out[2][1])
