"""GPU parity of the third level (level-2 aggregation of D_c and the level-1 K-cycle) through the C
ABI, against the FP64 oracle's third level on the same seeded fields and test vectors.

* P2 (orthonormalised level-2 basis), P2^dag, P2 and D_cc(mu): FP64 to 1e-12, FP32 to 1e-6;
* the level-1 smoother, cycle and K-cycle solve in FP64 against the oracle's Level1 to 1e-10;
* the level-2 setup in FP64 against the oracle's Level1.setup from the same vectors;
* three-level solves (FP64 and mixed) to a true FP64 residual of 1e-12, agreeing with the oracle's
  three-level solution.
"""
import numpy as np
import pytest

from oracle import dirac, mg
from synth import fields
from tests.conftest import rel

tmg = pytest.importorskip("paper_1710_06198_gb300")
pytestmark = pytest.mark.gpu

F64, F32 = tmg.PREC_F64, tmg.PREC_F32

DIMS, BLOCK = (16, 8, 8, 8), (4, 2, 2, 2)     # level 1: 4^4 sites, level 2: 2^4 sites
NV, NV2, AGG2 = 3, 4, (2, 2, 2, 2)


def build(prec_coarse=F64, n_init=0, n_iter=0, n_init2=0, n_iter2=0, coarse_rtol=5e-2, mu=0.04, nv=NV, nv2=NV2):
    U = fields.gauge_field(DIMS, 0.45, 140)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.3), csw=1.1, mu=mu, tbc=-1)
    ctx = tmg.Context(DIMS, BLOCK)
    ctx.set_params(p.kappa, p.csw, p.mu)
    ctx.load_gauge(U, -1)
    prm = tmg.Context.mg_defaults()
    prm.nv, prm.sap_sweeps, prm.sap_mr = nv, 2, 3
    prm.coarse_m, prm.coarse_rtol = 30, coarse_rtol
    prm.n_init, prm.n_iter, prm.restart = n_init, n_iter, 10
    prm.prec_fine, prm.prec_coarse = F64, prec_coarse
    v0 = fields.gaussian_spinor(DIMS, 141, n=nv)
    ctx.setup(v0, prm)
    mgp = mg.MGParams(block=BLOCK, agg=BLOCK, nv=nv, sap_sweeps=2, sap_mr=3, coarse_m=30, coarse_rtol=coarse_rtol,
                      n_init=n_init, n_iter=n_iter, restart=10)
    p3 = mg.MGParams3(agg2=AGG2, nv2=nv2, smooth_m=3, k_restart=10, k_rtol=0.1, k_maxiter=10, coarse_m=30,
                      coarse_rtol=coarse_rtol, n_init=n_init2, n_iter=n_iter2)
    H = mg.Hierarchy3(U, p, mgp, p3)
    if n_init == 0 and n_iter == 0:
        H.set_vectors(v0)
    else:
        H.setup(v0)
    c1 = ctx.coarse_lat
    v1 = fields.gaussian_coarse((c1[3], c1[2], c1[1], c1[0]), 2 * nv, 142, n=nv2)
    q = tmg.Context.level2_defaults()
    q.agg[:] = AGG2
    q.nv, q.smooth_m, q.k_restart, q.k_rtol = nv2, 3, 10, 0.1
    q.coarse_m, q.coarse_rtol, q.n_init, q.n_iter = 30, coarse_rtol, n_init2, n_iter2
    ctx.setup_level2(v1, q)
    H.L1 = mg.Level1(H.Dc, p3)
    if n_init2 == 0 and n_iter2 == 0:
        H.L1.set_vectors(v1)
    else:
        H.L1.setup(v1, p.mu)
    return ctx, H, U, p


@pytest.fixture(scope="module")
def given():
    return build()


def _c1(ctx, seed):
    c1 = ctx.coarse_lat
    return fields.gaussian_coarse((c1[3], c1[2], c1[1], c1[0]), 2 * ctx.nv, seed)


def _c2(ctx, seed):
    c2 = ctx.coarse2_lat
    return fields.gaussian_coarse((c2[3], c2[2], c2[1], c2[0]), 2 * NV2, seed)


def test_level2_basis(given):
    ctx, H, U, p = given
    assert rel(ctx.get_vectors2(), H.L1.P2.W) < 1e-12


@pytest.mark.parametrize("prec,tol", [(F64, 1e-12), (F32, 1e-6)])
def test_restrict2_prolong2(given, prec, tol):
    ctx, H, U, p = given
    c = _c1(ctx, 143)
    assert rel(ctx.restrict2(c, prec), mg.restrict_c(H.L1.P2, c)) < tol
    c2 = _c2(ctx, 144)
    assert rel(ctx.prolong2(c2, prec), mg.prolong_c(H.L1.P2, c2)) < tol


@pytest.mark.parametrize("prec,tol", [(F64, 1e-12), (F32, 1e-6)])
@pytest.mark.parametrize("mu", [0.0, 0.04, -0.3])
def test_level2_operator(given, prec, tol, mu):
    ctx, H, U, p = given
    x = _c2(ctx, 145)
    assert rel(ctx.coarse_apply2(x, mu, prec), mg.coarse_apply(H.L1.Dcc, x, mu)) < tol


def test_level1_smoother_cycle_and_kcycle(given):
    ctx, H, U, p = given
    b = _c1(ctx, 146)
    mu = p.mu
    assert rel(ctx.kcycle(b, mu, 2, F64), H.L1.smooth(b, np.zeros_like(b), mu)) < 1e-10
    assert rel(ctx.kcycle(b, mu, 1, F64), H.L1.cycle(b, mu)) < 1e-10
    x = ctx.kcycle(b, mu, 0, F64)
    assert rel(x, H.L1.solve(b, mu)) < 1e-10
    # the K-cycle reaches its relative residual target on D_c
    assert rel(mg.coarse_apply(H.Dc, x, mu), b) < 1.0
    assert np.linalg.norm(b - mg.coarse_apply(H.Dc, x, mu)) <= 0.1 * np.linalg.norm(b) * (1 + 1e-9)


def test_kcycle_f32_close_to_f64(given):
    ctx, H, U, p = given
    b = _c1(ctx, 147)
    x64 = ctx.kcycle(b, p.mu, 0, F64)
    x32 = ctx.kcycle(b, p.mu, 0, F32)
    assert rel(x32, x64) < 1e-4
    assert np.linalg.norm(b - mg.coarse_apply(H.Dc, x32, p.mu)) <= 0.1 * np.linalg.norm(b) * (1 + 1e-4)


def test_level2_setup_matches_oracle():
    ctx, H, U, p = build(n_init2=2, n_iter2=1)
    assert rel(ctx.get_vectors2(), H.L1.P2.W) < 1e-9
    x = _c2(ctx, 148)
    assert rel(ctx.coarse_apply2(x, p.mu, F64), mg.coarse_apply(H.L1.Dcc, x, p.mu)) < 1e-9


@pytest.mark.parametrize("method", [tmg.SOLVE_MG_F64, tmg.SOLVE_MG_MIXED])
def test_three_level_solve(method):
    ctx, H, U, p = build(prec_coarse=F64 if method == tmg.SOLVE_MG_F64 else F32, n_init=2, n_iter=1,
                         n_init2=2, n_iter2=1)
    b = fields.gaussian_spinor(DIMS, 149)
    x, st = ctx.solve(b, tol=1e-12, method=method)
    assert rel(dirac.apply_D(U, x, p, clover=H.clover), b) <= 1.5e-12
    xo, steps, res = H.solve(b, tol=1e-12)
    assert res <= 1e-12
    assert rel(x, xo) < 1e-8
    assert st["coarse_iterations"] > 0


@pytest.fixture(scope="module")
def given_tc():
    """N_v = 4 on both coarse levels (8 dofs per site), the smallest shape of the tensor-core apply."""
    return build(nv=4, nv2=4)


@pytest.mark.parametrize("mode", [2, 1, 0])
def test_kcycle_multi_columns(given_tc, mode):
    """The lock-step K-cycle (FP32, tensor-core applies on both coarse levels) for three columns with
    their own twists, each against the single-column FP64 K-cycle kernel (itself equal to the
    oracle's Level1 to 1e-10): the smoother's three GMRES steps (mode 2), one level-1 cycle (mode 1)
    and the K-cycle solve (mode 0, also to its relative residual target 0.1 on D_c)."""
    ctx, H, U, p = given_tc
    mus = [p.mu, -p.mu, 2.5 * p.mu]
    b = np.stack([_c1(ctx, 150 + j) for j in range(3)])
    x = ctx.kcycle_multi(b, mus, mode)
    for j, mu in enumerate(mus):
        want = ctx.kcycle(b[j], mu, mode, F64)
        assert rel(x[j], want) < (2e-5 if mode == 2 else 1e-4), (mode, j)
        if mode == 0:
            r = b[j] - mg.coarse_apply(H.Dc, x[j], mu)
            assert np.linalg.norm(r) <= 0.1 * np.linalg.norm(b[j]) * (1 + 1e-4), j
    if mode == 2:   # the smoother itself is the oracle's GMRES on D_c from zero
        for j, mu in enumerate(mus):
            assert rel(x[j], H.L1.smooth(b[j], np.zeros_like(b[j]), mu)) < 2e-5, j


def test_batched_three_level_solve_uses_lockstep_kcycle():
    """The three-level batched solve with the lock-step K-cycle: every column to a true FP64
    residual of 1e-10, each agreeing with its own single-column three-level solve."""
    ctx, H, U, p = build(prec_coarse=F32, n_init=2, n_iter=1, n_init2=2, n_iter2=1, nv=4, nv2=4)
    b = np.stack([fields.gaussian_spinor(DIMS, 160 + j) for j in range(3)])
    mus = [p.mu, -p.mu, 0.5 * p.mu]
    x, st = ctx.solve(b, tol=1e-10, method=tmg.SOLVE_MG_BATCHED, mu_per_col=mus)
    for j, mu in enumerate(mus):
        pj = dirac.Params(kappa=p.kappa, csw=p.csw, mu=mu, tbc=-1)
        assert rel(dirac.apply_D(U, x[j], pj, clover=H.clover), b[j]) <= 1.5e-10, j
        xs, _ = ctx.solve(b[j], tol=1e-10, method=tmg.SOLVE_MG_MIXED, mu_per_col=[mu])
        assert rel(x[j], xs) < 1e-8, j
