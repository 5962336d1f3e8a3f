"""GPU parity of the doublet multigrid (Eq. 2 with P_ND = P x I2, Sec. 1.2) through the C ABI,
against the FP64 oracle (oracle/nd.py) on the same seeded fields and test vectors:

* SAP on D_ND, D_ND,c, the doublet coarse GMRES and one doublet cycle: FP64 to 1e-10..1e-12, FP32
  to 1e-5..1e-6;
* the level-1 doublet K-cycle kernel (smoother, cycle, solve) in FP64 against oracle Level1ND;
* two- and three-level doublet solves (FP64 and mixed) to a true FP64 residual of 1e-12 (computed
  with the oracle's D_ND), agreeing with the oracle's doublet solve.
"""
import numpy as np
import pytest

from oracle import dirac, krylov, mg, nd
from synth import fields
from tests.conftest import rel

tmg = pytest.importorskip("paper_1710_06198_gb300")
pytestmark = pytest.mark.gpu

F64, F32, F16 = tmg.PREC_F64, tmg.PREC_F32, tmg.PREC_F16

DIMS, BLOCK = (16, 8, 8, 8), (4, 2, 2, 2)
NV, NV2, AGG2 = 3, 4, (2, 2, 2, 2)


def build(prec=F64, levels=2, coarse_rtol=0.0, coarse_m=20, n_init=0, n_iter=0, n_init2=0, n_iter2=0):
    U = fields.gauge_field(DIMS, 0.45, 180)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.3), csw=1.1, mu=0.12, tbc=-1, mubar=0.12, epsbar=0.13)
    ctx = tmg.Context(DIMS, BLOCK)
    ctx.set_params(p.kappa, p.csw, p.mu, p.mubar, p.epsbar)
    ctx.load_gauge(U, -1)
    prm = tmg.Context.mg_defaults()
    prm.nv, prm.sap_sweeps, prm.sap_mr = NV, 2, 3
    prm.coarse_m, prm.coarse_rtol = coarse_m, coarse_rtol
    prm.n_init, prm.n_iter, prm.restart = n_init, n_iter, 10
    prm.prec_fine, prm.prec_coarse = prec, (F64 if prec == F64 else F32)
    v0 = fields.gaussian_spinor(DIMS, 181, n=NV)
    ctx.setup(v0, prm)
    mgp = mg.MGParams(block=BLOCK, agg=BLOCK, nv=NV, sap_sweeps=2, sap_mr=3, coarse_m=coarse_m,
                      coarse_rtol=coarse_rtol, n_init=n_init, n_iter=n_iter, restart=10)
    H = mg.Hierarchy(U, p, mgp)
    if n_init == 0 and n_iter == 0:
        H.set_vectors(v0)
    else:
        H.setup(v0)
    L1 = None
    if levels == 3:
        c1 = ctx.coarse_lat
        v1 = fields.gaussian_coarse((c1[3], c1[2], c1[1], c1[0]), 2 * NV, 182, n=NV2)
        q = tmg.Context.level2_defaults()
        q.agg[:] = AGG2
        q.nv, q.coarse_rtol, q.n_init, q.n_iter = NV2, 5e-2, n_init2, n_iter2
        ctx.setup_level2(v1, q)
        L1 = mg.Level1(H.Dc, mg.MGParams3(agg2=AGG2, nv2=NV2, coarse_rtol=5e-2, n_init=n_init2, n_iter=n_iter2))
        if n_init2 == 0 and n_iter2 == 0:
            L1.set_vectors(v1)
        else:
            L1.setup(v1, p.mu)
    return ctx, nd.HierarchyND(H, L1), U, p


@pytest.fixture(scope="module")
def two():
    return build()


def _coarse2(ctx, seed):
    c1 = ctx.coarse_lat
    return fields.gaussian_coarse((c1[3], c1[2], c1[1], c1[0]), 2 * NV, seed, n=2)


@pytest.mark.parametrize("prec,tol", [(F64, 1e-11), (F32, 1e-5), (F16, 5e-3)])
def test_sap_nd(two, prec, tol):
    ctx, HN, U, p = two
    b = fields.gaussian_spinor(DIMS, 183, n=2)
    x0 = fields.gaussian_spinor(DIMS, 184, n=2)
    want = HN.smooth(b, x0)
    assert rel(ctx.sap_nd(b, x0, prec), want) < tol


@pytest.mark.parametrize("prec,tol", [(F64, 1e-12), (F32, 1e-6)])
def test_coarse_doublet_operator(two, prec, tol):
    ctx, HN, U, p = two
    x = _coarse2(ctx, 185)
    assert rel(ctx.coarse_apply_nd(x, prec), mg.coarse_apply_nd(HN.H.Dc, x, p.mubar, p.epsbar)) < tol


def test_coarse_doublet_gmres_and_cycle(two):
    ctx, HN, U, p = two
    c = _coarse2(ctx, 186)
    want, _ = krylov.gmres_fixed(HN.coarse_apply, c, 20, 0.0)
    assert rel(ctx.coarse_solve_nd(c, F64), want) < 1e-10
    r = fields.gaussian_spinor(DIMS, 187, n=2)
    assert rel(ctx.cycle_nd(r), HN.cycle(r)) < 1e-10


def test_coarse_doublet_gmres_f32_vector_stencil():
    """FP32 doublet coarse GMRES with N_v = 4 (block rows read two at a time, flavour mixing added
    by the lane group that writes the row) against the oracle's GMRES, fixed step count."""
    dims, block = (8, 8, 4, 4), (4, 4, 2, 2)
    U = fields.gauge_field(dims, 0.45, 233)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.3), csw=1.1, mu=0.12, tbc=-1, mubar=0.12, epsbar=0.13)
    ctx = tmg.Context(dims, block)
    ctx.set_params(p.kappa, p.csw, p.mu, p.mubar, p.epsbar)
    ctx.load_gauge(U, -1)
    prm = tmg.Context.mg_defaults()
    prm.nv, prm.n_init, prm.n_iter, prm.coarse_m, prm.coarse_rtol = 4, 0, 0, 12, 0.0
    prm.prec_fine, prm.prec_coarse = F32, F32
    v0 = fields.gaussian_spinor(dims, 234, n=4)
    ctx.setup(v0, prm)
    H = mg.Hierarchy(U, p, mg.MGParams(block=block, agg=block, nv=4, coarse_m=12, coarse_rtol=0.0))
    H.set_vectors(v0)
    HN = nd.HierarchyND(H)
    c = fields.gaussian_coarse((2, 2, 2, 2), 8, 235, n=2)
    want, _ = krylov.gmres_fixed(HN.coarse_apply, c, 12, 0.0)
    assert rel(ctx.coarse_solve_nd(c, F32), want) < 1e-4


@pytest.mark.parametrize("method", [tmg.SOLVE_ND_F64, tmg.SOLVE_ND_MIXED])
def test_two_level_doublet_solve(method):
    ctx, HN, U, p = build(prec=F64 if method == tmg.SOLVE_ND_F64 else F32, coarse_rtol=5e-2, coarse_m=30,
                          n_init=2, n_iter=1)
    b = fields.gaussian_spinor(DIMS, 188, n=2)
    x, st = ctx.solve(b, tol=1e-12, method=method)
    assert x.shape == b.shape
    assert rel(dirac.apply_DND(U, x, p, HN.H.clover), b) <= 1.5e-12
    xo, steps, res = HN.solve(b, tol=1e-12)
    assert res <= 1e-12
    assert rel(x, xo) < 1e-8


@pytest.mark.parametrize("overlap", [1, 0])
def test_level1_doublet_kcycle(overlap):
    """Smoother, one level-1 cycle and the K-cycle solve of the doublet, with the Hessenberg update
    of the persistent GMRES overlapped with the next stencil and after it; FP64 takes two
    Gram-Schmidt passes per step, so this also covers partials written by one pass while other
    CTAs still read the previous pass's."""
    ctx, HN, U, p = build(levels=3, coarse_rtol=5e-2, coarse_m=30)
    ctx.tune("coarse_overlap", overlap)
    b = _coarse2(ctx, 189)
    L = HN.L1
    assert rel(ctx.kcycle_nd(b, 2, F64), L.smooth(b, np.zeros_like(b))) < 1e-10
    assert rel(ctx.kcycle_nd(b, 1, F64), L.cycle(b)) < 1e-10
    assert rel(ctx.kcycle_nd(b, 0, F64), L.solve(b)) < 1e-10


@pytest.mark.parametrize("method", [tmg.SOLVE_ND_F64, tmg.SOLVE_ND_MIXED])
def test_three_level_doublet_solve(method):
    ctx, HN, U, p = build(prec=F64 if method == tmg.SOLVE_ND_F64 else F32, levels=3, coarse_rtol=5e-2,
                          coarse_m=30, n_init=2, n_iter=1, n_init2=2, n_iter2=1)
    b = fields.gaussian_spinor(DIMS, 190, n=2)
    x, st = ctx.solve(b, tol=1e-12, method=method)
    assert rel(dirac.apply_DND(U, x, p, HN.H.clover), b) <= 1.5e-12
    xo, steps, res = HN.solve(b, tol=1e-12)
    assert res <= 1e-12
    assert rel(x, xo) < 1e-8


@pytest.mark.parametrize("levels", [2, 3])
def test_shifted_doublet_pieces_and_solve(levels):
    """The shifted doublet D_ND + i delta (G5 x tau1) of the rational approximation's systems
    (Sec. 3): fine operator, SAP, coarse operator and coarse solve (or K-cycle) in FP64 against the
    oracle with the same delta, and a mixed-precision doublet solve to 1e-12 with the oracle's
    operator as the reference."""
    import dataclasses
    ctx, HN, U, p = build(levels=levels)
    delta = 0.04
    ps = dataclasses.replace(p, ndshift=delta)
    HN.H.p = ps
    HN.p = ps
    if HN.L1 is not None:
        HN.L1.delta = delta
    ctx.set_ndshift(delta)
    C = HN.H.clover
    x2 = fields.gaussian_spinor(DIMS, 190, flavours=2)
    assert rel(ctx.apply(x2, tmg.OP_DND, F64), dirac.apply_DND(U, x2, ps, C)) < 1e-13
    b2 = fields.gaussian_spinor(DIMS, 191, flavours=2)
    assert rel(ctx.sap_nd(b2, 0.1 * x2, F64), HN.smooth(b2, 0.1 * x2)) < 1e-11
    c1 = ctx.coarse_lat
    xc = fields.gaussian_coarse((c1[3], c1[2], c1[1], c1[0]), 2 * NV, 192, n=2)
    assert rel(ctx.coarse_apply_nd(xc, F64), HN.coarse_apply(xc)) < 1e-12
    if levels == 3:
        assert rel(ctx.kcycle_nd(xc, 0, F64), HN.coarse_solve(xc)) < 1e-9
    else:
        assert rel(ctx.coarse_solve_nd(xc, F64), HN.coarse_solve(xc)) < 1e-10
    x, st = ctx.solve(b2, tol=1e-12, method=tmg.SOLVE_ND_MIXED)
    assert rel(dirac.apply_DND(U, x, ps, C), b2) <= 1e-12
    ctx.set_ndshift(0.0)
    assert rel(ctx.apply(x2, tmg.OP_DND, F64), dirac.apply_DND(U, x2, p, C)) < 1e-13
