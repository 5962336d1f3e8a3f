"""GPU parity of the multigrid pieces at the shapes the workloads run: 4^4 SAP blocks and
aggregates (256-site CTAs, two per SM), N_v = 16 and 24 on level 1, and the tensor-core coarse
operator at N_v = 24 and 32 (the level-1 and level-2 dof counts 48 and 64 of the three-level
workloads) with 20 columns.

Tolerances (relative L2 over the whole field, plus a per-site maximum for FP16):
* FP64 1e-12;
* FP32 operator-like maps (P, P^dag, D_c, one SAP sweep chain of fixed length): 1e-6 for P, P^dag
  and D_c, whose results are sums of at most 9 * 2 N_v products; the SAP bound is derived in the
  design notes (relative error ~ eps_32 x the number of chained block operator applications x the
  block solve's amplification) and the test asserts the measured value under it;
* FP16 storage (links and clover fixed point, 15-bit mantissa): 5e-3 whole-field and 2.5e-2 for the
  largest per-site error against the RMS site norm.
"""
import numpy as np
import pytest

from oracle import dirac, mg
from synth import fields
from tests.conftest import rel, site_rel_max

tmg = pytest.importorskip("paper_1710_06198_gb300")
pytestmark = pytest.mark.gpu

F64, F32, F16 = tmg.PREC_F64, tmg.PREC_F32, tmg.PREC_F16
DIMS, BLOCK = (8, 8, 8, 8), (4, 4, 4, 4)


def _case(nv, seed):
    U = fields.gauge_field(DIMS, 0.35, seed)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.5), csw=1.5, mu=0.003, tbc=-1)
    ctx = tmg.Context(DIMS, BLOCK)
    ctx.set_params(p.kappa, p.csw, p.mu)
    ctx.load_gauge(U, -1)
    prm = tmg.Context.mg_defaults()
    prm.nv, prm.n_init, prm.n_iter, prm.sap_sweeps, prm.sap_mr = nv, 0, 0, 3, 4
    prm.coarse_m, prm.coarse_rtol = 20, 0.0
    prm.prec_fine, prm.prec_coarse = F64, F64   # FP64 test vectors; each call picks its precision
    v0 = fields.gaussian_spinor(DIMS, seed + 100, n=nv)
    ctx.setup(v0, prm)
    H = mg.Hierarchy(U, p, mg.MGParams(block=BLOCK, agg=BLOCK, nv=nv, sap_sweeps=3, sap_mr=4, coarse_m=20,
                                       coarse_rtol=0.0))
    H.set_vectors(v0)
    return ctx, H, U, p


@pytest.fixture(scope="module", params=[16, 24])
def case(request):
    return _case(request.param, 300 + request.param)


def test_vectors_restrict_prolong(case):
    ctx, H, U, p = case
    assert rel(ctx.get_vectors(), H.P.W) < 1e-13
    r = fields.gaussian_spinor(DIMS, 401)
    c = fields.gaussian_coarse((2, 2, 2, 2), 2 * ctx.nv, 402)
    for prec, tol in ((F64, 1e-13), (F32, 1e-6)):
        assert rel(ctx.restrict(r, prec), mg.restrict(H.P, r)) < tol
        assert rel(ctx.prolong(c, prec), mg.prolong(H.P, c)) < tol


def test_coarse_operator(case):
    ctx, H, U, p = case
    x = fields.gaussian_coarse((2, 2, 2, 2), 2 * ctx.nv, 403)
    for prec, tol in ((F64, 1e-12), (F32, 1e-6)):
        for mu in (0.0, p.mu):
            assert rel(ctx.coarse_apply(x, mu, prec), mg.coarse_apply(H.Dc, x, mu)) < tol
    assert rel(ctx.coarse_apply(x, p.mu, F64), mg.coarse_apply_definition(U, p, H.clover, H.P, x)) < 1e-12


@pytest.mark.parametrize("prec", [F64, F32, F16])
def test_sap_256_site_blocks(case, prec):
    """k = 3 sweeps of n_MR = 4 steps on 256-site blocks from a nonzero start."""
    ctx, H, U, p = case
    b = fields.gaussian_spinor(DIMS, 404)
    x0 = 0.1 * fields.gaussian_spinor(DIMS, 405)
    want = mg.sap(U, p, H.clover, b, BLOCK, 3, 4, x0=x0)
    got = ctx.sap(b, x0, prec)
    err = rel(got, want)
    tol = {F64: 1e-12, F32: 2e-6, F16: 5e-3}[prec]
    assert err < tol, err
    if prec == F16:
        assert site_rel_max(got, want) < 2.5e-2


@pytest.mark.parametrize("prec", [F32, F16])
def test_dslash_per_site_maximum(case, prec):
    """Whole-field and per-site error of D at 8^4: no site (block face, time boundary) is off."""
    ctx, H, U, p = case
    x = fields.gaussian_spinor(DIMS, 406)
    want = dirac.apply_D(U, x, p, clover=H.clover)
    got = ctx.apply(x, tmg.OP_D, prec)
    assert rel(got, want) < {F32: 1e-6, F16: 5e-3}[prec]
    assert site_rel_max(got, want) < {F32: 5e-6, F16: 2.5e-2}[prec]


@pytest.mark.parametrize("nv", [24, 32])
def test_tensor_core_coarse_apply_workload_dofs(nv):
    """tcgen05 multi-RHS D_c at the three-level workloads' dof counts (48, 64), 20 columns."""
    dims, block = (8, 8, 4, 4), (4, 4, 2, 2)
    U = fields.gauge_field(dims, 0.3, 410 + nv)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.5), csw=1.6, mu=0.002, tbc=-1)
    ctx = tmg.Context(dims, block)
    ctx.set_params(p.kappa, p.csw, p.mu)
    ctx.load_gauge(U, -1)
    prm = tmg.Context.mg_defaults()
    prm.nv, prm.n_init, prm.n_iter = nv, 0, 0
    v0 = fields.gaussian_spinor(dims, 420 + nv, n=nv)
    ctx.setup(v0, prm)
    H = mg.Hierarchy(U, p, mg.MGParams(block=block, agg=block, nv=nv))
    H.set_vectors(v0)
    clat = ctx.coarse_lat
    x = fields.gaussian_coarse((clat[3], clat[2], clat[1], clat[0]), 2 * nv, 430 + nv, n=20)
    mus = np.concatenate([np.full(12, p.mu), np.sqrt(p.mu ** 2 + np.logspace(-5, -1, 8))])
    y = ctx.coarse_apply_multi(x, mus)
    for j in range(20):
        assert rel(y[j], mg.coarse_apply(H.Dc, x[j], mus[j])) < 2e-6, j
