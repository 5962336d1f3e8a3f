"""GPU parity of the even-odd reduced operator Dhat = M_o - H_oe M_e^-1 H_eo (Sec. 1.2 runs on the
even-odd reduced operator) and of the odd-even CG (Fig. 1's comparator) against the oracle:

* Dhat and Dhat^dag through tmg_apply: FP64 (12-real links) to 1e-13, FP32 (8-real links, FP32
  clover inverse) to 1e-6 whole-field and 5e-6 per site, with and without the bulk-copy staging of
  the clover stream, several twists, periodic and antiperiodic time;
* the odd-even CG reaches the full system's 1e-12 residual (oracle operator) and the oracle's
  solution, at the 8^4 workload shape too.
"""
import numpy as np
import pytest

from oracle import dirac, eo, krylov
from synth import fields
from tests.conftest import rel, site_rel_max

tmg = pytest.importorskip("paper_1710_06198_gb300")
pytestmark = pytest.mark.gpu


def _make(dims, block, seed, m0=-0.3, csw=1.4, mu=0.05, tbc=-1):
    U = fields.gauge_field(dims, 0.4, seed)
    p = dirac.Params(kappa=dirac.kappa_from_m0(m0), csw=csw, mu=mu, tbc=tbc)
    ctx = tmg.Context(dims, block)
    ctx.set_params(p.kappa, p.csw, p.mu)
    ctx.load_gauge(U, tbc)
    return ctx, U, p, dirac.clover_term(U, p.csw)


@pytest.mark.parametrize("stage", [1, 0])
@pytest.mark.parametrize("tbc", [-1, 1])
def test_schur_operator_matches_oracle(stage, tbc):
    dims = (8, 4, 4, 8)
    ctx, U, p, C = _make(dims, (4, 2, 2, 4), 150, tbc=tbc)
    ctx.tune("eo_stage", stage)
    par = eo.parity(fields.lattice_shape(dims))
    x = eo.restrict_parity(fields.gaussian_spinor(dims, 151), par, 1)
    for mu in (p.mu, -0.2):
        want = eo.schur_apply(U, x, p, mu, C)
        wantd = eo.schur_apply_dag(U, x, p, mu, C)
        for prec, tol, stol in ((tmg.PREC_F64, 1e-13, 1e-12), (tmg.PREC_F32, 1e-6, 5e-6)):
            got = ctx.apply(x, tmg.OP_DHAT, prec, mu_per_col=[mu])
            assert rel(got, want) < tol, (prec, mu)
            assert site_rel_max(got, want) < stol
            assert np.abs(got[par == 0]).max() == 0.0
            gotd = ctx.apply(x, tmg.OP_DHAT_DAG, prec, mu_per_col=[mu])
            assert rel(gotd, wantd) < tol, (prec, mu)


def test_schur_operator_8x4_blocks():
    """The workloads' 4^4-block shape (8^4), FP32 8-real links."""
    dims = (8, 8, 8, 8)
    ctx, U, p, C = _make(dims, (4, 4, 4, 4), 152, m0=-0.5, csw=1.5, mu=0.003)
    par = eo.parity(fields.lattice_shape(dims))
    x = eo.restrict_parity(fields.gaussian_spinor(dims, 153), par, 1)
    want = eo.schur_apply(U, x, p, p.mu, C)
    got = ctx.apply(x, tmg.OP_DHAT, tmg.PREC_F32)
    assert rel(got, want) < 1e-6
    assert site_rel_max(got, want) < 5e-6


@pytest.mark.parametrize("dims,block", [((8, 4, 4, 8), (4, 2, 2, 4)), ((8, 8, 8, 8), (4, 4, 4, 4))])
def test_odd_even_cg(dims, block):
    ctx, U, p, C = _make(dims, block, 154, m0=-0.3, mu=0.02)
    b = fields.gaussian_spinor(dims, 155)
    x, st = ctx.solve(b, tol=1e-12, method=tmg.SOLVE_CG_EO, maxiter=20000)
    assert rel(dirac.apply_D(U, x, p, clover=C), b) <= 1e-12 * 1.01
    x_full, st_full = ctx.solve(b, tol=1e-12, method=tmg.SOLVE_CG_F64, maxiter=20000)
    assert rel(x, x_full) < 1e-9
    assert st["iterations"] < st_full["iterations"]
