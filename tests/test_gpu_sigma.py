"""sigma_min(D_W) on the GPU (tmg_sigma_min: Lanczos on (D(mu_s)^dag D(mu_s))^-1 with two-step
solves) against the oracle's shift-invert Lanczos on the sparse Q = g5 D_W (scipy, a sparse LU), on
the same seeded field; with FP64 CG and with FP64 multigrid inner solves."""
import pytest

from oracle import dirac, kappa
from synth import fields

tmg = pytest.importorskip("paper_1710_06198_gb300")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method", [tmg.SOLVE_CG_F64, tmg.SOLVE_MG_F64])
@pytest.mark.parametrize("m0", [-0.3, -0.9])
def test_sigma_min_matches_sparse_shift_invert(method, m0):
    dims, block = (8, 4, 4, 4), (4, 2, 2, 2)
    U = fields.gauge_field(dims, 0.35, 140)
    p = dirac.Params(kappa=dirac.kappa_from_m0(m0), csw=1.5, tbc=-1)
    want = kappa.sigma_min(U, p)
    mu_s = 0.02
    ctx = tmg.Context(dims, block)
    ctx.set_params(p.kappa, p.csw, mu_s)
    ctx.load_gauge(U, -1)
    if method == tmg.SOLVE_MG_F64:
        prm = tmg.Context.mg_defaults()
        prm.nv, prm.n_init, prm.n_iter = 6, 3, 1
        prm.prec_fine, prm.prec_coarse = tmg.PREC_F64, tmg.PREC_F64
        ctx.setup(fields.gaussian_spinor(dims, 141, n=6), prm)
    sigma, rr, ns = ctx.sigma_min(fields.gaussian_spinor(dims, 142), mu_s, max_steps=64, rtol=1e-9, solve_tol=1e-12,
                                  method=method)
    assert rr <= 1e-9
    assert abs(sigma - want) <= 1e-6 * want, (sigma, want, ns)
