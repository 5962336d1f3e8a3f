"""GPU parity of the DD-alpha-AMG pieces (Eq. 1) and of the solves, through the C ABI, against the
FP64 oracle on the same seeded fields and the same initial test vectors.

* orthonormalised test vectors (P), P^dag, P, the coarse stencil D_c(mu), SAP sweeps and one
  preconditioner cycle: FP64 to <= 1e-11, FP32 to <= 1e-5 (SAP/cycle) and 1e-6 (P, P^dag, D_c);
* the adaptive setup in FP64 against the oracle's setup from the same random vectors;
* solves: FP64 multigrid, mixed-precision multigrid and FP64 CG reach a true FP64 residual
  <= 1e-10 measured with the oracle's own operator, and agree with the oracle's solution.
"""
import numpy as np
import pytest

from oracle import dirac, krylov, mg
from synth import fields
from tests.conftest import rel

tmg = pytest.importorskip("paper_1710_06198_gb300")
pytestmark = pytest.mark.gpu

F64, F32, F16 = tmg.PREC_F64, tmg.PREC_F32, tmg.PREC_F16


def build(dims, block, nv, eps, seed, m0=-0.25, csw=1.2, mu=0.05, sweeps=2, n_mr=3, coarse_m=20,
          coarse_rtol=0.0, prec_fine=F64, prec_coarse=F64, n_init=0, n_iter=0, restart=10):
    U = fields.gauge_field(dims, eps, seed)
    p = dirac.Params(kappa=dirac.kappa_from_m0(m0), csw=csw, mu=mu, tbc=-1)
    ctx = tmg.Context(dims, block)
    ctx.set_params(p.kappa, p.csw, p.mu)
    ctx.load_gauge(U, -1)
    prm = tmg.Context.mg_defaults()
    prm.nv, prm.sap_sweeps, prm.sap_mr = nv, sweeps, n_mr
    prm.coarse_m, prm.coarse_rtol = coarse_m, coarse_rtol
    prm.n_init, prm.n_iter, prm.restart = n_init, n_iter, restart
    prm.prec_fine, prm.prec_coarse = prec_fine, prec_coarse
    v0 = fields.gaussian_spinor(dims, seed + 100, n=nv)
    ctx.setup(v0, prm)
    mgp = mg.MGParams(block=block, agg=block, nv=nv, sap_sweeps=sweeps, sap_mr=n_mr, coarse_m=coarse_m,
                      coarse_rtol=coarse_rtol, n_init=n_init, n_iter=n_iter, restart=restart)
    H = mg.Hierarchy(U, p, mgp)
    if n_init == 0 and n_iter == 0:
        H.set_vectors(v0)
    else:
        H.setup(v0)
    return ctx, H, U, p


@pytest.fixture(scope="module")
def small():
    return build((8, 4, 4, 4), (4, 2, 2, 2), 3, 0.5, 31)


def test_prolongator_vectors(small):
    ctx, H, U, p = small
    assert rel(ctx.get_vectors(), H.P.W) < 1e-13


@pytest.mark.parametrize("prec", [F64, F32])
def test_restrict_prolong(small, prec):
    ctx, H, U, p = small
    r = fields.gaussian_spinor(ctx.dims, 32)
    tol = 1e-13 if prec == F64 else 1e-6
    assert rel(ctx.restrict(r, prec), mg.restrict(H.P, r)) < tol
    c = fields.gaussian_coarse((2, 2, 2, 2), 2 * ctx.nv, 33)
    assert rel(ctx.prolong(c, prec), mg.prolong(H.P, c)) < tol


@pytest.mark.parametrize("prec", [F64, F32])
def test_coarse_operator(small, prec):
    ctx, H, U, p = small
    x = fields.gaussian_coarse((2, 2, 2, 2), 2 * ctx.nv, 34)
    tol = 1e-12 if prec == F64 else 1e-6
    for mu in (0.0, p.mu, -0.3):
        assert rel(ctx.coarse_apply(x, mu, prec), mg.coarse_apply(H.Dc, x, mu)) < tol
    # and against the definition P^dag D P directly
    assert rel(ctx.coarse_apply(x, p.mu, F64), mg.coarse_apply_definition(U, p, H.clover, H.P, x)) < 1e-12


def test_coarse_operator_extent_three():
    """A coarse lattice with six sites along x separates the +mu and -mu stencil blocks."""
    ctx, H, U, p = build((24, 4, 4, 4), (4, 2, 2, 2), 2, 0.5, 35)
    clat = ctx.coarse_lat
    x = fields.gaussian_coarse((clat[3], clat[2], clat[1], clat[0]), 4, 36)
    assert rel(ctx.coarse_apply(x, 0.1, F64), mg.coarse_apply(H.Dc, x, 0.1)) < 1e-12


@pytest.mark.parametrize("prec", [F64, F32, F16])
def test_sap(small, prec):
    ctx, H, U, p = small
    b = fields.gaussian_spinor(ctx.dims, 37)
    x0 = fields.gaussian_spinor(ctx.dims, 38) * 0.1
    want = mg.sap(U, p, H.clover, b, ctx.block, 2, 3, x0=x0)
    tol = {F64: 1e-12, F32: 1e-5, F16: 5e-3}[prec]
    assert rel(ctx.sap(b, x0, prec), want) < tol


@pytest.mark.parametrize("prec", [F64, F32])
def test_coarse_solve(small, prec):
    """The coarse GMRES with rtol = 0 runs exactly coarse_m steps: the same Krylov solution as
    the oracle's (modified Gram-Schmidt there, classical with re-orthogonalisation here)."""
    ctx, H, U, p = small
    c = fields.gaussian_coarse((2, 2, 2, 2), 2 * ctx.nv, 42)
    want = H.coarse_solve(c, p.mu)
    tol = 1e-10 if prec == F64 else 1e-4
    assert rel(ctx.coarse_solve(c, p.mu, prec), want) < tol


@pytest.mark.parametrize("cache", [1, 0])
@pytest.mark.parametrize("overlap", [0, 1])
@pytest.mark.parametrize("passes", [1, 2])
def test_coarse_solve_launch_variants(small, overlap, passes, cache):
    """The persistent coarse GMRES with the Hessenberg update overlapped or not, one or two
    Gram-Schmidt passes, the own stencil blocks cached in shared memory or read from L2, and grids
    of 1, 3, 7 and 16 CTAs (ragged site ranges, several sites per CTA): every variant gives the
    oracle's Krylov solution."""
    ctx, H, U, p = small
    c = fields.gaussian_coarse((2, 2, 2, 2), 2 * ctx.nv, 43)
    want = H.coarse_solve(c, p.mu)
    try:
        ctx.tune("coarse_block_cache", cache)
        ctx.tune("coarse_overlap", overlap)
        ctx.tune("coarse_gs_passes", passes)
        for g in (1, 3, 7, 16):
            ctx.tune("coarse_grid", g)
            # one classical Gram-Schmidt pass loses a little orthogonality against the oracle's
            # modified Gram-Schmidt
            assert rel(ctx.coarse_solve(c, p.mu, F64), want) < (1e-10 if passes == 2 else 1e-8), (g, overlap, passes)
    finally:
        ctx.tune("coarse_grid", 0)
        ctx.tune("coarse_gs_passes", 0)
        ctx.tune("coarse_overlap", 1)
        ctx.tune("coarse_block_cache", 1)


@pytest.fixture(scope="module")
def nv8():
    return build((8, 8, 4, 4), (4, 4, 2, 2), 8, 0.5, 44, prec_fine=F32, prec_coarse=F32)


@pytest.mark.parametrize("tc", [1, 0])
def test_coarse_solve_multi(nv8, tc):
    """The batched coarse GMRES (rtol 0: exactly coarse_m lock-step steps) for 5 columns with their
    own twists, with D_c applied on the tensor cores (split TF32, all columns per launch) and by the
    CUDA-core kernel: every column is the oracle's Krylov solution to FP32 accuracy."""
    ctx, H, U, p = nv8
    c = fields.gaussian_coarse((2, 2, 2, 2), 2 * ctx.nv, 45, n=5)
    mus = [p.mu, -p.mu, 0.0, 0.2, -0.07]
    try:
        ctx.tune("batched_coarse_tc", tc)
        x = ctx.coarse_solve_multi(c, mus)
    finally:
        ctx.tune("batched_coarse_tc", 1)
    for j, m in enumerate(mus):
        assert rel(x[j], H.coarse_solve(c[j], m)) < 1e-4, j


@pytest.mark.parametrize("prec", [F64, F32])
def test_coarse_solve_odd_even(small, nv8, prec):
    """The coarse GMRES on the odd-even reduced system (Schur complement of the even sites; rtol 0:
    exactly coarse_m steps on S, then the even sites) against the oracle's odd-even coarse solve, on
    two operators and on grids of 1, 3, 7 and 16 CTAs (several sites of both parities per CTA)."""
    tol = 1e-10 if prec == F64 else 1e-4
    # the FP64 solve on the FP64-built context; the FP32 solve also on the FP32-built N_v = 8 one
    cases = ((small, 46),) if prec == F64 else ((small, 46), (nv8, 47))
    for case, seed in cases:
        ctx, H, U, p = case
        c = fields.gaussian_coarse((2, 2, 2, 2), 2 * ctx.nv, seed)
        for mu in (p.mu, -0.09):
            want = mg.coarse_solve_eo(H.Dc, c, mu, H.mg.coarse_m, 0.0)
            try:
                ctx.tune("coarse_eo", 1)
                for g in (1, 3, 7, 16):
                    ctx.tune("coarse_grid", g)
                    assert rel(ctx.coarse_solve(c, mu, prec), want) < tol, (g, mu)
            finally:
                ctx.tune("coarse_grid", 0)
                ctx.tune("coarse_eo", 0)


def test_mixed_solve_odd_even_coarse():
    """The mixed-precision solve with the odd-even coarse solve inside every cycle reaches 1e-10,
    measured with the oracle's operator, and agrees with the plain-coarse-solve solution."""
    ctx, H, U, p = build((8, 8, 8, 8), (4, 4, 2, 2), 4, 0.45, 48, prec_fine=F32, prec_coarse=F32, n_init=3, n_iter=1)
    b = fields.gaussian_spinor(ctx.dims, 49)
    x0, st0 = ctx.solve(b, tol=1e-12, method=tmg.SOLVE_MG_MIXED)
    try:
        ctx.tune("coarse_eo", 1)
        x1, st1 = ctx.solve(b, tol=1e-12, method=tmg.SOLVE_MG_MIXED)
    finally:
        ctx.tune("coarse_eo", 0)
    assert rel(dirac.apply_D(U, x1, p, clover=H.clover), b) <= 1e-12
    assert rel(x1, x0) < 1e-8
    assert st1["iterations"] <= st0["iterations"] + 1


def test_cycle_f64(small):
    ctx, H, U, p = small
    r = fields.gaussian_spinor(ctx.dims, 39)
    assert rel(ctx.cycle(r), H.cycle(r)) < 1e-11


def test_cycle_f32():
    ctx, H, U, p = build((8, 4, 4, 4), (4, 2, 2, 2), 3, 0.5, 31, prec_fine=F32, prec_coarse=F32)
    r = fields.gaussian_spinor(ctx.dims, 40)
    assert rel(ctx.cycle(r), H.cycle(r)) < 1e-4


def test_adaptive_setup_f64():
    ctx, H, U, p = build((8, 4, 4, 4), (4, 2, 2, 2), 3, 0.5, 41, n_init=2, n_iter=1)
    assert rel(ctx.get_vectors(), H.P.W) < 1e-9


@pytest.fixture(scope="module")
def solve_case():
    ctx, H, U, p = build((8, 8, 4, 4), (4, 4, 2, 2), 4, 0.4, 51, m0=-0.3, mu=0.02, sweeps=3, n_mr=4,
                         coarse_m=20, coarse_rtol=0.05, prec_fine=F32, prec_coarse=F32, n_init=3, n_iter=1)
    b = fields.gaussian_spinor(ctx.dims, 52)
    D = lambda v: dirac.apply_D(U, v, p, clover=H.clover)
    xo, _, _ = krylov.cg_normal(D, lambda v: dirac.apply_Ddag(U, v, p, clover=H.clover), b, tol=1e-13)
    return ctx, H, U, p, b, xo


@pytest.mark.parametrize("method", [tmg.SOLVE_MG_F64, tmg.SOLVE_MG_MIXED, tmg.SOLVE_CG_F64])
def test_solve(solve_case, method):
    ctx, H, U, p, b, xo = solve_case
    x, st = ctx.solve(b, tol=1e-12, method=method)
    res = rel(dirac.apply_D(U, x, p, clover=H.clover), b)
    assert res <= 1e-12 * 1.01 and st["true_residual"] <= 1e-12
    assert rel(x, xo) < 1e-9


def test_solve_1e10_and_multi_rhs(solve_case):
    ctx, H, U, p, b, xo = solve_case
    b2 = np.stack([b, fields.gaussian_spinor(ctx.dims, 53)])
    x, st = ctx.solve(b2, tol=1e-10, method=tmg.SOLVE_MG_MIXED, mu_per_col=[p.mu, -p.mu])
    for j, m in enumerate((p.mu, -p.mu)):
        assert rel(dirac.apply_D(U, x[j], p, mu=m, clover=H.clover), b2[j]) <= 1e-10


def test_solve_device_pointers(solve_case):
    torch = pytest.importorskip("torch")
    ctx, H, U, p, b, xo = solve_case
    x, st = ctx.solve(torch.from_numpy(b).cuda(), tol=1e-10, method=tmg.SOLVE_MG_MIXED)
    x = x.cpu().numpy()
    assert rel(dirac.apply_D(U, x, p, clover=H.clover), b) <= 1e-10


def test_solve_reports_noconv(solve_case):
    ctx, H, U, p, b, xo = solve_case
    x, st = ctx.solve(b, tol=1e-12, method=tmg.SOLVE_CG_F64, maxiter=2, check=False)
    assert st["true_residual"] > 1e-12
    with pytest.raises(tmg.TmgError) as e:
        ctx.solve(b, tol=1e-12, method=tmg.SOLVE_CG_F64, maxiter=2)
    assert e.value.code == -4


def test_solve_rejects_nan(solve_case):
    ctx, H, U, p, b, xo = solve_case
    bad = b.copy()
    bad[0, 0, 0, 0, 0, 0] = np.nan
    with pytest.raises(tmg.TmgError) as e:
        ctx.solve(bad, tol=1e-10, method=tmg.SOLVE_MG_MIXED)
    assert e.value.code == -5


@pytest.mark.parametrize("nv", [4, 8, 16])
def test_coarse_solve_f32_vector_stencil(nv):
    """FP32 coarse GMRES for N_v whose block rows are read two at a time (float4 tiles split over
    lane groups), against the oracle's GMRES with the same fixed step count."""
    dims, block = (8, 8, 4, 4), (4, 4, 2, 2)
    U = fields.gauge_field(dims, 0.5, 230)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.25), csw=1.2, mu=0.05, tbc=-1)
    ctx = tmg.Context(dims, block)
    ctx.set_params(p.kappa, p.csw, p.mu)
    ctx.load_gauge(U, -1)
    prm = tmg.Context.mg_defaults()
    prm.nv, prm.n_init, prm.n_iter, prm.coarse_m, prm.coarse_rtol = nv, 0, 0, 12, 0.0
    prm.prec_fine, prm.prec_coarse = F32, F32
    v0 = fields.gaussian_spinor(dims, 231, n=nv)
    ctx.setup(v0, prm)
    H = mg.Hierarchy(U, p, mg.MGParams(block=block, agg=block, nv=nv, coarse_m=12, coarse_rtol=0.0))
    H.set_vectors(v0)
    c = fields.gaussian_coarse((2, 2, 2, 2), 2 * nv, 232)
    assert rel(ctx.coarse_solve(c, p.mu, F32), H.coarse_solve(c, p.mu)) < 1e-4
