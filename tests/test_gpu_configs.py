"""Full-size GPU checks of the five synthetic workloads (lattices, fields, operator and multigrid
parameters of ``synth/workloads.py``), in the launch configurations bench.py uses.

At these sizes the oracle cannot solve, so parity is checked on what it can compute:
* the 8^4 FP64 workload is small enough for the oracle's CG and its own two-level DD-alpha-AMG:
  both GPU solves (FP64 multigrid, FP64 CG) agree with both oracle solves;
* elsewhere the operator is compared with the oracle site by site on sampled sites (tests.sampled),
  and solutions are checked by their true residual, computed with the oracle's operator on the
  whole lattice where that is affordable (16^3 x 32, 16^4) and with the GPU FP64 operator (itself
  compared site by site with the oracle at the same size) on 24^3 x 48;
* the force on 16^4 (FP64 force kernels, mixed-precision solves) against central finite
  differences of the action (32 random su(3) directions, step 1e-5), each action from a multigrid solve on the rotated field warm-started from
  the solution on the unrotated field.
"""
import numpy as np
import pytest

from oracle import dirac, krylov, mg
from synth import fields, workloads
from tests import sampled
from tests.conftest import rel

tmg = pytest.importorskip("paper_1710_06198_gb300")
pytestmark = pytest.mark.gpu

F64, F32, F16 = tmg.PREC_F64, tmg.PREC_F32, tmg.PREC_F16


def _params(name):
    w = workloads.WORKLOADS[name]
    kappa, _ = workloads.kappa(name)
    return w, dirac.Params(kappa=kappa, csw=w["csw"], mu=w["mu"], tbc=-1, mubar=w.get("mubar", 0.0),
                           epsbar=w.get("epsbar", 0.0))


def _context(w, U, p, prec_fine, prec_coarse, n_init=5, n_iter=3):
    ctx = tmg.Context(w["dims"], w["block"])
    ctx.set_params(p.kappa, p.csw, p.mu, p.mubar, p.epsbar)
    ctx.load_gauge(U, -1)
    prm = tmg.Context.mg_defaults()
    prm.nv, prm.restart, prm.n_init, prm.n_iter = w["nv"], w["restart"], n_init, n_iter
    prm.sap_mr = w.get("sap_mr", prm.sap_mr)
    prm.coarse_m = w.get("coarse_m", prm.coarse_m)
    ctx.tune("coarse_eo", w.get("coarse_eo", 0))
    prm.prec_fine, prm.prec_coarse = prec_fine, prec_coarse
    ctx.setup(fields.gaussian_spinor(w["dims"], w["seed"] + 100, n=w["nv"]), prm)
    return ctx, prm


def _sampled_operator(ctx, U, p, dims, seed, precs=((F64, 1e-13), (F32, 1e-6), (F16, 5e-3))):
    x = fields.gaussian_spinor(dims, seed)
    sites = sampled.random_sites(dims, 24, seed + 1)
    want = sampled.apply_D_at(U, x, p, dims, sites)
    for prec, tol in precs:
        got = sampled.values_at(ctx.apply(x, prec=prec), sites)
        assert rel(got, want) < tol, prec


def test_plain_fp64_8x8x8x8():
    name = "tm_clover_8x8x8x8_fp64_2lvl"
    w, p = _params(name)
    dims = w["dims"]
    U = fields.gauge_field(dims, w["eps"], w["seed"])
    b = fields.gaussian_spinor(dims, w["rhs_seed"])
    ctx, prm = _context(w, U, p, F64, F64)
    x_mg, st = ctx.solve(b, tol=1e-12, method=tmg.SOLVE_MG_F64)
    x_cg, st_cg = ctx.solve(b, tol=1e-12, method=tmg.SOLVE_CG_F64, maxiter=200000)
    clover = dirac.clover_term(U, p.csw)
    D = lambda v: dirac.apply_D(U, v, p, clover=clover)
    Dd = lambda v: dirac.apply_Ddag(U, v, p, clover=clover)
    assert rel(D(x_mg), b) <= 1.5e-12
    assert rel(D(x_cg), b) <= 1.5e-12
    xo_cg, _, res_cg = krylov.cg_normal(D, Dd, b, tol=1e-12)
    H = mg.Hierarchy(U, p, mg.MGParams(block=w["block"], agg=w["block"], nv=w["nv"], restart=w["restart"]), clover)
    H.setup(fields.gaussian_spinor(dims, w["seed"] + 100, n=w["nv"]))
    xo_mg, _, res_mg = H.solve(b, tol=1e-12)
    assert res_cg <= 1e-12 and res_mg <= 1e-12
    assert rel(xo_mg, xo_cg) < 1e-8
    assert rel(x_mg, xo_cg) < 1e-8
    assert rel(x_cg, xo_cg) < 1e-8
    assert st["iterations"] < st_cg["iterations"]


@pytest.mark.parametrize("prec_fine", [F32, F16])
def test_mixed_16x16x16x32(prec_fine):
    name = "tm_clover_16x16x16x32_mixed_2lvl"
    w, p = _params(name)
    dims = w["dims"]
    U = fields.gauge_field(dims, w["eps"], w["seed"])
    b = fields.gaussian_spinor(dims, w["rhs_seed"])
    ctx, prm = _context(w, U, p, prec_fine, F32)
    if prec_fine == F32:
        _sampled_operator(ctx, U, p, dims, 160)
    x, st = ctx.solve(b, tol=1e-10, method=tmg.SOLVE_MG_MIXED)
    assert rel(dirac.apply_D(U, x, p), b) <= 1.01e-10
    assert st["refinements"] >= 1


def test_batched_three_level_24x24x24x48():
    name = "tm_clover_24x24x24x48_batched_3lvl"
    w, p = _params(name)
    dims = w["dims"]
    U = fields.gauge_field(dims, w["eps"], w["seed"])
    ctx, prm = _context(w, U, p, F32, F32)
    _sampled_operator(ctx, U, p, dims, 161, precs=((F64, 1e-13), (F32, 1e-6)))
    q = workloads.level2_params(w, tmg.Context.level2_defaults())
    c1 = ctx.coarse_lat
    ctx.setup_level2(fields.gaussian_coarse((c1[3], c1[2], c1[1], c1[0]), 2 * w["nv"], w["seed"] + 200, n=w["nv2"]), q)
    # 12 point sources D(mu) x = b, and the first step D(-mu_k) y = g5 phi of the 8 shifted systems
    # (D^dag D + sigma_k) x = phi = D^dag(mu_k) D(mu_k) x with mu_k = sqrt(mu^2 + sigma_k)
    sig = workloads.shifts(w["n_shifts"])
    mu_k = [np.sqrt(p.mu ** 2 + s) for s in sig]
    phi = fields.gaussian_spinor(dims, w["phi_seed"])
    g5phi = dirac.apply_g5(phi)
    ps = fields.point_sources(dims)
    b1 = np.concatenate([ps, np.broadcast_to(g5phi, (len(sig),) + g5phi.shape)])
    b1 = np.ascontiguousarray(b1)
    mus1 = [p.mu] * len(ps) + [-m for m in mu_k]
    x1, st1 = ctx.solve(b1, tol=1e-10, method=tmg.SOLVE_MG_BATCHED, mu_per_col=mus1)
    y = x1[len(ps):]
    b2 = np.ascontiguousarray(dirac.apply_g5(y))
    x2, st2 = ctx.solve(b2, tol=1e-10, method=tmg.SOLVE_MG_BATCHED, mu_per_col=mu_k)
    # true residuals with the GPU FP64 operator (compared with the oracle site by site above)
    r1 = ctx.apply(x1, prec=F64, mu_per_col=mus1) - b1
    for c in range(len(mus1)):
        assert np.linalg.norm(r1[c]) <= 1.01e-10 * np.linalg.norm(b1[c]), c
    r2 = ctx.apply(x2, prec=F64, mu_per_col=mu_k) - b2
    for c in range(len(mu_k)):
        assert np.linalg.norm(r2[c]) <= 1.01e-10 * np.linalg.norm(b2[c]), c
    # one point source and one shifted system with the oracle's operator on the whole lattice
    clover = dirac.clover_term(U, p.csw)
    assert rel(dirac.apply_D(U, x1[0], p, clover=clover), b1[0]) <= 1.01e-10
    k = len(sig) - 1
    lhs = dirac.apply_Ddag(U, dirac.apply_D(U, x2[k], p, clover=clover), p, clover=clover) + sig[k] * x2[k]
    assert rel(lhs, phi) < 1e-8


def test_force_16x16x16x16_finite_differences():
    name = "tm_clover_16x16x16x16_force"
    w, p = _params(name)
    dims = w["dims"]
    U = fields.gauge_field(dims, w["eps"], w["seed"])
    phi = fields.gaussian_spinor(dims, w["phi_seed"])
    ctx, prm = _context(w, U, p, F32, F32)
    S, F, st = ctx.force(phi, tol=1e-12)
    y0, _ = ctx.solve(phi, tol=1e-12, method=tmg.SOLVE_MG_MIXED)
    W = ctx.get_vectors()
    prm0 = tmg.Context.mg_defaults()
    prm0.nv, prm0.restart, prm0.n_init, prm0.n_iter = w["nv"], w["restart"], 0, 0
    prm0.prec_fine, prm0.prec_coarse = F32, F32

    def action(Ur):
        # warm start from the base solution: y = y0 + D(U_r)^-1 (phi - D(U_r) y0), so the solve
        # error scales with the O(h) correction rather than with y
        ctx.load_gauge(Ur, -1)
        ctx.setup(W, prm0)                        # the base test vectors, re-orthonormalised
        r = phi - ctx.apply(y0, prec=F64)
        d, _ = ctx.solve(r, tol=1e-13, method=tmg.SOLVE_MG_MIXED)
        y = y0 + d
        return float(np.vdot(y.ravel(), y.ravel()).real)

    from oracle import force
    h = 1e-5
    for om in fields.su3_algebra_directions(dims, w["seed"] + 2000, 32):
        H = force.algebra_to_matrix(om)
        ev, V = np.linalg.eigh(H)
        Vh = np.conj(np.swapaxes(V, -1, -2))
        rot = lambda t: ((V * np.exp(1j * t * ev)[..., None, :]) @ Vh) @ U
        fd = (action(rot(h)) - action(rot(-h))) / (2 * h)
        an = float(np.real(np.einsum("...ab,...ba->...", H, F).sum()))
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def test_doublet_three_level_48x48x48x96():
    """The largest workload: D_ND (Eq. 2) on 48^3 x 96, three-level doublet multigrid, 8 right-hand
    sides solved one after another to 1e-10, with the device memory in use recorded."""
    torch = pytest.importorskip("torch")
    name = "nd_clover_48x48x48x96_3lvl"
    w, p = _params(name)
    dims = w["dims"]
    U = fields.gauge_field(dims, w["eps"], w["seed"])
    ctx = tmg.Context(dims, w["block"])
    ctx.set_params(p.kappa, p.csw, p.mubar, p.mubar, p.epsbar)   # setup on D(mubar)
    ctx.load_gauge(U, -1)
    # D_ND at sampled sites against the oracle
    x2 = fields.gaussian_spinor(dims, 190, flavours=2)
    sites = sampled.random_sites(dims, 16, 191)
    want = sampled.apply_DND_at(U, x2, p, dims, sites)
    for prec, tol in ((F64, 1e-13), (F32, 1e-6), (F16, 5e-3)):
        y = ctx.apply(x2, op=tmg.OP_DND, prec=prec)
        got = np.array([y[:, t, z, yy, x] for x, yy, z, t in sites])
        assert rel(got, want) < tol, prec
    del x2, y
    # setup from 24 Gaussian vectors streamed to the device one at a time
    shape = fields.lattice_shape(dims) + (4, 3)
    v0 = torch.empty((w["nv"],) + shape, dtype=torch.complex128, device="cuda")
    for j, v in enumerate(fields.gaussian_spinor_columns(dims, w["seed"] + 100, w["nv"])):
        v0[j].copy_(torch.from_numpy(v))
    prm = tmg.Context.mg_defaults()
    prm.nv, prm.restart = w["nv"], w["restart"]
    prm.prec_fine, prm.prec_coarse = F32, F32
    ctx.setup(v0, prm)
    del v0
    torch.cuda.empty_cache()
    q = tmg.Context.level2_defaults()
    q.agg[:] = w["agg2"]
    q.nv = w["nv2"]
    c1 = ctx.coarse_lat
    ctx.setup_level2(fields.gaussian_coarse((c1[3], c1[2], c1[1], c1[0]), 2 * w["nv"], w["seed"] + 200, n=w["nv2"]), q)
    free, total = torch.cuda.mem_get_info()
    used_setup = total - free
    for seed in w["rhs_seeds"]:
        b = torch.from_numpy(fields.gaussian_spinor(dims, seed, flavours=2)).cuda()
        x, st = ctx.solve(b, tol=1e-10, method=tmg.SOLVE_ND_MIXED)
        r = ctx.apply(x, op=tmg.OP_DND, prec=F64) - b
        assert float(torch.linalg.vector_norm(r)) <= 1.01e-10 * float(torch.linalg.vector_norm(b)), seed
        print(f"ND 48^3x96 rhs seed {seed}: iterations {st['iterations']} refinements {st['refinements']} "
              f"coarse {st['coarse_iterations']} seconds {st['seconds']:.3f}")
        del b, x, r
    free, total = torch.cuda.mem_get_info()
    print(f"ND 48^3x96 device memory in use: after setup {used_setup / 2**30:.1f} GiB, "
          f"after solves {(total - free) / 2**30:.1f} GiB of {total / 2**30:.1f} GiB")
    assert total - free < total
