"""GPU force (k_force.cu through the C ABI) against the oracle and against finite differences.

* tmg_force_xy on random X, Y (the formula is bilinear in X, Y) equals the oracle's
  traceless Hermitian part of -2 G to 1e-12 (FP64), with and without the clover term;
* tmg_force (both solves by the multigrid) equals the oracle's force with its own CG solves;
* central finite differences of S = ||D^-1 phi||^2 (step 1e-5, 32 random su(3) directions, FP64
  CG solves to 1e-14 on the rotated fields) agree with sum tr(H F) to 1e-6 relative;
* the device link update exp(i omega . lambda / 2) U equals the oracle's rotation (through D);
* tmg_pf_action / tmg_pf_force (one solve each) give the oracle's action and su(3) force
  coefficients, and the autograd Function runs the force kernels only in backward.
"""
import numpy as np
import pytest

from oracle import dirac, force, krylov
from synth import fields
from tests.conftest import rel

tmg = pytest.importorskip("paper_1710_06198_gb300")
pytestmark = pytest.mark.gpu

DIMS, BLOCK = (8, 4, 4, 4), (4, 2, 2, 2)


def _ctx(U, p):
    ctx = tmg.Context(DIMS, BLOCK)
    ctx.set_params(p.kappa, p.csw, p.mu)
    ctx.load_gauge(U, p.tbc)
    return ctx


@pytest.mark.parametrize("csw,tbc", [(1.3, -1), (0.0, 1)])
@pytest.mark.parametrize("prec,tol", [(tmg.PREC_F64, 1e-12), (tmg.PREC_F32, 1e-6)])
def test_force_xy_matches_oracle(csw, tbc, prec, tol):
    """FP64 force kernels to 1e-12; the default ones (FP32 copies of X, Y and of the 12-real links,
    every product summed in FP64) to 1e-6: only the inputs carry FP32 rounding (2^-24 relative per
    component), and F is multilinear in them."""
    U = fields.gauge_field(DIMS, 0.5, 81)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.2), csw=csw, mu=0.05, tbc=tbc)
    X = fields.gaussian_spinor(DIMS, 82)
    Y = fields.gaussian_spinor(DIMS, 83)
    want = force._traceless_hermitian(-2.0 * force.link_derivative(U, X, Y, p))
    ctx = _ctx(U, p)
    ctx.tune("force_prec", prec)
    got = ctx.force_xy(X, Y)
    assert rel(got, want) < tol


def _setup(ctx, nv=4):
    prm = tmg.Context.mg_defaults()
    prm.nv, prm.n_init, prm.n_iter = nv, 3, 1
    ctx.setup(fields.gaussian_spinor(DIMS, 84, n=nv), prm)


def test_force_with_multigrid_solves_matches_oracle():
    U = fields.gauge_field(DIMS, 0.4, 85)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.25), csw=1.0, mu=0.05, tbc=-1)
    phi = fields.gaussian_spinor(DIMS, 86)
    ctx = _ctx(U, p)
    _setup(ctx)
    S, F, st = ctx.force(phi, tol=1e-12)           # the default FP64 force kernels
    ctx.tune("force_prec", tmg.PREC_F32)           # FP32 inputs, FP64 sums
    S32, F32, _ = ctx.force(phi, tol=1e-12)
    ctx.tune("force_prec", tmg.PREC_F64)
    C = dirac.clover_term(U, p.csw)
    D = lambda v: dirac.apply_D(U, v, p, clover=C)
    Dd = lambda v: dirac.apply_Ddag(U, v, p, clover=C)

    def solve(b, dag):
        if dag:
            x, _, _ = krylov.cg_normal(Dd, D, b, tol=1e-13)
        else:
            x, _, _ = krylov.cg_normal(D, Dd, b, tol=1e-13)
        return x

    want = force.force(U, phi, p, solve)
    assert rel(F, want) < 1e-8
    assert rel(F32, want) < 1e-6
    assert abs(S - force.action(U, phi, p, solve)) < 1e-9 * S


def test_force_finite_differences_gpu_action():
    U = fields.gauge_field(DIMS, 0.4, 87)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.2), csw=1.2, mu=0.1, tbc=-1)
    phi = fields.gaussian_spinor(DIMS, 88)
    ctx = _ctx(U, p)
    _setup(ctx)
    _, F, _ = ctx.force(phi, tol=1e-13)

    def action(Ur):
        c2 = _ctx(Ur, p)
        y, st = c2.solve(phi, tol=1e-14, method=tmg.SOLVE_CG_F64, maxiter=100000)
        c2.close()
        return float(np.vdot(y.ravel(), y.ravel()).real)

    h = 1e-5
    for om in fields.su3_algebra_directions(DIMS, 89, 32):
        H = force.algebra_to_matrix(om)
        rot = lambda t: np.einsum("...ab,...bc->...ac", fields.exp_i_hermitian(H, t), U)
        fd = (action(rot(h)) - action(rot(-h))) / (2 * h)
        an = float(np.real(np.einsum("...ab,...ba->...", H, F).sum()))
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def test_rotate_gauge_matches_oracle_rotation():
    """D on the device-rotated field equals the oracle's D on U(omega) = exp(i omega . lambda / 2) U
    (eigen-decomposition exponential there, Taylor series with scaling and squaring here), for a
    small and a large rotation (the latter needs squaring), from host and device omega."""
    torch = pytest.importorskip("torch")
    U = fields.gauge_field(DIMS, 0.4, 95)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.2), csw=1.1, mu=0.05, tbc=-1)
    x = fields.gaussian_spinor(DIMS, 96)
    for scale, dev in ((1e-3, False), (1.7, True)):
        om = scale * fields.su3_algebra_directions(DIMS, 97, 1)[0]
        Ur = np.einsum("...ab,...bc->...ac", fields.exp_i_hermitian(force.algebra_to_matrix(om), 1.0), U)
        ctx = _ctx(U, p)
        ctx.rotate_gauge(torch.from_numpy(om).cuda() if dev else om)
        want = dirac.apply_D(Ur, x, p, clover=dirac.clover_term(Ur, p.csw))
        assert rel(ctx.apply(x, tmg.OP_D, tmg.PREC_F64), want) < 1e-13
        ctx.close()


def test_pf_action_and_force_match_oracle():
    """One solve for S and Y; the adjoint solve and the su(3) coefficients from Y alone."""
    U = fields.gauge_field(DIMS, 0.4, 85)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.25), csw=1.0, mu=0.05, tbc=-1)
    phi = fields.gaussian_spinor(DIMS, 86)
    ctx = _ctx(U, p)
    _setup(ctx)
    S, Y, st = ctx.pf_action(phi, tol=1e-12)
    f, st2 = ctx.pf_force(Y, tol=1e-12)
    C = dirac.clover_term(U, p.csw)
    D = lambda v: dirac.apply_D(U, v, p, clover=C)
    Dd = lambda v: dirac.apply_Ddag(U, v, p, clover=C)

    def solve(b, dag):
        x, _, _ = krylov.cg_normal(Dd, D, b, tol=1e-13) if dag else krylov.cg_normal(D, Dd, b, tol=1e-13)
        return x

    assert abs(S - force.action(U, phi, p, solve)) < 1e-9 * S
    assert rel(Y, solve(phi, False)) < 1e-9
    assert rel(f, force.matrix_to_algebra(force.force(U, phi, p, solve))) < 1e-6


def test_setup_update_after_rotation():
    """Rotate the field, update the setup by one iteration (Sec. 2), and solve to 1e-10 with the
    oracle's operator on the rotated field measuring the residual."""
    U = fields.gauge_field(DIMS, 0.4, 98)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.25), csw=1.0, mu=0.05, tbc=-1)
    ctx = _ctx(U, p)
    _setup(ctx)
    W0 = ctx.get_vectors()
    om = 0.05 * fields.su3_algebra_directions(DIMS, 99, 1)[0]
    ctx.rotate_gauge(om)
    Ur = np.einsum("...ab,...bc->...ac", fields.exp_i_hermitian(force.algebra_to_matrix(om), 1.0), U)
    b = fields.gaussian_spinor(DIMS, 100)
    ctx.setup_update(1)
    assert rel(ctx.get_vectors(), W0) > 1e-6
    x, st = ctx.solve(b, tol=1e-10, method=tmg.SOLVE_MG_MIXED)
    assert rel(dirac.apply_D(Ur, x, p, clover=dirac.clover_term(Ur, p.csw)), b) <= 1e-10


def test_autograd_function_gradient():
    """PseudofermionAction.backward at omega = 0 against central differences of its own forward."""
    torch = pytest.importorskip("torch")
    from paper_1710_06198_gb300.autograd import PseudofermionAction
    U = fields.gauge_field(DIMS, 0.4, 90)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.2), csw=1.0, mu=0.1, tbc=-1)
    phi = fields.gaussian_spinor(DIMS, 91)
    ctx = _ctx(U, p)
    prm = tmg.Context.mg_defaults()
    prm.nv, prm.n_init, prm.n_iter = 4, 3, 1
    setup = (fields.gaussian_spinor(DIMS, 92, n=4), prm)
    omega = torch.zeros(fields.lattice_shape(DIMS) + (4, 8), dtype=torch.float64, requires_grad=True)
    S = PseudofermionAction.apply(omega, phi, ctx, U, setup, 1e-13)
    n0 = tmg.launch_count(ctx)
    S.backward()
    assert tmg.launch_count(ctx) > n0          # backward launches the adjoint solve and force kernels
    g = omega.grad.numpy()
    d = fields.su3_algebra_directions(DIMS, 93, 1)[0]
    h = 1e-4
    with torch.no_grad():
        sp = PseudofermionAction.apply(torch.from_numpy(h * d), phi, ctx, U, setup, 1e-13).item()
        sm = PseudofermionAction.apply(torch.from_numpy(-h * d), phi, ctx, U, setup, 1e-13).item()
    fd = (sp - sm) / (2 * h)
    an = float(np.sum(g * d))
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
