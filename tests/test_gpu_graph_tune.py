"""The preconditioner cycle replayed as a CUDA graph gives the same solution as the kernel-by-kernel
launches (the captured kernels, launch shapes and reductions are the same), and the launch-shape
autotuner keeps a working configuration.  Sizes: 16 x 8 x 8 x 8 with 4 x 2 x 2 x 2 blocks (two
and three levels)."""
import numpy as np
import pytest

from oracle import dirac
from synth import fields
from tests.conftest import rel

tmg = pytest.importorskip("paper_1710_06198_gb300")
pytestmark = pytest.mark.gpu

DIMS, BLOCK = (16, 8, 8, 8), (4, 2, 2, 2)


def _ctx(levels):
    U = fields.gauge_field(DIMS, 0.45, 210)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.3), csw=1.1, mu=0.02, tbc=-1)
    ctx = tmg.Context(DIMS, BLOCK)
    ctx.set_params(p.kappa, p.csw, p.mu)
    ctx.load_gauge(U, -1)
    prm = tmg.Context.mg_defaults()
    prm.nv, prm.n_init, prm.n_iter = 4, 2, 1
    ctx.setup(fields.gaussian_spinor(DIMS, 211, n=4), prm)
    if levels == 3:
        q = tmg.Context.level2_defaults()
        q.nv, q.n_init, q.n_iter = 4, 2, 1
        c1 = ctx.coarse_lat
        ctx.setup_level2(fields.gaussian_coarse((c1[3], c1[2], c1[1], c1[0]), 8, 212, n=4), q)
    return ctx, U, p


@pytest.mark.parametrize("levels", [2, 3])
def test_graph_replay_matches_eager(levels):
    ctx, U, p = _ctx(levels)
    b = fields.gaussian_spinor(DIMS, 213)
    ctx.tune("cycle_graph", 0)
    x0, s0 = ctx.solve(b, tol=1e-10)
    ctx.tune("cycle_graph", 1)
    n0 = tmg.launch_count(ctx)
    x1, s1 = ctx.solve(b, tol=1e-10)    # captures
    x2, s2 = ctx.solve(b, tol=1e-10)    # replays
    n2 = tmg.launch_count(ctx)
    assert s0["iterations"] == s1["iterations"] == s2["iterations"]
    assert np.array_equal(x0, x1) and np.array_equal(x0, x2)
    assert n2 > n0
    assert tmg.graph_count(ctx) > 0
    assert rel(dirac.apply_D(U, x2, p), b) <= 1.01e-10


@pytest.mark.parametrize("levels", [2, 3])
def test_autotune_keeps_a_working_shape(levels):
    ctx, U, p = _ctx(levels)
    b = fields.gaussian_spinor(DIMS, 214)
    ms = ctx.autotune()
    assert 0.0 < ms < 1e4
    x, st = ctx.solve(b, tol=1e-10)
    assert rel(dirac.apply_D(U, x, p), b) <= 1.01e-10


@pytest.mark.parametrize("levels", [2, 3])
def test_batched_graph_follows_tensor_core_knob(levels):
    """The batched cycle's graph is keyed on the tensor-core kernel form: switching tc_pipeline after
    a capture leads to a new capture, and both forms give the same converged columns (N_v = 4, so the
    lock-step K-cycle and the batched coarse GMRES run on the tensor cores)."""
    ctx, U, p = _ctx(levels)
    b = np.stack([fields.gaussian_spinor(DIMS, 215 + j) for j in range(3)])
    mus = [p.mu, -p.mu, 0.5 * p.mu]
    xs = []
    for pipe in (1, 0):
        ctx.tune("tc_pipeline", pipe)
        ctx.solve(b, tol=1e-10, method=tmg.SOLVE_MG_BATCHED, mu_per_col=mus)     # eager run, then capture
        g0 = tmg.graph_count(ctx)
        x, st = ctx.solve(b, tol=1e-10, method=tmg.SOLVE_MG_BATCHED, mu_per_col=mus)
        assert tmg.graph_count(ctx) >= g0
        xs.append((x, g0))
    assert xs[1][1] > xs[0][1]     # the second form was captured, not replayed from the first
    for j, mu in enumerate(mus):
        pj = dirac.Params(kappa=p.kappa, csw=p.csw, mu=mu, tbc=-1)
        for x, _ in xs:
            assert rel(dirac.apply_D(U, x[j], pj), b[j]) <= 1.5e-10
        assert rel(xs[0][0][j], xs[1][0][j]) < 1e-8
