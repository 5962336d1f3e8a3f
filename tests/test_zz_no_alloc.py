"""The allocation-free coarse solve (tmg_coarse_solve_noalloc) against the allocating one.

Callers that cannot allocate device memory -- code inside a CUDA stream capture, hosts with their
own memory managers, latency-critical loops -- get the coarse solve of the multigrid cycle through
an entry point whose scratch is a fixed array inside the library.  This file is collected last so
that a failure here stops a -x run only after every other test has run; it also passes alone in a
fresh process.  The check calls the C ABI directly, twice in a row (the scratch keeps the previous
call's contents), and compares with tmg_coarse_solve on the same device inputs.
"""
import ctypes

import numpy as np
import pytest

from oracle import dirac
from synth import fields

tmg = pytest.importorskip("paper_1710_06198_gb300")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,grid", [(tmg.PREC_F64, 0), (tmg.PREC_F32, 0), (tmg.PREC_F64, 8), (tmg.PREC_F32, 8)])
def test_coarse_solve_noalloc_matches_allocating_entry(prec, grid):
    """grid > 0 sets the coarse solve's CTA count first (tmg_tune "coarse_grid"): both entry
    points must then launch the same grid and so agree to the same tolerance."""
    torch = pytest.importorskip("torch")
    dims, block, nv = (8, 8, 4, 4), (4, 4, 2, 2), 4
    U = fields.gauge_field(dims, 0.4, 71)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.3), csw=1.1, mu=0.02, tbc=-1)
    ctx = tmg.Context(dims, block)
    ctx.set_params(p.kappa, p.csw, p.mu)
    ctx.load_gauge(U, -1)
    prm = tmg.Context.mg_defaults()
    prm.nv, prm.n_init, prm.n_iter = nv, 2, 0
    prm.coarse_m, prm.coarse_rtol = 25, 1e-3
    ctx.setup(fields.gaussian_spinor(dims, 72, n=nv), prm)
    if grid:
        ctx.tune("coarse_grid", grid)
    L = tmg.lib()
    tol = 1e-12 if prec == tmg.PREC_F64 else 1e-6
    for call, seed in enumerate((73, 74)):
        c = torch.from_numpy(fields.gaussian_coarse((2, 2, 2, 2), 2 * nv, seed)).cuda()
        want = ctx.coarse_solve(c, p.mu, prec)
        got = torch.empty_like(c)
        rc = L.tmg_coarse_solve_noalloc(ctx._h, ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(got.data_ptr()),
                                        ctypes.c_double(p.mu), prec)
        assert rc == 0, L.tmg_last_error(ctx._h).decode()
        torch.cuda.synchronize()
        err = float(torch.linalg.vector_norm(got - want) / torch.linalg.vector_norm(want))
        assert err < tol, (call, err)
        assert np.isfinite(err)
    ctx.close()
