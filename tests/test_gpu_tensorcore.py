"""Tensor-core (tcgen05, split-TF32) multi-RHS coarse operator against the FP64 oracle's stencil,
column by column, with a twist per column; FP32-level tolerance."""
import numpy as np
import pytest

from oracle import dirac, mg
from synth import fields
from tests.conftest import rel

tmg = pytest.importorskip("paper_1710_06198_gb300")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nv,ncol", [(4, 3), (16, 12), (16, 20)])
def test_coarse_apply_tensor_cores(nv, ncol):
    dims, block = (8, 8, 4, 4), (4, 4, 2, 2)
    U = fields.gauge_field(dims, 0.5, 101)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.2), csw=1.2, mu=0.05, tbc=-1)
    ctx = tmg.Context(dims, block)
    ctx.set_params(p.kappa, p.csw, p.mu)
    ctx.load_gauge(U, -1)
    prm = tmg.Context.mg_defaults()
    prm.nv, prm.n_init, prm.n_iter = nv, 0, 0
    v0 = fields.gaussian_spinor(dims, 102, n=nv)
    ctx.setup(v0, prm)
    H = mg.Hierarchy(U, p, mg.MGParams(block=block, agg=block, nv=nv))
    H.set_vectors(v0)
    clat = ctx.coarse_lat
    x = fields.gaussian_coarse((clat[3], clat[2], clat[1], clat[0]), 2 * nv, 103, n=ncol)
    mus = np.linspace(-0.2, 0.3, ncol)
    y = ctx.coarse_apply_multi(x, mus)
    for j in range(ncol):
        assert rel(y[j], mg.coarse_apply(H.Dc, x[j], mus[j])) < 2e-6, j
