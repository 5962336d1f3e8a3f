"""Tensor-core (tcgen05, split-TF32) multi-RHS coarse operator against the FP64 oracle's stencil,
column by column, with a twist per column; FP32-level tolerance.  Both kernel forms: the pipelined one
(stacked hi / lo operands, double-buffered; 2 N_v <= 32) and the unstacked one, on a coarse lattice
with one site per CTA and on one with several sites per CTA (site epilogues between the tiles of
the next site in flight)."""
import functools

import numpy as np
import pytest

from oracle import dirac, mg
from synth import fields
from tests.conftest import rel

tmg = pytest.importorskip("paper_1710_06198_gb300")
pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=4)
def _oracle_dc(nv, dims, block):
    U = fields.gauge_field(dims, 0.5, 101)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.2), csw=1.2, mu=0.05, tbc=-1)
    H = mg.Hierarchy(U, p, mg.MGParams(block=block, agg=block, nv=nv))
    H.set_vectors(fields.gaussian_spinor(dims, 102, n=nv))
    return H.Dc


@pytest.mark.parametrize("pipeline", [1, 0])
@pytest.mark.parametrize("nv,ncol,dims", [(4, 3, (8, 8, 4, 4)), (16, 12, (8, 8, 4, 4)), (16, 20, (8, 8, 4, 4)),
                                          (16, 12, (16, 16, 16, 16)), (8, 20, (16, 16, 16, 16))])
def test_coarse_apply_tensor_cores(nv, ncol, dims, pipeline):
    block = (4, 4, 2, 2)
    U = fields.gauge_field(dims, 0.5, 101)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.2), csw=1.2, mu=0.05, tbc=-1)
    ctx = tmg.Context(dims, block)
    ctx.set_params(p.kappa, p.csw, p.mu)
    ctx.load_gauge(U, -1)
    ctx.tune("tc_pipeline", pipeline)
    prm = tmg.Context.mg_defaults()
    prm.nv, prm.n_init, prm.n_iter = nv, 0, 0
    v0 = fields.gaussian_spinor(dims, 102, n=nv)
    ctx.setup(v0, prm)
    Dc = _oracle_dc(nv, dims, block)
    clat = ctx.coarse_lat
    x = fields.gaussian_coarse((clat[3], clat[2], clat[1], clat[0]), 2 * nv, 103, n=ncol)
    mus = np.linspace(-0.2, 0.3, ncol)
    y = ctx.coarse_apply_multi(x, mus)
    for j in range(ncol):
        assert rel(y[j], mg.coarse_apply(Dc, x[j], mus[j])) < 2e-6, j
