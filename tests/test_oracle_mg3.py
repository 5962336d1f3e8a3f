"""Pins of the oracle's third level: P2^dag P2 = I and G5_c P2 = P2 G5_cc on level-1 vectors, the
level-2 stencil equals the definition P2^dag D_c P2, the level-2 twist identity, and the
three-level solve against an independent solve (CG on the normal equations)."""
import numpy as np
import pytest

from oracle import dirac, krylov, mg
from synth import fields
from tests.conftest import rel


def _level1(dims=(12, 4, 4, 4), block=(2, 2, 2, 2), nv=2, seed=120):
    U = fields.gauge_field(dims, 0.5, seed)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.2), csw=1.1, mu=0.05, tbc=-1)
    H = mg.Hierarchy(U, p, mg.MGParams(block=block, agg=block, nv=nv))
    H.set_vectors(fields.gaussian_spinor(dims, seed + 1, n=nv))
    return H


@pytest.mark.parametrize("agg2", [(2, 2, 2, 2), (2, 2, 1, 2), (6, 1, 2, 2)])
def test_level2_stencil_equals_definition(agg2):
    H = _level1()
    clat = H.Dc.self_blk.shape[:4]
    nv2 = 3
    v = fields.gaussian_coarse((clat[3], clat[2], clat[1], clat[0]), 2 * H.Dc.nv, 122, n=nv2)
    P2 = mg.Prolongator2(mg.orthonormalise_c(v, agg2, H.Dc.nv), agg2, H.Dc.nv)
    c2 = P2.coarse_lat
    x = fields.gaussian_coarse((c2[3], c2[2], c2[1], c2[0]), 2 * nv2, 123)
    # P2^dag P2 = I and G5 compatibility
    assert rel(mg.restrict_c(P2, mg.prolong_c(P2, x)), x) < 1e-14
    g1 = mg.coarse_gamma5(H.Dc.nv)
    assert rel(g1 * mg.prolong_c(P2, x), mg.prolong_c(P2, mg.coarse_gamma5(nv2) * x)) < 1e-15
    Dcc = mg.build_coarse_c(H.Dc, P2)
    for mu in (0.0, 0.07):
        want = mg.restrict_c(P2, mg.coarse_apply(H.Dc, mg.prolong_c(P2, x), mu))
        assert rel(mg.coarse_apply(Dcc, x, mu), want) < 1e-13


def test_three_level_solve():
    dims, block = (8, 4, 4, 4), (2, 2, 2, 2)
    U = fields.gauge_field(dims, 0.4, 124)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.3), csw=1.0, mu=0.02, tbc=-1)
    m = mg.MGParams(block=block, agg=block, nv=4, n_init=2, n_iter=1, restart=10)
    H = mg.Hierarchy3(U, p, m, mg.MGParams3(agg2=(2, 2, 2, 2), nv2=4, n_init=2, n_iter=1))
    clat = fields.lattice_shape(dims)
    c1 = tuple(clat[i] // block[3 - i] for i in range(4))
    H.setup3(fields.gaussian_spinor(dims, 125, n=4),
             fields.gaussian_coarse((c1[3], c1[2], c1[1], c1[0]), 8, 126, n=4))
    b = fields.gaussian_spinor(dims, 127)
    x, steps, res = H.solve(b, tol=1e-12)
    xo, _, _ = krylov.cg_normal(H.D, lambda v: dirac.apply_Ddag(U, v, p, clover=H.clover), b, tol=1e-13)
    assert res < 1e-12
    assert rel(x, xo) < 1e-9
