"""Pins of the oracle's doublet multigrid (oracle/nd.py): the Dirichlet block operator of D_ND, SAP
with exact block solves against the dense Schwarz error propagator, the coarse doublet operators
against their definitions P_ND^dag D_ND P_ND and P2_ND^dag D_ND,c P2_ND, and the two- and
three-level solves against dense LU and CG on the normal equations."""
import numpy as np
import pytest

from oracle import dirac, krylov, mg, nd
from synth import fields
from tests.conftest import rel


def _setup(dims, block, nv, seed, m0=-0.2, mubar=0.12, epsbar=0.13):
    U = fields.gauge_field(dims, 0.5, seed)
    p = dirac.Params(kappa=dirac.kappa_from_m0(m0), csw=1.2, mu=mubar, tbc=-1, mubar=mubar, epsbar=epsbar)
    H = mg.Hierarchy(U, p, mg.MGParams(block=block, agg=block, nv=nv, sap_sweeps=2, sap_mr=3, coarse_m=40,
                                       coarse_rtol=1e-3, restart=10))
    H.set_vectors(fields.gaussian_spinor(dims, seed + 1, n=nv))
    return U, p, H


def _block_mask(lat, bdims, which):
    c = mg.coords(lat)
    m = np.ones(lat, dtype=bool)
    for d in range(4):
        m &= (c[d] // bdims[d]) == which[d]
    return m[..., None, None]


def test_block_operator_is_restriction_of_DND():
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    U, p, H = _setup(dims, block, 2, 160)
    lat = fields.lattice_shape(dims)
    for which in [(0, 0, 0, 0), (1, 0, 1, 1)]:
        m = _block_mask(lat, block, which)
        x = fields.gaussian_spinor(dims, 161, n=2) * m
        full = dirac.apply_DND(U, x, p, H.clover) * m
        blk = nd.apply_DND_blocks(U, x, p, H.clover, block) * m
        assert rel(blk, full) < 1e-15


@pytest.fixture(scope="module")
def small():
    """4^4 lattice with 2^4 blocks and the dense D_ND (6144 x 6144)."""
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    U, p, H = _setup(dims, block, 4, 162)
    shape = (2,) + fields.lattice_shape(dims) + (4, 3)
    Dd = dirac.dense_matrix(lambda v: dirac.apply_DND(U, v, p, H.clover), shape)
    return dims, block, U, p, H, Dd


def test_sap_exact_block_solves_equal_dense_propagator(small):
    dims, block, U, p, H, Dd = small
    lat = fields.lattice_shape(dims)
    b = fields.gaussian_spinor(dims, 163, n=2)
    x0 = fields.gaussian_spinor(dims, 164, n=2)
    got = nd.sap_nd(U, p, H.clover, b, block, 1, 400, x0)
    # dense: for each colour, x += sum_{B of that colour} I_B D_ND,B^-1 I_B^T (b - D_ND x)
    shape = (2,) + lat + (4, 3)
    col = mg.block_colour(lat, block)
    x = x0.reshape(-1).copy()
    nb = [lat[3 - d] // block[d] for d in range(4)]
    for c in (0, 1):
        r = b.reshape(-1) - Dd @ x
        upd = np.zeros_like(x)
        for bt in range(nb[3]):
            for bz in range(nb[2]):
                for by in range(nb[1]):
                    for bx in range(nb[0]):
                        which = (bx, by, bz, bt)
                        m = np.broadcast_to(_block_mask(lat, block, which), shape).reshape(-1)
                        if not np.all(col[_block_mask(lat, block, which)[..., 0, 0]] == c):
                            continue
                        idx = np.nonzero(m)[0]
                        upd[idx] += np.linalg.solve(Dd[np.ix_(idx, idx)], r[idx])
        x = x + upd
    assert rel(got.reshape(-1), x) < 1e-11


def test_coarse_doublet_operators_equal_definitions():
    dims, block = (8, 4, 4, 4), (2, 2, 2, 2)
    U, p, H = _setup(dims, block, 3, 165)
    clat = H.Dc.self_blk.shape[:4]
    x = fields.gaussian_coarse((clat[3], clat[2], clat[1], clat[0]), 6, 166, n=2)
    want = nd.restrict_nd(H.P, dirac.apply_DND(U, nd.prolong_nd(H.P, x), p, H.clover))
    assert rel(mg.coarse_apply_nd(H.Dc, x, p.mubar, p.epsbar), want) < 1e-13
    p3 = mg.MGParams3(agg2=(2, 2, 2, 2), nv2=4)
    L1 = mg.Level1(H.Dc, p3)
    L1.set_vectors(fields.gaussian_coarse((clat[3], clat[2], clat[1], clat[0]), 6, 167, n=4))
    c2 = L1.P2.coarse_lat
    y = fields.gaussian_coarse((c2[3], c2[2], c2[1], c2[0]), 8, 168, n=2)
    want2 = nd.restrict_c_nd(L1.P2, mg.coarse_apply_nd(H.Dc, nd.prolong_c_nd(L1.P2, y), p.mubar, p.epsbar))
    assert rel(mg.coarse_apply_nd(L1.Dcc, y, p.mubar, p.epsbar), want2) < 1e-13


def test_two_level_doublet_solve_equals_dense_lu(small):
    dims, block, U, p, H, Dd = small
    HN = nd.HierarchyND(H)
    b = fields.gaussian_spinor(dims, 170, n=2)
    x, steps, res = HN.solve(b, tol=1e-12)
    shape = b.shape
    xe = np.linalg.solve(Dd, b.reshape(-1)).reshape(shape)
    assert res <= 1e-12
    assert rel(x, xe) < 1e-9


def test_three_level_doublet_solve_equals_cg():
    dims, block = (8, 4, 4, 4), (2, 2, 2, 2)
    U, p, H = _setup(dims, block, 3, 171)
    clat = H.Dc.self_blk.shape[:4]
    L1 = mg.Level1(H.Dc, mg.MGParams3(agg2=(2, 2, 2, 2), nv2=4, n_init=2, n_iter=1))
    L1.setup(fields.gaussian_coarse((clat[3], clat[2], clat[1], clat[0]), 6, 172, n=4), p.mubar)
    HN = nd.HierarchyND(H, L1)
    b = fields.gaussian_spinor(dims, 173, n=2)
    x, steps, res = HN.solve(b, tol=1e-12)
    g5t1 = lambda v: dirac.apply_g5(v[::-1])
    D = lambda v: dirac.apply_DND(U, v, p, H.clover)
    Dd = lambda v: g5t1(D(g5t1(v)))
    xo, _, _ = krylov.cg_normal(D, Dd, b, tol=1e-13)
    assert res <= 1e-12
    assert rel(x, xo) < 1e-9


def test_shifted_doublet_identities():
    """The shifted doublet of the rational approximation (Sec. 3): (G5 x tau1) D_ND(delta) =
    Q_ND + i delta, so solving D_ND(+delta) then D_ND(-delta) applies (Q_ND^2 + delta^2)^-1 (dense
    on 2^4); its coarse operator equals P_ND^dag D_ND(delta) P_ND."""
    import dataclasses
    dims = (2, 2, 2, 2)
    U = fields.gauge_field(dims, 0.5, 175)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.2), csw=1.2, tbc=-1, mubar=0.12, epsbar=0.13)
    C = dirac.clover_term(U, p.csw)
    delta = 0.07
    pp, pm = dataclasses.replace(p, ndshift=delta), dataclasses.replace(p, ndshift=-delta)
    g5t1 = lambda v: dirac.apply_g5(v[::-1])
    x = fields.gaussian_spinor(dims, 176, n=2)
    assert rel(g5t1(dirac.apply_DND(U, x, pp, C)), dirac.apply_QND(U, x, p, C) + 1j * delta * x) < 1e-15
    shape = (2,) + fields.lattice_shape(dims) + (4, 3)
    Q = dirac.dense_matrix(lambda v: dirac.apply_QND(U, v, p, C), shape)
    Dp = dirac.dense_matrix(lambda v: dirac.apply_DND(U, v, pp, C), shape)
    Dm = dirac.dense_matrix(lambda v: dirac.apply_DND(U, v, pm, C), shape)
    phi = x.reshape(-1)
    G = dirac.dense_matrix(g5t1, shape)
    u = np.linalg.solve(Dp, G @ phi)
    v = np.linalg.solve(Dm, G @ u)
    want = np.linalg.solve(Q @ Q + delta ** 2 * np.eye(len(phi)), phi)
    assert rel(v, want) < 1e-12


def test_shifted_coarse_doublet_and_solve(small):
    import dataclasses
    dims, block, U, p, H, Dd = small
    delta = 0.05
    ps = dataclasses.replace(p, ndshift=delta)
    clat = H.Dc.self_blk.shape[:4]
    xc = fields.gaussian_coarse((clat[3], clat[2], clat[1], clat[0]), 8, 177, n=2)
    want = nd.restrict_nd(H.P, dirac.apply_DND(U, nd.prolong_nd(H.P, xc), ps, H.clover))
    assert rel(mg.coarse_apply_nd(H.Dc, xc, p.mubar, p.epsbar, delta), want) < 1e-13
    H.p = ps
    try:
        HN = nd.HierarchyND(H)
        b = fields.gaussian_spinor(dims, 178, n=2)
        x, steps, res = HN.solve(b, tol=1e-12)
        shape = (2,) + fields.lattice_shape(dims) + (4, 3)
        Ds = dirac.dense_matrix(lambda v: dirac.apply_DND(U, v, ps, H.clover), shape)
        assert res <= 1e-12
        assert rel(x.reshape(-1), np.linalg.solve(Ds, b.reshape(-1))) < 1e-9
    finally:
        H.p = p
