"""Pins of the oracle's multigrid pieces (Eq. 1 and Sec. 1.1 of arXiv:1710.06198).

* P^dag P = I and G5 P = P G5_c (Gamma5-compatible aggregation);
* the stored 9-point D_c equals the definition P^dag D P;
* D_c(mu) - D_c(0) = i mu G5_c and D_c^dag = G5_c D_c G5_c;
* the coarse-grid correction depends only on span(P) (basis invariance);
* full-rank P makes the coarse-grid correction exact;
* SAP with converged block solves equals the dense product of block projections;
* Krylov solvers and the two-level solve agree with dense LU.
"""
import numpy as np
import pytest

from oracle import dirac, krylov, mg
from synth import fields
from tests.conftest import rel


def _params(m0=-0.2, csw=1.2, mu=0.05, tbc=-1):
    return dirac.Params(kappa=dirac.kappa_from_m0(m0), csw=csw, mu=mu, tbc=tbc)


def _prolongator(dims, adims, nv, seed, eps=0.5):
    U = fields.gauge_field(dims, eps, seed)
    v = fields.gaussian_spinor(dims, seed + 1, n=nv)
    return U, mg.Prolongator(mg.orthonormalise(v, adims), tuple(adims))


def test_prolongator_orthonormal_and_gamma5_compatible():
    dims, adims, nv = (4, 4, 2, 4), (2, 2, 2, 2), 4
    _, P = _prolongator(dims, adims, nv, 30)
    clat = P.coarse_lat
    c = fields.gaussian_coarse((2, 2, 1, 2), 2 * nv, 31)
    assert c.shape[:4] == clat
    assert rel(mg.restrict(P, mg.prolong(P, c)), c) < 1e-14           # P^dag P = I
    g5c = mg.coarse_gamma5(nv)
    assert rel(dirac.apply_g5(mg.prolong(P, c)), mg.prolong(P, g5c * c)) < 1e-15
    # dense: P^dag P = identity exactly as a matrix
    n = int(np.prod(clat)) * 2 * nv
    Pm = np.stack([mg.prolong(P, e.reshape(clat + (2 * nv,))).ravel() for e in np.eye(n)], axis=1)
    assert np.abs(Pm.conj().T @ Pm - np.eye(n)).max() < 1e-14


@pytest.mark.parametrize("dims,adims", [((6, 4, 4, 6), (2, 2, 2, 2)),   # coarse extent 3
                                        ((4, 4, 4, 4), (2, 2, 4, 4)),   # coarse extent 1
                                        ((8, 4, 4, 4), (4, 4, 4, 4))])  # coarse extent 2
def test_coarse_stencil_equals_definition(dims, adims):
    nv = 3
    U, P = _prolongator(dims, adims, nv, 40)
    p = _params()
    C = dirac.clover_term(U, p.csw)
    Dc = mg.build_coarse(U, p, C, P)
    clat = P.coarse_lat
    x = fields.gaussian_coarse((clat[3], clat[2], clat[1], clat[0]), 2 * nv, 41)
    for mu in (0.0, 0.3):
        want = mg.coarse_apply_definition(U, p, C, P, x, mu)
        got = mg.coarse_apply(Dc, x, mu)
        assert rel(got, want) < 1e-13
    # twist on the coarse grid: D_c(mu) - D_c(0) = i mu G5_c
    d = mg.coarse_apply_definition(U, p, C, P, x, 0.3) - mg.coarse_apply_definition(U, p, C, P, x, 0.0)
    assert rel(d, 0.3j * mg.coarse_gamma5(nv) * x) < 1e-13


def test_coarse_gamma5_hermiticity():
    dims, adims, nv = (6, 4, 4, 4), (2, 2, 2, 2), 2
    U, P = _prolongator(dims, adims, nv, 50)
    p = _params(mu=0.0)
    Dc = mg.build_coarse(U, p, dirac.clover_term(U, p.csw), P)
    A = mg.coarse_dense(Dc, 0.0)
    g = np.tile(mg.coarse_gamma5(nv), A.shape[0] // (2 * nv))
    assert np.abs(A.conj().T - (g[:, None] * A * g[None, :])).max() < 1e-13


def test_coarse_backward_blocks_from_forward_blocks():
    """Per stencil slot: the -mu block of site a equals G5_c (+mu block of a - mu)^dag G5_c, also on
    coarse extents 2 (where a + mu = a - mu but the two hops are separate slots) and 3, with the
    antiperiodic time boundary.  The tensor-core coarse apply reads only the self and forward
    blocks and builds the backward ones from this relation."""
    dims, adims, nv = (6, 4, 4, 4), (2, 2, 2, 2), 2          # coarse lattice 3 x 2 x 2 x 2
    U, P = _prolongator(dims, adims, nv, 51)
    p = _params(mu=0.0)
    Dc = mg.build_coarse(U, p, dirac.clover_term(U, p.csw), P)
    g = mg.coarse_gamma5(nv)
    for m in range(4):
        f = np.roll(Dc.fwd[m], 1, axis=-3 - m)               # the +mu block of site a - mu, at a
        want = g[:, None] * np.swapaxes(f.conj(), -1, -2) * g[None, :]
        assert np.abs(Dc.bwd[m] - want).max() < 1e-13 * np.abs(Dc.bwd[m]).max(), m
        # a dropped sign or conjugation does not pass
        assert np.abs(Dc.bwd[m] - np.swapaxes(f.conj(), -1, -2)).max() > 1e-6, m


def test_coarse_correction_basis_invariance():
    """I - P D_c^-1 P^dag D depends on span(P) only: mixing the test vectors by any invertible
    matrix leaves the coarse-grid correction unchanged."""
    dims, adims, nv = (4, 4, 2, 4), (2, 2, 2, 2), 3
    U = fields.gauge_field(dims, 0.5, 60)
    p = _params(mu=0.1)
    C = dirac.clover_term(U, p.csw)
    v = fields.gaussian_spinor(dims, 61, n=nv)
    rng = np.random.default_rng(62)
    R = rng.standard_normal((nv, nv)) + 1j * rng.standard_normal((nv, nv))
    v2 = np.einsum("jk,k...->j...", R, v)
    e = fields.gaussian_spinor(dims, 63)
    out = []
    for vv in (v, v2):
        P = mg.Prolongator(mg.orthonormalise(vv, adims), adims)
        Dc = mg.build_coarse(U, p, C, P)
        A = mg.coarse_dense(Dc, p.mu)
        c = mg.restrict(P, dirac.apply_D(U, e, p, clover=C))
        sol = np.linalg.solve(A, c.ravel()).reshape(c.shape)
        out.append(e - mg.prolong(P, sol))
    assert rel(out[1], out[0]) < 1e-11


def test_full_rank_prolongator_exact_correction():
    """Aggregates of one site and N_v = 6 per chirality: P is unitary, D_c is unitarily similar to
    D and FGMRES preconditioned by P D_c^-1 P^dag converges in one step."""
    dims = (2, 2, 2, 2)
    U = fields.gauge_field(dims, 0.6, 70)
    p = _params(mu=0.1)
    C = dirac.clover_term(U, p.csw)
    P = mg.Prolongator(mg.orthonormalise(fields.gaussian_spinor(dims, 71, n=6), (1, 1, 1, 1)),
                       (1, 1, 1, 1))
    Dc = mg.build_coarse(U, p, C, P)
    A = mg.coarse_dense(Dc, p.mu)
    b = fields.gaussian_spinor(dims, 72)
    prec = lambda r: mg.prolong(P, np.linalg.solve(A, mg.restrict(P, r).ravel()).reshape(
        P.coarse_lat + (12,)))
    x, steps, res = krylov.fgmres(lambda v: dirac.apply_D(U, v, p, clover=C), b, prec, m=5, tol=1e-12)
    assert steps == 1 and res < 1e-12
    D = dirac.dense_matrix(lambda v: dirac.apply_D(U, v, p, clover=C), fields.lattice_shape(dims) + (4, 3))
    ev_f = np.sort_complex(np.round(np.linalg.eigvals(D), 10))
    ev_c = np.sort_complex(np.round(np.linalg.eigvals(A), 10))
    assert np.abs(ev_f - ev_c).max() < 1e-9


def test_sap_converged_equals_block_projection_product():
    """With converged block solves, one SAP sweep from x = 0 maps b to
    x = K1 (b - D K0 b) + K0 b, K_c = sum over colour-c blocks of I_B D_B^-1 I_B^T."""
    dims, bdims = (4, 4, 4, 4), (2, 2, 2, 2)
    U = fields.gauge_field(dims, 0.3, 80)
    p = _params(m0=0.4, mu=0.05)
    C = dirac.clover_term(U, p.csw)
    shape = fields.lattice_shape(dims) + (4, 3)
    D = dirac.dense_matrix(lambda v: dirac.apply_D(U, v, p, clover=C), shape)
    col = mg.block_colour(fields.lattice_shape(dims), bdims)
    bid = mg.coords(fields.lattice_shape(dims))
    block_index = sum((bid[mu] // bdims[mu]) * (10 ** mu) for mu in range(4))
    site_block = np.repeat(block_index.ravel(), 12)
    site_col = np.repeat(col.ravel(), 12)
    K = []
    for c in (0, 1):
        Kc = np.zeros_like(D)
        for bval in np.unique(site_block[site_col == c]):
            idx = np.where(site_block == bval)[0]
            Kc[np.ix_(idx, idx)] = np.linalg.inv(D[np.ix_(idx, idx)])
        K.append(Kc)
    b = fields.gaussian_spinor(dims, 81)
    bv = b.ravel()
    x0 = K[0] @ bv
    want = x0 + K[1] @ (bv - D @ x0)
    got = mg.sap(U, p, C, b, bdims, n_sweeps=1, n_mr=120)
    assert rel(got.ravel(), want) < 1e-11


def test_block_operator_is_block_diagonal_part_of_D():
    dims, bdims = (4, 8, 4, 2), (2, 4, 2, 1)
    U = fields.gauge_field(dims, 0.5, 82)
    p = _params()
    C = dirac.clover_term(U, p.csw)
    shape = fields.lattice_shape(dims) + (4, 3)
    D = dirac.dense_matrix(lambda v: dirac.apply_D(U, v, p, clover=C), shape)
    DB = dirac.dense_matrix(lambda v: mg.apply_D_blocks(U, v, p, C, bdims), shape)
    bid = mg.coords(fields.lattice_shape(dims))
    blk = np.repeat(sum((bid[mu] // bdims[mu]) * (10 ** mu) for mu in range(4)).ravel(), 12)
    same = blk[:, None] == blk[None, :]
    assert np.abs(DB - np.where(same, D, 0)).max() < 1e-15


def test_krylov_against_dense_lu():
    dims = (2, 2, 2, 4)
    U = fields.gauge_field(dims, 0.6, 90)
    p = _params(mu=0.05)
    C = dirac.clover_term(U, p.csw)
    shape = fields.lattice_shape(dims) + (4, 3)
    D = dirac.dense_matrix(lambda v: dirac.apply_D(U, v, p, clover=C), shape)
    b = fields.gaussian_spinor(dims, 91)
    x_lu = np.linalg.solve(D, b.ravel())
    Dop = lambda v: dirac.apply_D(U, v, p, clover=C)
    x_cg, _, r_cg = krylov.cg_normal(Dop, lambda v: dirac.apply_Ddag(U, v, p, clover=C), b, tol=1e-13)
    x_gm, _, r_gm = krylov.gmres(Dop, b, m=20, tol=1e-13)
    for x in (x_cg, x_gm):
        assert rel(x.ravel(), x_lu) < 1e-10
    e = krylov.mr(Dop, b, 1)
    a = np.vdot(D @ b.ravel(), b.ravel()) / np.vdot(D @ b.ravel(), D @ b.ravel())
    assert rel(e.ravel(), a * b.ravel()) < 1e-14


def test_two_level_solve_against_dense_lu():
    dims = (4, 4, 4, 4)
    U = fields.gauge_field(dims, 0.4, 100)
    p = _params(m0=-0.3, mu=0.02)
    m = mg.MGParams(block=(2, 2, 2, 2), agg=(2, 2, 2, 2), nv=4, n_init=2, n_iter=1, restart=10)
    H = mg.Hierarchy(U, p, m)
    H.setup(fields.gaussian_spinor(dims, 101, n=m.nv))
    b = fields.gaussian_spinor(dims, 102)
    x, steps, res = H.solve(b, tol=1e-12)
    shape = fields.lattice_shape(dims) + (4, 3)
    D = dirac.dense_matrix(H.D, shape)
    x_lu = np.linalg.solve(D, b.ravel())
    assert res < 1e-12
    assert rel(x.ravel(), x_lu) < 1e-9
    # two-step solve of D^dag D (Sec. 1.1): D(-mu) x1 = G5 b, then D(mu) y = G5 x1
    x1, _, _ = H.solve(dirac.apply_g5(b), tol=1e-12, mu=-p.mu)
    y, _, _ = H.solve(dirac.apply_g5(x1), tol=1e-12)
    want = np.linalg.solve(D.conj().T @ D, b.ravel())
    assert rel(y.ravel(), want) < 1e-8


def test_cycle_error_propagator_is_eq1_product():
    """Eq. 1 fixes the order of the two factors: with exact block solves and an exact coarse
    solve, the error propagator of one cycle applied to the zero initial guess is
        I - C D = (I - M D)^k (I - P D_c^-1 P^dag D),
    with one SAP sweep's propagator (I - K1 D)(I - K0 D) (colour 0 first), K_c the sum of the
    colour-c block inverses.  The cycle is linear once its inner solves are exact, so the identity
    is checked on random errors e (r = D e).  Swapping the factors (smoothing first), starting the
    smoother from zero instead of from the coarse correction, or dropping a sweep all fail it."""
    dims, bdims, nv, k = (4, 4, 4, 4), (2, 2, 2, 2), 2, 2
    U = fields.gauge_field(dims, 0.3, 110)
    p = _params(m0=0.4, mu=0.05)
    # the GMRES coarse solve is exact when it may take as many steps as D_c has rows (16 x 4)
    prm = mg.MGParams(block=bdims, agg=bdims, nv=nv, sap_sweeps=k, sap_mr=120, coarse_m=64,
                      coarse_rtol=1e-15)
    H = mg.Hierarchy(U, p, prm)
    H.set_vectors(fields.gaussian_spinor(dims, 111, n=nv))
    shape = fields.lattice_shape(dims) + (4, 3)
    D = dirac.dense_matrix(H.D, shape)
    n = D.shape[0]
    # dense P from the oracle's prolongation of unit coarse vectors; dense D_c = P^dag D P
    clat = H.P.coarse_lat + (2 * nv,)
    nc = int(np.prod(clat))
    Pm = np.stack([mg.prolong(H.P, e.reshape(clat)).ravel() for e in np.eye(nc)], axis=1)
    Ac = Pm.conj().T @ D @ Pm
    cgc = np.eye(n) - Pm @ np.linalg.solve(Ac, Pm.conj().T @ D)
    col = np.repeat(mg.block_colour(fields.lattice_shape(dims), bdims).ravel(), 12)
    bid = mg.coords(fields.lattice_shape(dims))
    blk = np.repeat(sum((bid[mu] // bdims[mu]) * (10 ** mu) for mu in range(4)).ravel(), 12)
    sweep = np.eye(n)
    for c in (0, 1):
        Kc = np.zeros_like(D)
        for bval in np.unique(blk[col == c]):
            idx = np.where(blk == bval)[0]
            Kc[np.ix_(idx, idx)] = np.linalg.inv(D[np.ix_(idx, idx)])
        sweep = (np.eye(n) - Kc @ D) @ sweep
    smooth = np.linalg.matrix_power(sweep, k)
    want_prop = smooth @ cgc
    wrong = {"smoothing first": cgc @ smooth, "smoother from zero": smooth,
             "one sweep fewer": np.linalg.matrix_power(sweep, k - 1) @ cgc}
    for seed in (112, 113):
        e = fields.gaussian_spinor(dims, seed).ravel()
        r = (D @ e).reshape(shape)
        got = e - H.cycle(r).ravel()
        want = want_prop @ e
        assert rel(got, want) < 1e-10
        for name, Wp in wrong.items():
            assert rel(Wp @ e, want) > 1e-3, name


def _coarse_small(mu=0.07):
    """A coarse operator on a 2^4 coarse lattice (4^4 fine lattice, 2^4 aggregates, N_v = 2)."""
    dims, adims, nv = (4, 4, 4, 4), (2, 2, 2, 2), 2
    U = fields.gauge_field(dims, 0.4, 71)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.4), csw=1.2, mu=mu, tbc=-1)
    H = mg.Hierarchy(U, p, mg.MGParams(block=adims, agg=adims, nv=nv))
    H.set_vectors(fields.gaussian_spinor(dims, 72, n=nv))
    return H.Dc, mu


def _dense_coarse(Dc, mu):
    shp = Dc.self_blk.shape[:-1]
    N = int(np.prod(shp))
    A = np.zeros((N, N), dtype=complex)
    for i in range(N):
        e = np.zeros(N, dtype=complex)
        e[i] = 1.0
        A[:, i] = mg.coarse_apply(Dc, e.reshape(shp), mu).reshape(-1)
    return A, shp


def test_coarse_schur_complement_is_block_elimination():
    """D_c(mu) applied to (x_o, -A_ee^-1 A_eo x_o) gives S x_o on the odd sites and zero on the even
    ones, and the assembled S equals A_oo - A_oe A_ee^-1 A_eo of the dense operator."""
    Dc, mu = _coarse_small()
    par = mg.coarse_parity(Dc)[..., None]
    rng = np.random.default_rng(73)
    shp = Dc.self_blk.shape[:-1]
    xo = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) * (par == 1)
    inv = mg.coarse_site_inverse(Dc, mu)
    xe = -np.einsum("...kl,...l->...k", inv, mg.coarse_hops(Dc, xo)) * (par == 0)
    y = mg.coarse_apply(Dc, xo + xe, mu)
    assert np.abs(y * (par == 0)).max() < 1e-12 * np.abs(y).max()
    assert rel(y * (par == 1), mg.coarse_schur_apply(Dc, xo, mu)) < 1e-13
    A, _ = _dense_coarse(Dc, mu)
    odd = np.broadcast_to(par == 1, shp).reshape(-1)
    E, O = np.where(~odd)[0], np.where(odd)[0]
    S_dense = A[np.ix_(O, O)] - A[np.ix_(O, E)] @ np.linalg.solve(A[np.ix_(E, E)], A[np.ix_(E, O)])
    S_op = np.zeros((len(O), len(O)), dtype=complex)
    for c, i in enumerate(O):
        e = np.zeros(int(np.prod(shp)), dtype=complex)
        e[i] = 1.0
        S_op[:, c] = mg.coarse_schur_apply(Dc, e.reshape(shp), mu).reshape(-1)[O]
    assert rel(S_op, S_dense) < 1e-12


def test_coarse_eo_solve_full_dimension_equals_dense_solve():
    """A reduced-system GMRES cycle as long as the odd dimension is exact: the odd-even coarse solve
    then equals the dense solution of D_c(mu) x = b (and a short cycle is not)."""
    Dc, mu = _coarse_small()
    A, shp = _dense_coarse(Dc, mu)
    rng = np.random.default_rng(74)
    b = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    want = np.linalg.solve(A, b.reshape(-1)).reshape(shp)
    n_odd = A.shape[0] // 2
    assert rel(mg.coarse_solve_eo(Dc, b, mu, n_odd, 0.0), want) < 1e-9
    assert rel(mg.coarse_solve_eo(Dc, b, mu, 3, 0.0), want) > 1e-4


def test_coarse_parity_needs_even_extents():
    Dc, _ = _coarse_small()
    odd = mg.CoarseOp(Dc.self_blk[:1], Dc.fwd[:, :1], Dc.bwd[:, :1], Dc.nv)
    with pytest.raises(ValueError):
        mg.coarse_parity(odd)
