"""Pins of the FP64 oracle's fine operators against facts the paper and the mathematics fix.

* free field: plane waves are eigenvectors of the closed-form lattice symbol;
* uniform abelian field: closed-form clover term;
* gamma5-hermiticity (Sec. 1.1), twist identity / mu^2 bound (Sec. 1), gauge covariance;
* Hermiticity of Q = G5 D(0) (Eq. 3) and Q_ND = (G5 x tau1) D_ND (Eq. 4);
* dense brute force on a 2^4 lattice.
"""
import numpy as np
import pytest

from oracle import dirac
from synth import fields
from tests.conftest import rel


def _params(m0=-0.2, csw=1.3, mu=0.05, tbc=-1, **kw):
    return dirac.Params(kappa=dirac.kappa_from_m0(m0), csw=csw, mu=mu, tbc=tbc, **kw)


@pytest.mark.parametrize("tbc", [1, -1])
def test_free_field_plane_waves(tbc):
    dims = (4, 6, 2, 8)
    U = fields.unit_gauge(dims)
    p = _params(m0=0.17, csw=1.7, mu=0.3, tbc=tbc)
    rng = np.random.default_rng(11)
    lat = fields.lattice_shape(dims)
    t, z, y, x = np.indices(lat)
    for _ in range(6):
        n = [rng.integers(0, d) for d in dims]
        pm = [2 * np.pi * n[k] / dims[k] for k in range(3)]
        pm.append((2 * n[3] + (1 if tbc == -1 else 0)) * np.pi / dims[3])
        chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (pm[0] * x + pm[1] * y + pm[2] * z + pm[3] * t))
        psi = phase[..., None, None] * chi
        M = p.m0 + sum(1 - np.cos(q) for q in pm)
        sym = M * np.eye(4) + 1j * sum(dirac.GAMMA[k] * np.sin(pm[k]) for k in range(4)) \
            + 1j * p.mu * dirac.GAMMA5
        want = phase[..., None, None] * (sym @ chi)
        got = dirac.apply_D(U, psi, p)
        assert rel(got, want) < 1e-13
        # eigenvalues of the symbol: M +- i sqrt(sum sin^2 + mu^2), each twice (x3 colours)
        ev = np.linalg.eigvals(sym)
        ev = ev[np.argsort(ev.imag)]
        s = np.sqrt(sum(np.sin(q) ** 2 for q in pm) + p.mu ** 2)
        want_ev = np.array([M - 1j * s, M - 1j * s, M + 1j * s, M + 1j * s])
        assert np.allclose(ev, want_ev, atol=1e-12)


def test_free_field_clover_vanishes():
    U = fields.unit_gauge((4, 4, 4, 4))
    assert np.abs(dirac.clover_term(U, 1.9)).max() == 0.0


@pytest.mark.parametrize("plane", [(0, 1), (1, 3), (2, 3)])
def test_uniform_abelian_field_clover(plane):
    """Constant flux phi_c per plaquette in the (mu, nu) plane gives
    C = -(c_sw/2) sin(phi_c) sigma_mu_nu on every site (and nothing from the other planes)."""
    dims = (4, 6, 4, 6)
    csw = 1.4
    U, phi, q = fields.uniform_abelian_field(dims, plane, n_flux=1)
    C = dirac.clover_term(U, csw)
    mu, nu = plane
    want = -0.5 * csw * np.einsum("st,ab->satb", dirac.sigma(mu, nu), np.diag(np.sin(q * phi)))
    assert np.abs(C - want).max() < 1e-13


def test_clover_hermitian_and_chiral():
    U = fields.gauge_field((4, 4, 4, 4), 0.6, 3)
    C = dirac.clover_term(U, 1.7).reshape(fields.lattice_shape((4, 4, 4, 4)) + (12, 12))
    assert np.abs(C - np.conj(np.swapaxes(C, -1, -2))).max() < 1e-14
    g5 = np.kron(dirac.GAMMA5, np.eye(3))
    assert np.abs(C @ g5 - g5 @ C).max() < 1e-14
    assert np.abs(dirac.clover_term(U, 0.0)).max() == 0.0


def test_gamma5_hermiticity():
    dims = (4, 4, 2, 6)
    U = fields.gauge_field(dims, 0.5, 4)
    p = _params()
    x = fields.gaussian_spinor(dims, 5)
    y = fields.gaussian_spinor(dims, 6)
    lhs = dirac.vdot(y, dirac.apply_g5(dirac.apply_D(U, dirac.apply_g5(x), p, p.mu)))
    rhs = dirac.vdot(dirac.apply_D(U, y, p, -p.mu), x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-14


def test_twist_identity_and_bound():
    dims = (4, 4, 4, 4)
    U = fields.gauge_field(dims, 0.5, 7)
    p = _params(mu=0.37)
    x = fields.gaussian_spinor(dims, 8)
    a = dirac.norm2(dirac.apply_D(U, x, p))
    b = dirac.norm2(dirac.apply_DW(U, x, p)) + p.mu ** 2 * dirac.norm2(x)
    assert abs(a - b) / b < 1e-14
    assert a >= p.mu ** 2 * dirac.norm2(x)


def test_gauge_covariance():
    dims = (4, 2, 4, 6)
    U = fields.gauge_field(dims, 0.7, 9)
    g = fields.gauge_transform(dims, 10)
    p = _params()
    Ug = np.empty_like(U)
    for mu in range(4):
        gfwd = dirac.shift_fwd(g, mu)     # g(x + mu), no boundary sign for the transform
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ dirac.dagger(gfwd)
    psi = fields.gaussian_spinor(dims, 11)
    psig = dirac.colour_mul(g, psi)
    lhs = dirac.apply_D(U=Ug, psi=psig, p=p)
    rhs = dirac.colour_mul(g, dirac.apply_D(U, psi, p))
    assert rel(lhs, rhs) < 1e-13


def test_hermitian_forms():
    dims = (2, 4, 2, 4)
    U = fields.gauge_field(dims, 0.5, 12)
    p = _params(mu=0.0, mubar=0.12, epsbar=0.13)
    x = fields.gaussian_spinor(dims, 13)
    y = fields.gaussian_spinor(dims, 14)
    q = lambda v: dirac.apply_g5(dirac.apply_D(U, v, p, 0.0))
    assert abs(dirac.vdot(y, q(x)) - dirac.vdot(q(y), x)) / abs(dirac.vdot(y, q(x))) < 1e-14
    x2 = fields.gaussian_spinor(dims, 15, flavours=2)
    y2 = fields.gaussian_spinor(dims, 16, flavours=2)
    a = dirac.vdot(y2, dirac.apply_QND(U, x2, p))
    b = dirac.vdot(dirac.apply_QND(U, y2, p), x2)
    assert abs(a - b) / abs(a) < 1e-14


def test_nd_reduces_to_doublet():
    dims = (2, 2, 4, 4)
    U = fields.gauge_field(dims, 0.5, 17)
    p = _params(mu=0.21, mubar=0.21, epsbar=0.0)
    x2 = fields.gaussian_spinor(dims, 18, flavours=2)
    assert rel(dirac.apply_DND(U, x2, p), dirac.apply_doublet(U, x2, p)) < 1e-15


def test_nd_mass_block_eigenvalues():
    """Free field at p = 0: D_ND has the mass block m0 + i mubar g5 tau3 - epsbar tau1 whose
    eigenvalues are m0 +- sqrt(epsbar^2 - mubar^2) (real when epsbar > mubar)."""
    dims = (2, 2, 2, 2)
    U = fields.unit_gauge(dims)
    p = _params(m0=0.3, tbc=1, mubar=0.12, epsbar=0.13)
    shape = (2,) + fields.lattice_shape(dims) + (4, 3)
    D = dirac.dense_matrix(lambda v: dirac.apply_DND(U, v, p), shape)
    const = np.ones(shape[:-2] + (1, 1))  # zero-momentum subspace: constant in x
    ev = np.linalg.eigvals(D)
    s = np.sqrt(p.epsbar ** 2 - p.mubar ** 2)
    for target in (p.m0 + s, p.m0 - s):
        assert np.min(np.abs(ev - target)) < 1e-12
    assert const.sum() > 0


def test_dense_brute_force_2x4():
    dims = (2, 2, 2, 2)
    U = fields.gauge_field(dims, 0.8, 19)
    p = _params(m0=-0.1, mu=0.2)
    shape = fields.lattice_shape(dims) + (4, 3)
    D = dirac.dense_matrix(lambda v: dirac.apply_D(U, v, p), shape)
    Dm = dirac.dense_matrix(lambda v: dirac.apply_D(U, v, p, -p.mu), shape)
    G5 = np.kron(np.eye(16), np.kron(dirac.GAMMA5, np.eye(3)))
    assert np.abs(D.conj().T - G5 @ Dm @ G5).max() < 1e-14
    smin = np.linalg.svd(D, compute_uv=False).min()
    assert smin >= p.mu - 1e-12
    # D^dag D = D_W^dag D_W + mu^2 exactly (twist identity as matrices)
    DW = dirac.dense_matrix(lambda v: dirac.apply_DW(U, v, p), shape)
    assert np.abs(D.conj().T @ D - DW.conj().T @ DW - p.mu ** 2 * np.eye(D.shape[0])).max() < 1e-13
