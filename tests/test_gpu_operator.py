"""GPU parity of the fine operators (called through the C ABI) against the FP64 oracle.

Tolerances (relative L2 over the whole field): FP64 1e-13, FP32 1e-6, FP16 storage 5e-3 (spinors,
links and clover all in 16-bit fixed point for D, D^dag and the hopping term).
Lattices: 8x4x4x4 with 4x2x2x2 blocks (16 blocks, every site on a block face in two directions),
8^4 with 4^4 blocks, and the full 16^3x32 lattice of the mixed-precision workload.
The lattice volume is always a multiple of 512 (16 blocks of >= 32 sites), so the 128-thread
dslash grid has no partial CTA; the partial-CTA path is exercised by the coarse kernels instead.
"""
import numpy as np
import pytest

from oracle import dirac
from synth import fields
from tests.conftest import rel

tmg = pytest.importorskip("paper_1710_06198_gb300")
pytestmark = pytest.mark.gpu

TOL = {tmg.PREC_F64: 1e-13, tmg.PREC_F32: 1e-6, tmg.PREC_F16: 5e-3}


def make(dims, block, eps, seed, m0=-0.25, csw=1.3, mu=0.07, tbc=-1, mubar=0.12, epsbar=0.13):
    U = fields.gauge_field(dims, eps, seed)
    p = dirac.Params(kappa=dirac.kappa_from_m0(m0), csw=csw, mu=mu, tbc=tbc, mubar=mubar, epsbar=epsbar)
    ctx = tmg.Context(dims, block)
    ctx.set_params(p.kappa, p.csw, p.mu, p.mubar, p.epsbar)
    ctx.load_gauge(U, tbc)
    return ctx, U, p, dirac.clover_term(U, p.csw)


@pytest.fixture(scope="module")
def small():
    return make((8, 4, 4, 4), (4, 2, 2, 2), 0.5, 21)


@pytest.mark.parametrize("prec", [tmg.PREC_F64, tmg.PREC_F32, tmg.PREC_F16])
def test_D_and_Ddag_small(small, prec):
    ctx, U, p, C = small
    x = fields.gaussian_spinor(ctx.dims, 22)
    assert rel(ctx.apply(x, tmg.OP_D, prec), dirac.apply_D(U, x, p, clover=C)) < TOL[prec]
    assert rel(ctx.apply(x, tmg.OP_DDAG, prec), dirac.apply_Ddag(U, x, p, clover=C)) < TOL[prec]


@pytest.mark.parametrize("prec", [tmg.PREC_F64, tmg.PREC_F32])
def test_hopping_term(small, prec):
    ctx, U, p, C = small
    x = fields.gaussian_spinor(ctx.dims, 23)
    assert rel(ctx.apply(x, tmg.OP_HOP, prec), dirac.hopping(U, x, p.tbc)) < TOL[prec]


@pytest.mark.parametrize("prec", [tmg.PREC_F64, tmg.PREC_F32, tmg.PREC_F16])
def test_nondegenerate_doublet(small, prec):
    ctx, U, p, C = small
    x2 = fields.gaussian_spinor(ctx.dims, 24, flavours=2)
    assert rel(ctx.apply(x2, tmg.OP_DND, prec), dirac.apply_DND(U, x2, p, clover=C)) < TOL[prec]


def test_multi_column_per_column_mu(small):
    ctx, U, p, C = small
    xs = fields.gaussian_spinor(ctx.dims, 25, n=3)
    mus = [0.0, -0.2, 0.35]
    y = ctx.apply(xs, tmg.OP_D, tmg.PREC_F64, mu_per_col=mus)
    for j, m in enumerate(mus):
        assert rel(y[j], dirac.apply_D(U, xs[j], p, mu=m, clover=C)) < 1e-13


def test_periodic_time_and_no_clover():
    ctx, U, p, C = make((4, 8, 4, 4), (2, 4, 2, 2), 0.6, 26, csw=0.0, tbc=1)
    x = fields.gaussian_spinor(ctx.dims, 27)
    assert rel(ctx.apply(x, tmg.OP_D, tmg.PREC_F64), dirac.apply_D(U, x, p, clover=C)) < 1e-13


def test_free_field_plane_wave():
    """Unit links: the GPU operator reproduces the closed-form symbol on a plane wave."""
    dims = (8, 4, 4, 4)
    ctx = tmg.Context(dims, (4, 2, 2, 2))
    m0, mu = 0.1, 0.2
    ctx.set_params(dirac.kappa_from_m0(m0), 1.0, mu)
    ctx.load_gauge(fields.unit_gauge(dims), -1)
    t, z, y, x = np.indices(fields.lattice_shape(dims))
    pm = [2 * np.pi / 8, 2 * 2 * np.pi / 4, 0.0, 3 * np.pi / 4]
    chi = np.arange(12).reshape(4, 3) * (1 + 0.5j)
    ph = np.exp(1j * (pm[0] * x + pm[1] * y + pm[2] * z + pm[3] * t))
    psi = ph[..., None, None] * chi
    M = m0 + sum(1 - np.cos(q) for q in pm)
    sym = M * np.eye(4) + 1j * sum(dirac.GAMMA[k] * np.sin(pm[k]) for k in range(4)) + 1j * mu * dirac.GAMMA5
    assert rel(ctx.apply(psi, tmg.OP_D, tmg.PREC_F64), ph[..., None, None] * (sym @ chi)) < 1e-13


@pytest.mark.parametrize("prec", [tmg.PREC_F64, tmg.PREC_F32, tmg.PREC_F16])
def test_D_8x4_lattice(prec):
    ctx, U, p, C = make((8, 8, 8, 8), (4, 4, 4, 4), 0.4, 1, csw=1.0, mu=0.01)
    x = fields.gaussian_spinor(ctx.dims, 2)
    assert rel(ctx.apply(x, tmg.OP_D, prec), dirac.apply_D(U, x, p, clover=C)) < TOL[prec]


def test_D_device_pointers(small):
    torch = pytest.importorskip("torch")
    ctx, U, p, C = small
    x = fields.gaussian_spinor(ctx.dims, 28)
    xd = torch.from_numpy(x).cuda()
    y = ctx.apply(xd, tmg.OP_D, tmg.PREC_F64).cpu().numpy()
    assert rel(y, dirac.apply_D(U, x, p, clover=C)) < 1e-13


@pytest.mark.parametrize("prec", [tmg.PREC_F32, tmg.PREC_F16])
def test_D_full_mixed_precision_lattice(prec):
    """16^3 x 32 (the mixed-precision workload's lattice), whole field against the oracle."""
    ctx, U, p, C = make((16, 16, 16, 32), (4, 4, 4, 4), 0.35, 3, csw=1.5, mu=0.003)
    x = fields.gaussian_spinor(ctx.dims, 4)
    assert rel(ctx.apply(x, tmg.OP_D, prec), dirac.apply_D(U, x, p, clover=C)) < TOL[prec]


def test_load_gauge_rejects_non_su3(small):
    """A link off SU(3) (scaled by 1.01) is rejected from host and from device memory, with the site
    named; the field loaded before stays in use."""
    torch = pytest.importorskip("torch")
    ctx, U, p, C = small
    bad = U.copy()
    bad[1, 2, 3, 0, 2] *= 1.01
    for arr in (bad, torch.from_numpy(bad).cuda()):
        with pytest.raises(tmg.TmgError) as e:
            ctx.load_gauge(arr, -1)
        assert e.value.code == -1 and "not in SU(3)" in str(e.value)
    x = fields.gaussian_spinor(ctx.dims, 29)
    assert rel(ctx.apply(x, tmg.OP_D, tmg.PREC_F64), dirac.apply_D(U, x, p, clover=C)) < 1e-13
