"""The single-site patch evaluation used by the full-size GPU tests equals the oracle's operator
applied to the whole lattice (including sites next to the antiperiodic time boundary)."""
import numpy as np

from oracle import dirac
from synth import fields
from tests import sampled
from tests.conftest import rel


def test_patch_values_equal_full_lattice():
    dims = (6, 5, 7, 6)
    U = fields.gauge_field(dims, 0.6, 150)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.4), csw=1.3, mu=0.07, tbc=-1, mubar=0.12, epsbar=0.13)
    psi = fields.gaussian_spinor(dims, 151)
    psi2 = fields.gaussian_spinor(dims, 152, n=2)
    sites = sampled.random_sites(dims, 6, 153) + [(0, 0, 0, 0), (5, 4, 6, 5), (2, 3, 1, 0), (1, 1, 1, 5)]
    full = dirac.apply_D(U, psi, p)
    assert rel(sampled.apply_D_at(U, psi, p, dims, sites), sampled.values_at(full, sites)) < 1e-14
    full_nd = dirac.apply_DND(U, psi2, p)
    got = sampled.apply_DND_at(U, psi2, p, dims, sites)
    assert rel(got, np.array([full_nd[:, t, z, y, x] for x, y, z, t in sites])) < 1e-14
