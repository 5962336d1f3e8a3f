"""Pins of the oracle's kappa-search pieces: the sparse D_W equals the matrix-free operator,
sigma_min on the free field equals its closed form, and the convergence-edge walk."""
import itertools

import numpy as np

from oracle import dirac, kappa
from synth import fields
from tests.conftest import rel


def test_sparse_matrix_equals_matrix_free_operator():
    dims = (4, 2, 2, 4)
    U = fields.gauge_field(dims, 0.6, 200)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.35), csw=1.3, tbc=-1)
    A = kappa.sparse_DW(U, p)
    for seed in (201, 202):
        v = fields.gaussian_spinor(dims, seed)
        assert rel((A @ v.reshape(-1)).reshape(v.shape), dirac.apply_DW(U, v, p)) < 1e-14


def test_free_field_sigma_min_closed_form():
    dims = (2, 4, 2, 6)
    U = fields.unit_gauge(dims)
    for m0 in (0.2, -0.3):
        p = dirac.Params(kappa=dirac.kappa_from_m0(m0), csw=1.0, tbc=-1)
        best = np.inf
        lx, ly, lz, lt = dims
        for nx, ny, nz, nt in itertools.product(range(lx), range(ly), range(lz), range(lt)):
            pm = (2 * np.pi * nx / lx, 2 * np.pi * ny / ly, 2 * np.pi * nz / lz, (2 * nt + 1) * np.pi / lt)
            M = m0 + sum(1 - np.cos(q) for q in pm)
            best = min(best, np.sqrt(M ** 2 + sum(np.sin(q) ** 2 for q in pm)))
        assert abs(kappa.sigma_min(U, p) - best) < 1e-10 * best


def test_convergence_edge_walk_and_bisection(monkeypatch):
    """search_m0_mg keeps the most critical converging m0: walk in steps of 0.1, then bisect."""
    edge = -1.23
    monkeypatch.setattr(kappa, "mg_steps", lambda U, m0, *a, **k: 20 if m0 > edge else 51)
    log = []
    m0 = kappa.search_m0_mg(None, 1.0, 0.01, (4, 4, 4, 4), 8, None, None, log=log)
    assert -1.25 <= m0 <= -1.2 + 1e-12
    assert [m for m, _ in log][:3] == [0.0, -0.1, -0.2]
    assert all(n == 20 for m, n in log if m > edge) and all(n == 51 for m, n in log if m <= edge)


def test_margin_rule_selects_most_critical_m0_within_twice_the_base_steps():
    log = [(0.0, 6), (-0.1, 7), (-0.2, 9), (-0.3, 12), (-0.4, 13), (-0.5, 30), (-0.45, 20)]
    assert kappa.select_m0(log) == -0.3
    assert kappa.select_m0(log, ratio=5.0) == -0.5
