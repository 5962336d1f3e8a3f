"""Pins of the oracle's rational approximation and multi-shift CG (Sec. 3, Eqs. 4-5):

* n = 10 on [6.5e-5, 4.7]: the largest relative deviation of Zolotarev's R from 1/sqrt(x) is the
  paper's printed 1.4e-6 to the two digits it prints (1.428e-6 here; see the design notes);
* equioscillation: the relative error alternates in sign at 2n + 2 extrema of equal size (the
  characterisation of the optimal approximation the paper invokes);
* the deviation falls with n; partial fractions equal the product form;
* the multi-shift CG equals one dense solve per shift;
* R(Q_ND^2) phi on a 2^4 doublet lattice against (Q_ND^2)^-1/2 phi from a dense eigendecomposition,
  within the deviation for the lattice's own spectral interval.
"""
import json
import os

import numpy as np

from oracle import dirac, rational
from synth import fields
from tests.conftest import rel


def test_paper_interval_deviation():
    """The worked example of Sec. 3 (tests/golden/rational_approximation.json): the deviation for
    the printed order and interval rounds to the printed bound."""
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "rational_approximation.json")))
    n, lo, hi, bound = g["n"], g["lambda_min"], g["lambda_max"], g["deviation_bound_printed"]
    a, p, q, delta = rational.zolotarev(n, lo, hi)
    assert float(f"{delta:.{g['printed_digits'] - 1}e}") == bound
    d_less = rational.zolotarev(n - 1, lo, hi)[3]
    d_more = rational.zolotarev(n + 1, lo, hi)[3]
    assert d_more < delta < d_less


def test_equioscillation():
    n = 6
    a, p, q, delta = rational.zolotarev(n, 1e-3, 2.0)
    x, e = rational.relative_error_curve(a, p, q, 1e-3, 2.0, grid=400001)
    # extrema: the end points and the interior sign changes of the slope
    de = np.diff(e)
    ext = [0] + [k for k in range(1, len(de)) if de[k - 1] * de[k] < 0] + [len(e) - 1]
    vals = e[ext]
    assert len(ext) == 2 * n + 2
    assert np.all(np.sign(vals[1:]) == -np.sign(vals[:-1]))
    assert np.allclose(np.abs(vals), delta, rtol=1e-3)


def test_partial_fractions_equal_product():
    a, p, q, _ = rational.zolotarev(10, 6.5e-5, 4.7)
    r = rational.partial_fractions(a, p, q)
    x = np.logspace(-5, 1, 37)
    pf = a * (1.0 + np.sum(r[None, :] / (x[:, None] + q[None, :]), axis=1))
    assert np.max(np.abs(pf / rational.rational_eval(x, a, p, q) - 1.0)) < 1e-10


def test_mms_cg_equals_separate_solves():
    rng = np.random.default_rng(7)
    n = 60
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = M.conj().T @ M / n + 1e-3 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    sig = np.array([0.0, 1e-3, 0.05, 1.0, 7.0])
    xs, it = rational.mms_cg(lambda v: A @ v, b, sig, tol=1e-13)
    for s, x in zip(sig, xs):
        assert rel(x, np.linalg.solve(A + s * np.eye(n), b)) < 1e-9


def test_rational_q_nd_squared_against_dense():
    dims = (2, 2, 2, 2)
    U = fields.gauge_field(dims, 0.4, 160)
    p = dirac.Params(kappa=dirac.kappa_from_m0(-0.2), csw=1.0, mubar=0.12, epsbar=0.13, tbc=-1)
    C = dirac.clover_term(U, p.csw)
    shape = (2,) + fields.lattice_shape(dims) + (4, 3)
    Q = dirac.dense_matrix(lambda v: dirac.apply_QND(U, v, p, clover=C), shape)
    A = Q @ Q
    w, V = np.linalg.eigh(A)
    a, pp, qq, delta = rational.zolotarev(10, 0.99 * w[0], 1.01 * w[-1])
    phi = fields.gaussian_spinor(dims, 161, flavours=2).ravel()
    want = V @ ((V.conj().T @ phi) / np.sqrt(w))
    got, _ = rational.rational_apply(lambda v: A @ v, phi, a, pp, qq, tol=1e-14)
    assert rel(got, want) <= 1.05 * delta
