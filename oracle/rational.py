"""FP64 oracle of the RHMC rational approximation and of the multi-shift CG (test infrastructure only).

Sec. 3 (Eqs. 4-5) of arXiv:1710.06198 writes det D_ND through |Q_ND| = sqrt(Q_ND^2) and replaces
1/sqrt(Q_ND^2) by Zolotarev's optimal rational function of order n on the interval
[lambda_min, lambda_max] that holds the spectrum of Q_ND^2,

    1/sqrt(x) ~ R(x) = a prod_{l=1..n} (x + p_l) / (x + q_l),

optimal in the sense that the relative error 1 - sqrt(x) R(x) has the smallest maximum over the
interval (it equioscillates at 2n + 2 points, de la Vallee-Poussin / Chebyshev).  Zolotarev's
solution, written for y = x / lambda_min in [1, b], b = lambda_max / lambda_min, with the Jacobi
elliptic function sn of parameter m = 1 - 1/b and the complete elliptic integral K(m):

    c_l = sn^2(l K / (2n+1)) / (1 - sn^2(l K / (2n+1))),  l = 1 .. 2n,
    1/sqrt(y) ~ D prod_{l=1..n} (y + c_{2l}) / (y + c_{2l-1}),

with D the constant that centres the relative error.  The sums over shifted inverses come from the
partial fractions R(x) = a (1 + sum_l r_l / (x + q_l)), solved at once by the multi-shift CG, the
comparator of Sec. 3 (MMS-CG).

Pinned by tests/test_oracle_rational.py: for n = 10 on [6.5e-5, 4.7] the deviation equals the
paper's printed bound 1.4e-6 to its two digits; the error equioscillates at 2n + 2 points; partial
fractions equal the product; the multi-shift CG equals one CG per shift; R(Q^2) phi against
(Q^2)^-1/2 phi from a dense eigendecomposition, within the deviation.
"""
from __future__ import annotations

import numpy as np
from scipy.special import ellipj, ellipk


def zolotarev(n, lmin, lmax, grid=200001):
    """(a, p[n], q[n], delta): 1/sqrt(x) ~ a prod (x + p_l)/(x + q_l) on [lmin, lmax] and its
    maximal relative deviation delta (measured on a logarithmic grid of the interval)."""
    b = lmax / lmin
    m = 1.0 - 1.0 / b
    K = ellipk(m)
    l = np.arange(1, 2 * n + 1)
    sn, _, _, _ = ellipj(l * K / (2 * n + 1), m)
    c = sn ** 2 / (1.0 - sn ** 2)
    num, den = c[1::2], c[0::2]                  # c_{2l} over c_{2l-1}
    y = np.logspace(0.0, np.log10(b), grid)
    g = np.sqrt(y) * np.prod((y[None, :] + num[:, None]) / (y[None, :] + den[:, None]), axis=0)
    D = 2.0 / (g.max() + g.min())
    delta = (g.max() - g.min()) / (g.max() + g.min())
    return D / np.sqrt(lmin), lmin * num, lmin * den, float(delta)


def rational_eval(x, a, p, q):
    x = np.asarray(x, dtype=np.float64)
    return a * np.prod((x[..., None] + p) / (x[..., None] + q), axis=-1)


def partial_fractions(a, p, q):
    """R(x) = a (1 + sum_l r_l / (x + q_l)) for distinct q_l: returns r."""
    n = len(q)
    r = np.empty(n)
    for l in range(n):
        others = np.delete(q, l)
        r[l] = np.prod(p - q[l]) / np.prod(others - q[l])
    return r


def relative_error_curve(a, p, q, lmin, lmax, grid=200001):
    x = np.logspace(np.log10(lmin), np.log10(lmax), grid)
    return x, 1.0 - np.sqrt(x) * rational_eval(x, a, p, q)


def mms_cg(apply_A, b, sigma, tol=1e-12, maxiter=100000):
    """Multi-shift CG: x_s = (A + sigma_s)^-1 b for every shift at once, A Hermitian positive
    definite, sigma_s >= 0.  The Krylov space is that of the seed system A x = b (plain CG); the
    residual of system s stays collinear with the seed's, r_s = zeta_s r, and its coefficients
    follow from the seed's alpha_k, beta_k by the recurrences of the shifted-CG literature
    (Jegerlehner).  Stops when every shifted residual is <= tol ||b||.  Returns (x[list], iterations)."""
    sig = np.asarray(sigma, dtype=np.float64)
    ns = len(sig)
    bn = float(np.sqrt(np.real(np.vdot(b.ravel(), b.ravel()))))
    xs = [np.zeros_like(b) for _ in range(ns)]
    if bn == 0.0:
        return xs, 0
    r = b.copy()
    p = b.copy()                                  # seed direction
    ps = [b.copy() for _ in range(ns)]            # shifted directions
    z_cur = np.ones(ns)                           # zeta_s^k
    z_old = np.ones(ns)                           # zeta_s^{k-1}
    alpha_old, beta_old = 1.0, 0.0
    rr = bn * bn
    active = np.ones(ns, dtype=bool)
    it = 0
    while it < maxiter and active.any():
        Ap = apply_A(p)
        alpha = rr / float(np.real(np.vdot(p.ravel(), Ap.ravel())))
        r = r - alpha * Ap
        rr_new = float(np.real(np.vdot(r.ravel(), r.ravel())))
        beta = rr_new / rr
        for s in np.where(active)[0]:
            z_new = z_cur[s] * z_old[s] * alpha_old / (
                alpha * beta_old * (z_old[s] - z_cur[s]) + z_old[s] * alpha_old * (1.0 + sig[s] * alpha))
            a_s = alpha * z_new / z_cur[s]
            b_s = beta * (z_new / z_cur[s]) ** 2
            xs[s] = xs[s] + a_s * ps[s]
            ps[s] = z_new * r + b_s * ps[s]
            z_old[s], z_cur[s] = z_cur[s], z_new
            if abs(z_new) * np.sqrt(rr_new) <= tol * bn:
                active[s] = False
        p = r + beta * p
        alpha_old, beta_old, rr = alpha, beta, rr_new
        it += 1
    return xs, it


def rational_apply(apply_A, b, a, p, q, tol=1e-12):
    """R(A) b = a (b + sum_l r_l (A + q_l)^-1 b) through the multi-shift CG."""
    r = partial_fractions(a, p, q)
    xs, it = mms_cg(apply_A, b, q, tol)
    out = b.copy()
    for l in range(len(q)):
        out = out + r[l] * xs[l]
    return a * out, it
