"""FP64 oracle of the pseudofermion force (test infrastructure only).

Action (Sec. 1, 2 of arXiv:1710.06198; the HMC force terms use solves of D^dag D with the two-step
scheme of Sec. 1.1):  S(U) = phi^dag (D D^dag)^-1 phi = ||D(mu)^-1 phi||^2.

Convention: under U_mu(x) -> exp(i t H_mu(x)) U_mu(x), H traceless Hermitian, the force F is the
traceless Hermitian field with dS/dt|_0 = sum_{x, mu} tr(H_mu(x) F_mu(x)).  With Y = D^-1 phi and
X = D^-dag Y:   dS/dt = -2 Re(X^dag (dD/dt) Y).  dD/dt has two pieces, written out here from the
operator definition in ``oracle.dirac``:

* hopping term: the link U_mu(x) enters row x / column x+mu as -1/2 (1 - g_mu) U_mu(x) and row x+mu
  / column x as -1/2 (1 + g_mu) U_mu(x)^dag (times the time boundary sign);
* clover term: C(y) = (i c_sw / 32) sum_{rho != sigma} sigma_rho_sigma (x) (Q_rho_sigma(y) -
  Q_sigma_rho(y)); every leaf of every Q containing the link contributes through the product of the
  leaf's other three links with the spin-traced colour matrix of X and Y at the leaf's corner.

For a leaf L = L1 L2 L3 L4 whose factor k is the link (or its dagger), and the corner matrix
Lam with X^dag (s (x) M) Y = tr(M Lam), d tr(L Lam)/dt = i tr(H U L_{k+1}..L4 Lam L1..L_{k-1}) for
a plain factor and -i tr(H L_{k+1}..L4 Lam L1..L_{k-1} U^dag) for a daggered one.

Pinned by tests/test_oracle_force.py: central finite differences of S (dense LU solves) along
random su(3) directions, gauge covariance F' = g F g^dag, and c_sw = 0 / mu sign special cases.
"""
from __future__ import annotations

import numpy as np

from . import dirac


def _shift(field, offset):
    """field(y + offset) for an integer offset vector (x, y, z, t), periodic, no boundary sign."""
    out = field
    for mu in range(4):
        for _ in range(abs(offset[mu])):
            out = dirac.shift_fwd(out, mu) if offset[mu] > 0 else dirac.shift_bwd(out, mu)
    return out


def _unit(mu):
    e = [0, 0, 0, 0]
    e[mu] = 1
    return e


def _add(*vs):
    return [sum(v[i] for v in vs) for i in range(4)]


def _neg(v):
    return [-a for a in v]


def _leaves(rho, sig):
    """The four counter-clockwise (rho -> sig) leaves ending at y as lists of
    (offset of the link's base site, direction, daggered)."""
    r, s = _unit(rho), _unit(sig)
    z = [0, 0, 0, 0]
    return [
        [(z, rho, False), (r, sig, False), (s, rho, True), (z, sig, True)],
        [(z, sig, False), (_add(s, _neg(r)), rho, True), (_neg(r), sig, True), (_neg(r), rho, False)],
        [(_neg(r), rho, True), (_add(_neg(r), _neg(s)), sig, True), (_add(_neg(r), _neg(s)), rho, False),
         (_neg(s), sig, False)],
        [(_neg(s), sig, True), (_neg(s), rho, False), (_add(r, _neg(s)), sig, False), (z, rho, True)],
    ]


def _traceless_hermitian(m):
    h = 0.5 * (m + dirac.dagger(m))
    tr = np.trace(h, axis1=-2, axis2=-1) / 3.0
    return h - tr[..., None, None] * np.eye(3)


def link_derivative(U, X, Y, p: dirac.Params):
    """G with X^dag (dD/dt) Y = sum_{x, mu} tr(H_mu(x) G_mu(x)); G[T, Z, Y, X, mu, 3, 3]."""
    lat = U.shape[:4]
    G = np.zeros(lat + (4, 3, 3), dtype=np.complex128)
    t_idx = np.indices(lat)[0]
    T = lat[0]
    for mu in range(4):
        Umu = U[..., mu, :, :]
        sgn = np.ones(lat)
        if mu == 3 and p.tbc != 1:
            sgn[t_idx == T - 1] = p.tbc
        # forward piece at row x: -1/2 (1 - g) (i H U) Y(x+mu);  A1[c, a] = sum_s P[s, c] conj(X[s, a])
        P = dirac.spin_mul(dirac.I4 - dirac.GAMMA[mu], dirac.colour_mul(Umu, dirac.shift_fwd(Y, mu)))
        A1 = np.einsum("...sc,...sa->...ca", P, np.conj(X))
        # backward piece at row x+mu: -1/2 (1 + g) (-i U^dag H) Y(x);  A2[b, c] = sum_s W[s, b] conj((U X')[s, c])
        W = dirac.spin_mul(dirac.I4 + dirac.GAMMA[mu], Y)
        UX = dirac.colour_mul(Umu, dirac.shift_fwd(X, mu))
        A2 = np.einsum("...sb,...sc->...bc", W, np.conj(UX))
        G[..., mu, :, :] += (sgn[..., None, None] * 0.5j) * (A2 - A1)
    if p.csw != 0.0:
        coef = 1j * p.csw / 32.0
        for rho in range(4):
            for sig in range(4):
                if rho == sig:
                    continue
                sg = dirac.sigma(rho, sig)
                # Lam[b, a] = sum_{s,t} sigma[s, t] Y[t, b] conj(X[s, a])
                lam = np.einsum("st,...tb,...sa->...ba", sg, Y, np.conj(X))
                for orient, sign in (((rho, sig), 1.0), ((sig, rho), -1.0)):
                    for leaf in _leaves(*orient):
                        mats = []
                        for off, d, dag in leaf:
                            m = _shift(U[..., d, :, :], off)
                            mats.append(dirac.dagger(m) if dag else m)
                        for k, (off, d, dag) in enumerate(leaf):
                            after = np.broadcast_to(np.eye(3, dtype=np.complex128), lam.shape).copy()
                            for q in range(k + 1, 4):
                                after = after @ mats[q]
                            before = np.broadcast_to(np.eye(3, dtype=np.complex128), lam.shape).copy()
                            for q in range(0, k):
                                before = before @ mats[q]
                            if not dag:
                                M = 1j * (mats[k] @ after @ lam @ before)
                            else:
                                M = -1j * (after @ lam @ before @ mats[k])
                            # the link sits at x = y + off: G_d(x) += coef * sign * M(x - off)
                            G[..., d, :, :] += coef * sign * _shift(M, _neg(off))
    return G


def force(U, phi, p: dirac.Params, solve):
    """F_mu(x) (traceless Hermitian, [T, Z, Y, X, mu, 3, 3]) of S = ||D^-1 phi||^2.

    solve(b, dagger) must return D^-1 b (dagger False) or D^-dag b (dagger True)."""
    Y = solve(phi, False)
    X = solve(Y, True)
    G = link_derivative(U, X, Y, p)
    return _traceless_hermitian(-2.0 * G)


def action(U, phi, p: dirac.Params, solve):
    Y = solve(phi, False)
    return float(np.real(np.vdot(Y.ravel(), Y.ravel())))


def gell_mann():
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7][0, 0] = l[7][1, 1] = 1 / np.sqrt(3)
    l[7][2, 2] = -2 / np.sqrt(3)
    return l


def algebra_to_matrix(omega):
    """omega[..., 8] -> H = sum_a omega_a lambda_a / 2 (traceless Hermitian)."""
    return np.einsum("...a,aij->...ij", omega, gell_mann()) * 0.5


def matrix_to_algebra(F):
    """F traceless Hermitian -> f_a = tr(lambda_a / 2 F), so tr(H F) = sum_a omega_a f_a."""
    return np.real(np.einsum("aij,...ji->...a", gell_mann() * 0.5, F))
