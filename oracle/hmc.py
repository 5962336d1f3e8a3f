"""FP64 oracle of the Hasenbusch-split HMC trajectory (test infrastructure only).

Sec. 2 of arXiv:1710.06198 splits det[Q^2 + mu^2] (Q = G5 D_W Hermitian, Eq. 3) into ratios
det[(Q^2 + mu_i^2)/(Q^2 + mu_{i+1}^2)] and a last det[Q^2 + mu_N^2], places every factor on its own
time scale of a nested second-order minimal-norm integrator, and the gauge action innermost.  With
Q^2 + m^2 = D(m)^dag D(m) (the twist identity of Sec. 1.1) the monomials read:

* gauge:  S_g = beta sum_{x, mu<nu} (1 - Re tr P_mu_nu(x) / 3)      (Wilson plaquette action; the
          paper does not print its gauge action, this is the reading used here);
* det:    S = || D(mu)^-1 phi ||^2,                 heat bath phi = D(mu) eta;
* ratio:  S = || D(mu)^-dag D(mu')^dag phi ||^2,    heat bath phi = D(mu')^-dag D(mu)^dag eta,
          for det[D(mu)^dag D(mu)] / det[D(mu')^dag D(mu')], mu' = mu + rho.

Forces F (traceless Hermitian, dS/dt = sum tr(H F) under U -> exp(i t H) U, as in oracle.force):
* gauge: F = (beta / 3) TH[(W - W^dag) / (2 i)], W = U_mu(x) x (sum of the six staples);
* det:   F = TH(-2 G(X, Y)), Y = D^-1 phi, X = D^-dag Y                 (oracle.force);
* ratio: F = TH(-2 G(Y - phi, X)), Y = D(mu)^-dag D(mu')^dag phi, X = D(mu)^-1 Y, from
         dS/dt = 2 Re (phi - Y)^dag (dD/dt) X (dD(mu')/dt = dD(mu)/dt: the twist is constant).

Momenta P = sum_a P_a lambda_a / 2, kinetic energy sum_a P_a^2 / 2, equations of motion
dU/dt = i P U, dP_a/dt = -f_a with f_a = tr(lambda_a / 2 F).  One step of size e of the
minimal-norm scheme on a time scale: P -= lam e f; inner(e / 2); P -= (1 - 2 lam) e f;
inner(e / 2); P -= lam e f, lam = 0.1931833275037836, where inner() runs the next time scale (the
link update U <- exp(i t P) U innermost).

Pinned by tests/test_oracle_hmc.py: the gauge and ratio forces against central finite differences;
the integrator's second order (|dH| falls by about 4 when the step halves); reversibility (momenta
flipped after a trajectory, a second trajectory returns to the start).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import dirac, force as fforce

LAMBDA_MN = 0.1931833275037836


def plaquette(U, mu, nu):
    Um, Un = U[..., mu, :, :], U[..., nu, :, :]
    return Um @ dirac.shift_fwd(Un, mu) @ dirac.dagger(dirac.shift_fwd(Um, nu)) @ dirac.dagger(Un)


def gauge_action(U, beta):
    s = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            s += np.sum(1.0 - np.real(np.trace(plaquette(U, mu, nu), axis1=-2, axis2=-1)) / 3.0)
    return beta * float(s)


def gauge_force(U, beta):
    F = np.zeros(U.shape, dtype=np.complex128)
    f, b = dirac.shift_fwd, dirac.shift_bwd
    for mu in range(4):
        Um = U[..., mu, :, :]
        S = np.zeros_like(Um)
        for nu in range(4):
            if nu == mu:
                continue
            Un = U[..., nu, :, :]
            # upper staple U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
            S += f(Un, mu) @ dirac.dagger(f(Um, nu)) @ dirac.dagger(Un)
            # lower staple U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)
            S += dirac.dagger(b(f(Un, mu), nu)) @ dirac.dagger(b(Um, nu)) @ b(Un, nu)
        W = Um @ S
        F[..., mu, :, :] = (beta / 3.0) * fforce._traceless_hermitian((W - dirac.dagger(W)) / 2j)
    return F


@dataclasses.dataclass
class Monomial:
    kind: str            # "gauge", "det" or "ratio"
    mu: float = 0.0      # twist of D(mu) (det, ratio)
    mu2: float = 0.0     # mu' of the ratio's denominator factor
    beta: float = 0.0    # gauge coupling
    phi: np.ndarray = None


class Trajectory:
    """Monomials, their time scales and FP64 solves (CG on the normal equations, tolerance tol)."""

    def __init__(self, U, p: dirac.Params, monomials, levels, tol=1e-13):
        self.U, self.p, self.mons, self.levels, self.tol = U.copy(), p, monomials, levels, tol

    def _D(self, x, mu, U=None):
        U = self.U if U is None else U
        return dirac.apply_D(U, x, self.p, mu, dirac.clover_term(U, self.p.csw))

    def _Ddag(self, x, mu, U=None):
        U = self.U if U is None else U
        return dirac.apply_Ddag(U, x, self.p, mu, dirac.clover_term(U, self.p.csw))

    def _solve(self, b, mu, dag=False):
        """D(mu)^-1 b (dag False) or D(mu)^-dag b (dag True), CG on the normal equations."""
        from . import krylov
        C = dirac.clover_term(self.U, self.p.csw)
        D = lambda v: dirac.apply_D(self.U, v, self.p, mu, C)
        Dd = lambda v: dirac.apply_Ddag(self.U, v, self.p, mu, C)
        x, _, _ = krylov.cg_normal(Dd, D, b, tol=self.tol) if dag else krylov.cg_normal(D, Dd, b, tol=self.tol)
        return x

    def heatbath(self, etas):
        k = 0
        for m in self.mons:
            if m.kind == "det":
                m.phi = self._D(etas[k], m.mu)
                k += 1
            elif m.kind == "ratio":
                m.phi = self._solve(self._Ddag(etas[k], m.mu), m.mu2, dag=True)
                k += 1

    def action(self, m):
        if m.kind == "gauge":
            return gauge_action(self.U, m.beta)
        if m.kind == "det":
            y = self._solve(m.phi, m.mu)
        else:
            y = self._solve(self._Ddag(m.phi, m.mu2), m.mu, dag=True)
        return float(np.real(np.vdot(y.ravel(), y.ravel())))

    def force(self, m):
        if m.kind == "gauge":
            return gauge_force(self.U, m.beta)
        p = dataclasses.replace(self.p, mu=m.mu)
        if m.kind == "det":
            Y = self._solve(m.phi, m.mu)
            X = self._solve(Y, m.mu, dag=True)
            return fforce._traceless_hermitian(-2.0 * fforce.link_derivative(self.U, X, Y, p))
        Y = self._solve(self._Ddag(m.phi, m.mu2), m.mu, dag=True)
        X = self._solve(Y, m.mu)
        return fforce._traceless_hermitian(-2.0 * fforce.link_derivative(self.U, Y - m.phi, X, p))

    def hamiltonian(self, P):
        return 0.5 * float(np.sum(P * P)) + sum(self.action(m) for m in self.mons)

    def _update_P(self, P, level, e):
        for m in self.levels[level][0]:
            P -= e * fforce.matrix_to_algebra(self.force(m))

    def _evolve(self, P, level, t):
        if level == len(self.levels):
            H = fforce.algebra_to_matrix(P)
            w, V = np.linalg.eigh(H)
            E = np.einsum("...ab,...b,...cb->...ac", V, np.exp(1j * t * w), np.conj(V))
            self.U = E @ self.U
            return
        n = self.levels[level][1]
        e = t / n
        for _ in range(n):
            self._update_P(P, level, LAMBDA_MN * e)
            self._evolve(P, level + 1, 0.5 * e)
            self._update_P(P, level, (1.0 - 2.0 * LAMBDA_MN) * e)
            self._evolve(P, level + 1, 0.5 * e)
            self._update_P(P, level, LAMBDA_MN * e)

    def run(self, P0, tau):
        """Integrate (U, P0) for a time tau; returns (P, dH)."""
        P = P0.copy()
        H0 = self.hamiltonian(P)
        self._evolve(P, 0, tau)
        return P, self.hamiltonian(P) - H0
