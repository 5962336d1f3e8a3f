"""FP64 oracle of the fine-grid operators (test infrastructure only).

Operators (Sec. 1.1 and Eq. 2 of arXiv:1710.06198; the paper fixes their algebraic form, the
conventions below are the readings this project adopts):

* Wilson-clover operator in mass normalisation, m0 = 1/(2 kappa) - 4:
    D_W psi(x) = (4 + m0) psi(x)
                 - 1/2 sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu) ]
                 + (i c_sw / 32) sum_{mu != nu} sigma_mu_nu (Q_mu_nu(x) - Q_nu_mu(x)) psi(x),
  sigma_mu_nu = (i/2) [g_mu, g_nu], Q_mu_nu(x) = sum of the four counter-clockwise (mu -> nu)
  plaquette leaves ending at x.  Periodic in space; the time boundary sign ``tbc`` multiplies every
  hop that crosses t = T-1 <-> 0 (-1: antiperiodic).
* Twisted mass (Sec. 1.1): D(mu) = D_W + i mu G5 (G5 = g5 on the fine grid).
* Degenerate doublet: diag(D(mu), D(-mu)).
* Non-degenerate doublet (Eq. 2): D_ND = D_W x I2 + i mubar (G5 x tau3) - epsbar (I x tau1).
* Hermitian forms: Q = G5 D (Eq. 3); Q_ND = (G5 x tau1) D_ND (Eq. 4).

Gamma matrices: Euclidean chiral basis, g_k = [[0, -i s_k], [i s_k, 0]], g_4 = [[0, 1], [1, 0]],
g5 = g1 g2 g3 g4 = diag(1, 1, -1, -1), so chirality is a spin block (spins 0,1 = +, 2,3 = -).

Pins (tests/test_oracle_dirac.py): free-field plane-wave eigenvalues (closed form), uniform abelian
field clover (closed form), gamma5-hermiticity, twist identity ||D(mu)x||^2 = ||D_W x||^2 +
mu^2||x||^2, gauge covariance, Hermiticity of Q_ND, dense LU brute force.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_S = [np.array([[0, 1], [1, 0]], dtype=np.complex128),
      np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
      np.array([[1, 0], [0, -1]], dtype=np.complex128)]
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)

GAMMA = [np.block([[_Z2, -1j * s], [1j * s, _Z2]]) for s in _S] + [np.block([[_Z2, _I2], [_I2, _Z2]])]
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
I4 = np.eye(4, dtype=np.complex128)


def sigma(mu, nu):
    """sigma_mu_nu = (i/2) [g_mu, g_nu]."""
    return 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])


@dataclass
class Params:
    """Operator parameters.  kappa -> m0 = 1/(2 kappa) - 4 (mass normalisation)."""
    kappa: float
    csw: float = 0.0
    mu: float = 0.0
    tbc: int = -1
    mubar: float = 0.0
    epsbar: float = 0.0
    ndshift: float = 0.0   # delta of the shifted doublet D_ND + i delta G5 x tau1 (Sec. 3)

    @property
    def m0(self):
        return 1.0 / (2.0 * self.kappa) - 4.0


def kappa_from_m0(m0):
    return 1.0 / (2.0 * (m0 + 4.0))


# ---------------------------------------------------------------- lattice shifts
def _axis(mu):
    # fields carry (..., T, Z, Y, X, i, j): the lattice axis of direction mu (x=0 .. t=3)
    return -3 - mu


def _time_slice(field, index):
    sl = [slice(None)] * field.ndim
    sl[_axis(3)] = index
    return tuple(sl)


def shift_fwd(field, mu, tbc=1):
    """f(x + mu_hat), with the time boundary sign on the hop from t = T-1 to t = 0."""
    out = np.roll(field, -1, axis=_axis(mu))
    if mu == 3 and tbc != 1:
        out[_time_slice(out, -1)] *= tbc
    return out


def shift_bwd(field, mu, tbc=1):
    """f(x - mu_hat), with the time boundary sign on the hop from t = 0 to t = T-1."""
    out = np.roll(field, 1, axis=_axis(mu))
    if mu == 3 and tbc != 1:
        out[_time_slice(out, 0)] *= tbc
    return out


# ---------------------------------------------------------------- algebra helpers
def colour_mul(u, psi):
    """(U psi)_{s a} = sum_b U_ab psi_{s b}  (psi[..., s, b] times U^T)."""
    return np.matmul(psi, np.swapaxes(u, -1, -2))


def colour_mul_dag(u, psi):
    """(U^dag psi)_{s a} = sum_b conj(U_ba) psi_{s b}  (psi[..., s, b] times conj(U))."""
    return np.matmul(psi, np.conj(u))


def spin_mul(g, psi):
    """(G psi)_{s a} = sum_t G_st psi_{t a}."""
    return np.matmul(g, psi)


def dagger(m):
    return np.conj(np.swapaxes(m, -1, -2))


def vdot(a, b):
    """<a, b> = sum conj(a) b over all entries."""
    return np.vdot(a.ravel(), b.ravel())


def norm2(a):
    return float(np.real(np.vdot(a.ravel(), a.ravel())))


# ---------------------------------------------------------------- clover
def plaquette_leaves(U, mu, nu):
    """Q_mu_nu(x): sum of the four counter-clockwise (mu -> nu) plaquettes that start and end at x."""
    Um, Un = U[..., mu, :, :], U[..., nu, :, :]
    f, b = shift_fwd, shift_bwd
    Um_pn = f(Um, nu)            # U_mu(x+nu)
    Un_pm = f(Un, mu)            # U_nu(x+mu)
    Um_mm = b(Um, mu)            # U_mu(x-mu)
    Un_mm = b(Un, mu)            # U_nu(x-mu)
    Um_mn = b(Um, nu)            # U_mu(x-nu)
    Un_mn = b(Un, nu)            # U_nu(x-nu)
    Um_mm_pn = f(Um_mm, nu)      # U_mu(x-mu+nu)
    Um_mm_mn = b(Um_mm, nu)      # U_mu(x-mu-nu)
    Un_mm_mn = b(Un_mm, nu)      # U_nu(x-mu-nu)
    Un_pm_mn = b(Un_pm, nu)      # U_nu(x+mu-nu)
    mm = np.matmul
    leaf1 = mm(mm(mm(Um, Un_pm), dagger(Um_pn)), dagger(Un))
    leaf2 = mm(mm(mm(Un, dagger(Um_mm_pn)), dagger(Un_mm)), Um_mm)
    leaf3 = mm(mm(mm(dagger(Um_mm), dagger(Un_mm_mn)), Um_mm_mn), Un_mn)
    leaf4 = mm(mm(mm(dagger(Un_mn), Um_mn), Un_pm_mn), dagger(Um))
    return leaf1 + leaf2 + leaf3 + leaf4


def clover_term(U, csw):
    """C(x) = (i c_sw/32) sum_{mu != nu} sigma_mu_nu (x) (Q_mu_nu - Q_nu_mu), as [..., s, a, t, b].

    Pinned by: the uniform abelian-field closed form, Hermiticity, [C, g5] = 0, gauge covariance.
    """
    shp = U.shape[:-3]
    c = np.zeros(shp + (4, 3, 4, 3), dtype=np.complex128)
    if csw == 0.0:
        return c
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            f = plaquette_leaves(U, mu, nu) - plaquette_leaves(U, nu, mu)
            c += np.einsum("st,...ab->...satb", sigma(mu, nu), f)
    return (1j * csw / 32.0) * c


def site_matrix_mul(a, psi):
    """(A psi)(x) = sum_{t b} A[x, s, a, t, b] psi[x, t, b] for per-site 12x12 matrices."""
    lat = a.shape[:-4]
    am = a.reshape(lat + (12, 12))
    v = psi.reshape(psi.shape[:-2] + (12, 1))
    return np.matmul(am, v).reshape(psi.shape)


# ---------------------------------------------------------------- operators
def hopping(U, psi, tbc):
    """H psi(x) = -1/2 sum_mu [(1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu)]."""
    out = np.zeros_like(psi)
    for mu in range(4):
        Umu = U[..., mu, :, :]
        fwd = colour_mul(Umu, shift_fwd(psi, mu, tbc))
        bwd = shift_bwd(colour_mul_dag(Umu, psi), mu, tbc)
        out += spin_mul(I4 - GAMMA[mu], fwd) + spin_mul(I4 + GAMMA[mu], bwd)
    return -0.5 * out


def apply_DW(U, psi, p: Params, clover=None):
    """Wilson-clover D_W psi (twist excluded)."""
    if clover is None:
        clover = clover_term(U, p.csw)
    return (4.0 + p.m0) * psi + hopping(U, psi, p.tbc) + site_matrix_mul(clover, psi)


def apply_g5(psi):
    return spin_mul(GAMMA5, psi)


def apply_D(U, psi, p: Params, mu=None, clover=None):
    """Twisted-mass operator D(mu) psi = D_W psi + i mu g5 psi (Sec. 1.1)."""
    mu = p.mu if mu is None else mu
    return apply_DW(U, psi, p, clover) + 1j * mu * apply_g5(psi)


def apply_Ddag(U, psi, p: Params, mu=None, clover=None):
    """D(mu)^dag = g5 D(-mu) g5 (gamma5-hermiticity, Sec. 1.1)."""
    mu = p.mu if mu is None else mu
    return apply_g5(apply_D(U, apply_g5(psi), p, -mu, clover))


def apply_doublet(U, psi2, p: Params, clover=None):
    """Degenerate doublet D_W x I2 + i mu g5 x tau3 on psi2[2, ...] = diag(D(mu), D(-mu))."""
    return np.stack([apply_D(U, psi2[0], p, p.mu, clover), apply_D(U, psi2[1], p, -p.mu, clover)])


def apply_DND(U, psi2, p: Params, clover=None):
    """Non-degenerate doublet of Eq. 2 on psi2[2, ...]:
       [[D(mubar), -epsbar], [-epsbar, D(-mubar)]], plus i delta G5 x tau1 when p.ndshift = delta:
       (G5 x tau1)(D_ND + i delta G5 x tau1) = Q_ND + i delta, the shifted systems of the rational
       approximation (Sec. 3: Q_ND^2 + delta^2 = (Q_ND - i delta)(Q_ND + i delta))."""
    u = apply_D(U, psi2[0], p, p.mubar, clover) - p.epsbar * psi2[1]
    d = apply_D(U, psi2[1], p, -p.mubar, clover) - p.epsbar * psi2[0]
    if p.ndshift:
        u = u + 1j * p.ndshift * apply_g5(psi2[1])
        d = d + 1j * p.ndshift * apply_g5(psi2[0])
    return np.stack([u, d])


def apply_QND(U, psi2, p: Params, clover=None):
    """Q_ND = (G5 x tau1) D_ND (Eq. 4): g5 on the swapped flavours."""
    y = apply_DND(U, psi2, p, clover)
    return np.stack([apply_g5(y[1]), apply_g5(y[0])])


def dense_matrix(apply, shape):
    """Columns apply(e_k) for unit vectors e_k of a field of the given shape (tiny lattices only)."""
    n = int(np.prod(shape))
    cols = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for k in range(n):
        e[k] = 1.0
        cols[:, k] = apply(e.reshape(shape)).ravel()
        e[k] = 0.0
    return cols
