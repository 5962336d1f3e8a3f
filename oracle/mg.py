"""FP64 oracle of the DD-alpha-AMG pieces (test infrastructure only).

Eq. 1 of arXiv:1710.06198 gives the two-level error propagation

    eps <- (I - M D)^k (I - P D_c^-1 P^dag D) eps,

with M the SAP smoother (Sec. 1.1, Luescher's Schwarz alternating procedure), P the
aggregation-based prolongation built from N_v test vectors, Gamma5-compatible (G5 P = P G5_c), and
D_c = P^dag D P.  The paper fixes only this structure; the details below are the readings this
project adopts (listed with their reasons in the design notes):

* SAP: lattice cut into blocks; a block's colour is the parity of its block coordinates.  One sweep
  visits colour 0 then colour 1; for every block of the colour, r_B = (b - D x)|_B, then n_mr
  minimal-residual steps on D_B (D restricted to the block with zero Dirichlet data outside; clover
  and twist included), then x_B += e_B.
* Aggregation: aggregates are lattice blocks.  Each test vector is split into its chirality halves
  (spins 0,1 = +, spins 2,3 = -); within each (aggregate, chirality) the N_v pieces are
  orthonormalised by modified Gram-Schmidt, applied twice, in the order j = 0..N_v-1.  Coarse
  degrees of freedom per coarse site are ordered [+: 0..N_v-1, -: 0..N_v-1], so
  G5_c = diag(+1 x N_v, -1 x N_v).
* D_c is stored as a 9-point stencil: a self block and one block per face (+mu, -mu), each built
  from the fine hops that cross that face.  The twist is excluded from the stored blocks and added
  as +i mu G5_c on application (D_c(mu) = D_c + i mu G5_c, Sec. 1.1).
* Cycle (right preconditioner of FGMRES): from z = 0, coarse correction first,
  z = P D_c^-1 P^dag r, with D_c^-1 replaced by one GMRES cycle from zero (at most m_c steps,
  stopping at relative residual rtol_c), then k SAP sweeps on D z = r.  This is Eq. 1 applied to
  the error of the zero initial guess.
* Setup: N_v caller-given random vectors; n_init passes of v_j <- normalise(M_SAP^k v_j) from
  x = 0; build P and D_c; then n_iter passes of v_j <- normalise(cycle(v_j)) with P and D_c
  rebuilt after each pass (the adaptive setup iterations of Sec. 2).

* Optionally the coarse solve runs on the odd-even reduced system (not in the paper; an addition of
  this project): with even coarse extents, S x_o = b_o - A_oe A_ee^-1 b_e with the Schur complement
  S = A_oo - A_oe A_ee^-1 A_eo, then x_e = A_ee^-1 (b_e - A_eo x_o).

Pinned by (tests/test_oracle_mg.py): P^dag P = I, G5 P = P G5_c, D_c x_c = P^dag D P x_c,
D_c(mu) - D_c(0) = i mu G5_c, D_c^dag = G5_c D_c G5_c, the dense SAP error propagator, exact
coarse correction with full-rank P, dense LU solutions, the cycle's dense error propagator
I - C D = (I - M D)^k (I - P D_c^-1 P^dag D) of Eq. 1 with exact inner solves, and for the
odd-even coarse solve: D_c applied to (x_o, -A_ee^-1 A_eo x_o) equals (S x_o, 0), the assembled
dense S equals the dense block elimination, and a full-dimension cycle equals the dense solve.

Parity unpinned: Hierarchy.setup.  The adaptive setup has many correct results (any test vectors
that span the near-null space do); it is compared only through what it feeds, never by value.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import dirac, krylov

# ---------------------------------------------------------------- block geometry


def _lat(shape_tail_dims, f):
    return f.shape[f.ndim - 4 - shape_tail_dims: f.ndim - shape_tail_dims]


def to_blocks(f, bdims, ntail):
    """f[..., T, Z, Y, X, *tail] -> f[..., nT, nZ, nY, nX, bt, bz, by, bx, *tail]."""
    bx, by, bz, bt = bdims
    lead = f.shape[: f.ndim - 4 - ntail]
    T, Z, Y, X = f.shape[f.ndim - 4 - ntail: f.ndim - ntail]
    tail = f.shape[f.ndim - ntail:]
    g = f.reshape(lead + (T // bt, bt, Z // bz, bz, Y // by, by, X // bx, bx) + tail)
    nl = len(lead)
    perm = list(range(nl)) + [nl + 0, nl + 2, nl + 4, nl + 6, nl + 1, nl + 3, nl + 5, nl + 7] + \
        list(range(nl + 8, nl + 8 + ntail))
    return g.transpose(perm)


def from_blocks(g, ntail):
    nl = g.ndim - 8 - ntail
    lead = g.shape[:nl]
    nT, nZ, nY, nX, bt, bz, by, bx = g.shape[nl: nl + 8]
    tail = g.shape[nl + 8:]
    perm = list(range(nl)) + [nl + 0, nl + 4, nl + 1, nl + 5, nl + 2, nl + 6, nl + 3, nl + 7] + \
        list(range(nl + 8, nl + 8 + ntail))
    return g.transpose(perm).reshape(lead + (nT * bt, nZ * bz, nY * by, nX * bx) + tail)


def coords(lat_shape):
    """(x, y, z, t) coordinate arrays of a (T, Z, Y, X) lattice."""
    c = np.indices(lat_shape)
    return [c[3], c[2], c[1], c[0]]


def block_colour(lat_shape, bdims):
    """Colour (0/1) of the block containing each site: parity of the block coordinates."""
    c = coords(lat_shape)
    return sum(c[mu] // bdims[mu] for mu in range(4)) % 2


# ---------------------------------------------------------------- SAP (Sec. 1.1, Eq. 1: M)
def hopping_masked(U, psi, tbc, fwd_mask, bwd_mask):
    """Hopping term with the hops selected by per-site masks (fwd_mask[mu], bwd_mask[mu])."""
    out = np.zeros_like(psi)
    for mu in range(4):
        Umu = U[..., mu, :, :]
        fwd = dirac.colour_mul(Umu, dirac.shift_fwd(psi, mu, tbc))
        bwd = dirac.shift_bwd(dirac.colour_mul_dag(Umu, psi), mu, tbc)
        out += fwd_mask[mu][..., None, None] * dirac.spin_mul(dirac.I4 - dirac.GAMMA[mu], fwd)
        out += bwd_mask[mu][..., None, None] * dirac.spin_mul(dirac.I4 + dirac.GAMMA[mu], bwd)
    return -0.5 * out


def inner_masks(lat_shape, bdims):
    """Masks of the hops that stay inside a block (x_mu+1 resp. x_mu-1 in the same block)."""
    c = coords(lat_shape)
    fwd = [(c[mu] % bdims[mu]) != bdims[mu] - 1 for mu in range(4)]
    bwd = [(c[mu] % bdims[mu]) != 0 for mu in range(4)]
    return fwd, bwd


def apply_D_blocks(U, psi, p: dirac.Params, clover, bdims, mu=None, twist=True):
    """Block-diagonal Dirichlet operator: sum_B D_B (hops across block faces dropped)."""
    mu = p.mu if mu is None else mu
    lat = U.shape[:4]
    fm, bm = inner_masks(lat, bdims)
    out = (4.0 + p.m0) * psi + dirac.site_matrix_mul(clover, psi) + hopping_masked(U, psi, p.tbc, fm, bm)
    if twist:
        out = out + 1j * mu * dirac.apply_g5(psi)
    return out


def block_inner(a, b, bdims):
    """Per-block <a, b> over sites and spin-colour: result[..., nT, nZ, nY, nX]."""
    g = to_blocks(np.conj(a) * b, bdims, 2)
    return g.sum(axis=(-6, -5, -4, -3, -2, -1))


def block_broadcast(vals, bdims):
    """Per-block scalars -> per-site field [..., T, Z, Y, X, 1, 1]."""
    bx, by, bz, bt = bdims
    v = np.repeat(vals, bt, axis=-4)
    v = np.repeat(v, bz, axis=-3)
    v = np.repeat(v, by, axis=-2)
    v = np.repeat(v, bx, axis=-1)
    return v[..., None, None]


def block_mr(U, p, clover, r, bdims, n_mr, mu=None):
    """n_mr MR steps on every block simultaneously, each block with its own step length."""
    e = np.zeros_like(r)
    r = r.copy()
    for _ in range(n_mr):
        q = apply_D_blocks(U, r, p, clover, bdims, mu)
        qq = np.real(block_inner(q, q, bdims))
        qr = block_inner(q, r, bdims)
        a = np.where(qq > 0, qr / np.where(qq > 0, qq, 1.0), 0.0)
        ab = block_broadcast(a, bdims)
        e += ab * r
        r -= ab * q
    return e


def sap(U, p, clover, b, bdims, n_sweeps, n_mr, x0=None, mu=None):
    """Multiplicative SAP: n_sweeps x (colour 0, colour 1) block-MR updates of D x = b.

    Needs an even number (>= 2) of blocks along every direction so that blocks of one colour never
    touch and every hop that leaves a block really couples two different blocks.
    """
    lat = U.shape[:4]
    for d in range(4):
        nb = lat[3 - d] // bdims[d]
        if nb < 2 or nb % 2 or lat[3 - d] % bdims[d]:
            raise ValueError("SAP needs an even number of blocks >= 2 in every direction")
    col = block_colour(lat, bdims)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    for _ in range(n_sweeps):
        for c in (0, 1):
            r = b - dirac.apply_D(U, x, p, mu, clover)
            rc = r * (col == c)[..., None, None]
            x = x + block_mr(U, p, clover, rc, bdims, n_mr, mu)
    return x


# ---------------------------------------------------------------- aggregation P (Sec. 1.1)
def orthonormalise(vectors, adims):
    """Per (aggregate, chirality) modified Gram-Schmidt, twice, over j = 0..N_v-1.

    vectors[Nv, T, Z, Y, X, 4, 3] -> W of the same shape; P e_(a, chi, j) = W_j restricted to
    aggregate a and to the spins of chirality chi.
    """
    nv = vectors.shape[0]
    b = to_blocks(vectors, adims, 2)                    # [Nv, nT,nZ,nY,nX, bt,bz,by,bx, 4, 3]
    shp = b.shape
    b = b.reshape(shp[:5] + (-1, 2, 2, 3))              # [..., sites, chi, 2 spins, 3]
    b = np.moveaxis(b, -3, 5)                           # [Nv, agg4, chi, sites, 2, 3]
    w = b.reshape(shp[:5] + (2, -1)).copy()            # [Nv, agg4, chi, n_loc]
    for _ in range(2):
        for j in range(nv):
            for i in range(j):
                ov = np.sum(np.conj(w[i]) * w[j], axis=-1, keepdims=True)
                w[j] = w[j] - ov * w[i]
            nrm = np.sqrt(np.sum(np.abs(w[j]) ** 2, axis=-1, keepdims=True))
            w[j] = w[j] / nrm
    w = w.reshape(b.shape)
    w = np.moveaxis(w, 5, -3).reshape(shp)
    return from_blocks(w, 2)


@dataclass
class Prolongator:
    W: np.ndarray          # [Nv, T, Z, Y, X, 4, 3]
    adims: tuple

    @property
    def nv(self):
        return self.W.shape[0]

    @property
    def coarse_lat(self):
        T, Z, Y, X = self.W.shape[1:5]
        ax, ay, az, at = self.adims
        return (T // at, Z // az, Y // ay, X // ax)


def prolong(P: Prolongator, c):
    """e(x)_chi = sum_j W_j(x)_chi c[a(x), chi, j]; c[..., nT, nZ, nY, nX, 2 Nv]."""
    nv = P.nv
    lead = c.shape[:-5]
    ax, ay, az, at = P.adims
    cf = np.repeat(np.repeat(np.repeat(np.repeat(c, at, axis=-5), az, axis=-4), ay, axis=-3), ax, axis=-2)
    cp = cf[..., :nv]   # [..., T, Z, Y, X, Nv]
    cm = cf[..., nv:]
    e = np.zeros(lead + P.W.shape[1:], dtype=np.complex128)
    e[..., 0:2, :] = np.einsum("j...sa,...j->...sa", P.W[..., 0:2, :], cp)
    e[..., 2:4, :] = np.einsum("j...sa,...j->...sa", P.W[..., 2:4, :], cm)
    return e


def restrict(P: Prolongator, r):
    """c[a, chi, j] = sum_{x in a} W_j(x)_chi^dag r(x)_chi  (P^dag r)."""
    nv = P.nv
    sp = np.einsum("j...sa,...sa->...j", np.conj(P.W[..., 0:2, :]), r[..., 0:2, :])
    sm = np.einsum("j...sa,...sa->...j", np.conj(P.W[..., 2:4, :]), r[..., 2:4, :])
    s = np.concatenate([sp, sm], axis=-1)              # [..., T, Z, Y, X, 2Nv]
    g = to_blocks(s, P.adims, 1)
    return g.sum(axis=(-5, -4, -3, -2))


def coarse_gamma5(nv):
    return np.concatenate([np.ones(nv), -np.ones(nv)])


# ---------------------------------------------------------------- coarse operator D_c = P^dag D P
@dataclass
class CoarseOp:
    self_blk: np.ndarray   # [nT, nZ, nY, nX, nd, nd]
    fwd: np.ndarray        # [4, nT, nZ, nY, nX, nd, nd]  block coupling a to a+mu
    bwd: np.ndarray        # [4, nT, nZ, nY, nX, nd, nd]  block coupling a to a-mu
    nv: int
    extra: dict = field(default_factory=dict)


def build_coarse(U, p: dirac.Params, clover, P: Prolongator):
    """Stencil blocks of P^dag D_W P (twist excluded), one column per coarse dof l:

    w_l = P e_l on every aggregate at once; self = P^dag (aggregate-Dirichlet D_W) w_l;
    fwd[mu] = P^dag (hops x -> x+mu crossing the +mu face) w_l;
    bwd[mu] = P^dag (hops x -> x-mu crossing the -mu face) w_l.
    """
    nv = P.nv
    nd = 2 * nv
    lat = U.shape[:4]
    clat = P.coarse_lat
    c = coords(lat)
    self_blk = np.zeros(clat + (nd, nd), dtype=np.complex128)
    fwd = np.zeros((4,) + clat + (nd, nd), dtype=np.complex128)
    bwd = np.zeros((4,) + clat + (nd, nd), dtype=np.complex128)
    for l in range(nd):
        chi, j = divmod(l, nv)
        w = np.zeros(lat + (4, 3), dtype=np.complex128)
        sl = slice(0, 2) if chi == 0 else slice(2, 4)
        w[..., sl, :] = P.W[j][..., sl, :]
        s = apply_D_blocks(U, w, p, clover, P.adims, mu=0.0, twist=False)
        self_blk[..., :, l] = restrict(P, s)
        for mu in range(4):
            Umu = U[..., mu, :, :]
            face_f = (c[mu] % P.adims[mu]) == P.adims[mu] - 1
            face_b = (c[mu] % P.adims[mu]) == 0
            hf = -0.5 * dirac.spin_mul(dirac.I4 - dirac.GAMMA[mu],
                                       dirac.colour_mul(Umu, dirac.shift_fwd(w, mu, p.tbc)))
            hb = -0.5 * dirac.spin_mul(dirac.I4 + dirac.GAMMA[mu],
                                       dirac.shift_bwd(dirac.colour_mul_dag(Umu, w), mu, p.tbc))
            fwd[mu][..., :, l] = restrict(P, hf * face_f[..., None, None])
            bwd[mu][..., :, l] = restrict(P, hb * face_b[..., None, None])
    return CoarseOp(self_blk, fwd, bwd, nv)


def _cshift(c, mu, sign):
    # coarse fields carry (..., nT, nZ, nY, nX, dof): the axis of direction mu is -2 - mu
    return np.roll(c, -sign, axis=-2 - mu)


def coarse_apply(Dc: CoarseOp, x, mu=0.0):
    """y(a) = A_self(a) x(a) + sum_mu [A_+mu(a) x(a+mu) + A_-mu(a) x(a-mu)] + i mu G5_c x(a)."""
    y = np.einsum("...kl,...l->...k", Dc.self_blk, x)
    for m in range(4):
        y += np.einsum("...kl,...l->...k", Dc.fwd[m], _cshift(x, m, +1))
        y += np.einsum("...kl,...l->...k", Dc.bwd[m], _cshift(x, m, -1))
    return y + 1j * mu * coarse_gamma5(Dc.nv) * x


def coarse_parity(Dc: CoarseOp):
    """Parity (0 even, 1 odd) of every coarse site, from the sum of its coarse coordinates."""
    lat = Dc.self_blk.shape[:-2]
    if any(n % 2 for n in lat):
        raise ValueError("odd-even splitting of the coarse lattice needs even extents")
    return np.indices(lat).sum(axis=0) % 2


def coarse_hops(Dc: CoarseOp, x):
    """The nearest-neighbour part of D_c: y(a) = sum_mu [A_+mu(a) x(a+mu) + A_-mu(a) x(a-mu)]."""
    y = np.zeros_like(x)
    for m in range(4):
        y += np.einsum("...kl,...l->...k", Dc.fwd[m], _cshift(x, m, +1))
        y += np.einsum("...kl,...l->...k", Dc.bwd[m], _cshift(x, m, -1))
    return y


def coarse_site_term(Dc: CoarseOp, x, mu=0.0):
    """The site-local part of D_c(mu): A_self(a) x(a) + i mu G5_c x(a)."""
    return np.einsum("...kl,...l->...k", Dc.self_blk, x) + 1j * mu * coarse_gamma5(Dc.nv) * x


def coarse_site_inverse(Dc: CoarseOp, mu=0.0):
    """(A_self(a) + i mu G5_c)^-1 for every coarse site (dense inverse of each block)."""
    nd = Dc.self_blk.shape[-1]
    blk = Dc.self_blk + 1j * mu * np.diag(coarse_gamma5(Dc.nv)).reshape((1,) * (Dc.self_blk.ndim - 2) + (nd, nd))
    return np.linalg.inv(blk)


def coarse_schur_apply(Dc: CoarseOp, x, mu, inv=None):
    """S x on the odd sites, S = A_oo - A_oe A_ee^-1 A_eo: the Schur complement of D_c(mu) after
    eliminating the even sites (with even coarse extents every hop joins sites of opposite parity,
    so A_ee and A_oo are the site-local blocks).  x and the result carry zeros on the even sites."""
    par = coarse_parity(Dc)[..., None]
    inv = coarse_site_inverse(Dc, mu) if inv is None else inv
    t = np.einsum("...kl,...l->...k", inv, coarse_hops(Dc, x)) * (par == 0)
    return (coarse_site_term(Dc, x, mu) - coarse_hops(Dc, t)) * (par == 1)


def coarse_solve_eo(Dc: CoarseOp, b, mu, m, rtol):
    """D_c(mu)^-1 b by odd-even reduction: one GMRES cycle from zero (at most m steps, stop at
    relative residual rtol of the reduced system) on S x_o = b_o - A_oe A_ee^-1 b_e, then
    x_e = A_ee^-1 (b_e - A_eo x_o)."""
    par = coarse_parity(Dc)[..., None]
    inv = coarse_site_inverse(Dc, mu)
    te = np.einsum("...kl,...l->...k", inv, b * (par == 0))
    rhs = (b - coarse_hops(Dc, te)) * (par == 1)
    xo, k = krylov.gmres_fixed(lambda v: coarse_schur_apply(Dc, v, mu, inv), rhs, m, rtol)
    xe = np.einsum("...kl,...l->...k", inv, (b - coarse_hops(Dc, xo)) * (par == 0)) * (par == 0)
    return xo * (par == 1) + xe


def coarse_apply_definition(U, p, clover, P, x, mu=None):
    """D_c(mu) x = P^dag D(mu) P x, straight from the definition (Sec. 1.1)."""
    return restrict(P, dirac.apply_D(U, prolong(P, x), p, mu, clover))


def coarse_apply_nd(Dc: CoarseOp, x2, mubar, epsbar, delta=0.0):
    """D_ND,c = D_c x I2 + i mubar G5_c x tau3 - epsbar I x tau1 (Sec. 1.1, Eq. 2 coarsened), plus
    i delta G5_c x tau1 for the shifted doublet (P_ND^dag (G5 x tau1) P_ND = G5_c x tau1)."""
    u = coarse_apply(Dc, x2[0], mubar) - epsbar * x2[1]
    d = coarse_apply(Dc, x2[1], -mubar) - epsbar * x2[0]
    if delta:
        g = coarse_gamma5(Dc.nv)
        u = u + 1j * delta * g * x2[1]
        d = d + 1j * delta * g * x2[0]
    return np.stack([u, d])


def coarse_dense(Dc: CoarseOp, mu=0.0):
    shp = Dc.self_blk.shape[:4] + (2 * Dc.nv,)
    return dirac.dense_matrix(lambda v: coarse_apply(Dc, v, mu), shp)


# ---------------------------------------------------------------- cycle, setup, solve
@dataclass
class MGParams:
    block: tuple = (4, 4, 4, 4)       # SAP block (x, y, z, t)
    agg: tuple = (4, 4, 4, 4)         # aggregate (x, y, z, t)
    nv: int = 8
    sap_sweeps: int = 3               # k of Eq. 1
    sap_mr: int = 4                   # MR steps per block solve
    coarse_m: int = 30                # max GMRES steps of the coarse solve
    coarse_rtol: float = 5e-2
    n_init: int = 5                   # initial SAP inverse-iteration passes
    n_iter: int = 3                   # adaptive setup iterations
    restart: int = 10                 # outer FGMRES restart length
    coarse_eo: bool = False           # coarse solve on the odd-even reduced system (coarse_solve_eo)


class Hierarchy:
    """Two-level DD-alpha-AMG hierarchy: operator data, P and D_c."""

    def __init__(self, U, p: dirac.Params, mg: MGParams, clover=None):
        self.U, self.p, self.mg = U, p, mg
        self.clover = dirac.clover_term(U, p.csw) if clover is None else clover
        self.P = None
        self.Dc = None

    def D(self, x, mu=None):
        return dirac.apply_D(self.U, x, self.p, mu, self.clover)

    def smooth(self, b, x0, mu=None):
        return sap(self.U, self.p, self.clover, b, self.mg.block, self.mg.sap_sweeps, self.mg.sap_mr,
                   x0, mu)

    def set_vectors(self, v):
        self.P = Prolongator(orthonormalise(v, self.mg.agg), tuple(self.mg.agg))
        self.Dc = build_coarse(self.U, self.p, self.clover, self.P)

    def coarse_solve(self, c, mu=None):
        mu = self.p.mu if mu is None else mu
        if self.mg.coarse_eo:
            return coarse_solve_eo(self.Dc, c, mu, self.mg.coarse_m, self.mg.coarse_rtol)
        e, _ = krylov.gmres_fixed(lambda v: coarse_apply(self.Dc, v, mu), c, self.mg.coarse_m,
                                  self.mg.coarse_rtol)
        return e

    def cycle(self, r, mu=None):
        """Eq. 1 on the zero initial guess: coarse correction, then k SAP sweeps."""
        z = prolong(self.P, self.coarse_solve(restrict(self.P, r), mu))
        return self.smooth(r, z, mu)

    def setup(self, v0):
        """Adaptive setup (Sec. 1.1, Sec. 2).  Parity unpinned: its result is not unique."""
        v = np.array(v0, dtype=np.complex128, copy=True)
        for _ in range(self.mg.n_init):
            for j in range(v.shape[0]):
                x = self.smooth(v[j], None)
                v[j] = x / np.sqrt(dirac.norm2(x))
        self.set_vectors(v)
        for _ in range(self.mg.n_iter):
            for j in range(v.shape[0]):
                x = self.cycle(v[j])
                v[j] = x / np.sqrt(dirac.norm2(x))
            self.set_vectors(v)
        return v

    def solve(self, b, tol=1e-10, maxiter=2000, mu=None):
        return krylov.fgmres(lambda x: self.D(x, mu), b, lambda r: self.cycle(r, mu),
                             m=self.mg.restart, tol=tol, maxiter=maxiter)


# ---------------------------------------------------------------- third level (coarse aggregation)
# Readings for three levels (the paper runs three levels, Sec. 1.2, without further detail): the
# level-1 operator D_c is coarsened again by aggregating blocks of level-1 sites with N_v2 level-1
# test vectors, split by the level-1 chirality (G5_c), orthonormalised like the fine level; the
# level-1 system is solved by FGMRES (a K-cycle) preconditioned by a level-1 cycle made of the
# level-2 coarse-grid correction followed by a few GMRES steps on D_c (SAP needs an even number of
# blocks, which the level-1 lattices of the workloads do not have).


def to_blocks_c(f, bdims):
    return to_blocks(f, bdims, 1)


def orthonormalise_c(vectors, adims, nv1):
    """vectors[Nv2, nT, nZ, nY, nX, 2 nv1] -> W2 orthonormalised per (level-2 aggregate, level-1
    chirality) by modified Gram-Schmidt applied twice, j = 0..Nv2-1."""
    nv2 = vectors.shape[0]
    b = to_blocks_c(vectors, adims)                      # [Nv2, agg4, bt,bz,by,bx, 2 nv1]
    shp = b.shape
    b = b.reshape(shp[:5] + (-1, 2, nv1))                # [..., sites, chi, nv1]
    b = np.moveaxis(b, -2, 5)                            # [Nv2, agg4, chi, sites, nv1]
    w = b.reshape(shp[:5] + (2, -1)).copy()
    for _ in range(2):
        for j in range(nv2):
            for i in range(j):
                ov = np.sum(np.conj(w[i]) * w[j], axis=-1, keepdims=True)
                w[j] = w[j] - ov * w[i]
            w[j] = w[j] / np.sqrt(np.sum(np.abs(w[j]) ** 2, axis=-1, keepdims=True))
    w = w.reshape(b.shape)
    w = np.moveaxis(w, 5, -2).reshape(shp)
    return from_blocks(w, 1)


@dataclass
class Prolongator2:
    W: np.ndarray          # [Nv2, nT, nZ, nY, nX, 2 nv1]
    adims: tuple
    nv1: int

    @property
    def nv(self):
        return self.W.shape[0]

    @property
    def coarse_lat(self):
        T, Z, Y, X = self.W.shape[1:5]
        ax, ay, az, at = self.adims
        return (T // at, Z // az, Y // ay, X // ax)


def prolong_c(P: Prolongator2, c):
    """level-1 vector e(a)_chi = sum_j W2_j(a)_chi c[a2(a), chi, j]."""
    nv, nv1 = P.nv, P.nv1
    ax, ay, az, at = P.adims
    cf = np.repeat(np.repeat(np.repeat(np.repeat(c, at, axis=-5), az, axis=-4), ay, axis=-3), ax, axis=-2)
    e = np.zeros(c.shape[:-5] + P.W.shape[1:], dtype=np.complex128)
    e[..., :nv1] = np.einsum("j...k,...j->...k", P.W[..., :nv1], cf[..., :nv])
    e[..., nv1:] = np.einsum("j...k,...j->...k", P.W[..., nv1:], cf[..., nv:])
    return e


def restrict_c(P: Prolongator2, r):
    """c[a2, chi, j] = sum_{a in a2} W2_j(a)_chi^dag r(a)_chi."""
    nv1 = P.nv1
    sp = np.einsum("j...k,...k->...j", np.conj(P.W[..., :nv1]), r[..., :nv1])
    sm = np.einsum("j...k,...k->...j", np.conj(P.W[..., nv1:]), r[..., nv1:])
    s = np.concatenate([sp, sm], axis=-1)
    return to_blocks_c(s, P.adims).sum(axis=(-5, -4, -3, -2))


def coarse_inner_masks(clat, adims):
    c = coords(clat)
    fwd = [(c[mu] % adims[mu]) != adims[mu] - 1 for mu in range(4)]
    bwd = [(c[mu] % adims[mu]) != 0 for mu in range(4)]
    return fwd, bwd


def build_coarse_c(Dc: CoarseOp, P: Prolongator2):
    """Stencil blocks of P2^dag D_c P2 (twist excluded), column by column like build_coarse."""
    nv2 = P.nv
    nd2 = 2 * nv2
    nv1 = P.nv1
    clat = Dc.self_blk.shape[:4]
    c2 = P.coarse_lat
    c = coords(clat)
    fm, bm = coarse_inner_masks(clat, P.adims)
    self_blk = np.zeros(c2 + (nd2, nd2), dtype=np.complex128)
    fwd = np.zeros((4,) + c2 + (nd2, nd2), dtype=np.complex128)
    bwd = np.zeros((4,) + c2 + (nd2, nd2), dtype=np.complex128)
    mv = lambda A, v: np.einsum("...kl,...l->...k", A, v)
    for l in range(nd2):
        chi, j = divmod(l, nv2)
        w = np.zeros(clat + (2 * nv1,), dtype=np.complex128)
        sl = slice(0, nv1) if chi == 0 else slice(nv1, 2 * nv1)
        w[..., sl] = P.W[j][..., sl]
        s = mv(Dc.self_blk, w)
        for mu in range(4):
            s = s + fm[mu][..., None] * mv(Dc.fwd[mu], _cshift(w, mu, +1))
            s = s + bm[mu][..., None] * mv(Dc.bwd[mu], _cshift(w, mu, -1))
        self_blk[..., :, l] = restrict_c(P, s)
        for mu in range(4):
            face_f = (c[mu] % P.adims[mu]) == P.adims[mu] - 1
            face_b = (c[mu] % P.adims[mu]) == 0
            hf = mv(Dc.fwd[mu], _cshift(w, mu, +1)) * face_f[..., None]
            hb = mv(Dc.bwd[mu], _cshift(w, mu, -1)) * face_b[..., None]
            fwd[mu][..., :, l] = restrict_c(P, hf)
            bwd[mu][..., :, l] = restrict_c(P, hb)
    return CoarseOp(self_blk, fwd, bwd, nv2)


@dataclass
class MGParams3:
    agg2: tuple = (2, 2, 2, 2)     # level-2 aggregate in level-1 sites (x, y, z, t)
    nv2: int = 8
    smooth_m: int = 3              # GMRES steps of the level-1 smoother
    k_restart: int = 10            # level-1 FGMRES (K-cycle) restart
    k_rtol: float = 1e-1
    k_maxiter: int = 10
    coarse_m: int = 30             # level-2 GMRES
    coarse_rtol: float = 5e-2
    n_init: int = 5
    n_iter: int = 3


class Level1:
    """The level-1 operator D_c with its own aggregation: cycle and K-cycle solve."""

    def __init__(self, Dc: CoarseOp, prm: MGParams3):
        self.Dc, self.prm = Dc, prm
        self.P2 = None
        self.Dcc = None

    def A(self, x, mu):
        return coarse_apply(self.Dc, x, mu)

    def set_vectors(self, v):
        self.P2 = Prolongator2(orthonormalise_c(v, self.prm.agg2, self.Dc.nv), tuple(self.prm.agg2), self.Dc.nv)
        self.Dcc = build_coarse_c(self.Dc, self.P2)

    def smooth(self, b, x, mu):
        """x + (at most smooth_m GMRES steps on D_c(mu) e = b - D_c x, from zero)."""
        r = b - self.A(x, mu)
        e, _ = krylov.gmres_fixed(lambda v: self.A(v, mu), r, self.prm.smooth_m, 0.0)
        return x + e

    def cycle(self, r, mu):
        c = restrict_c(self.P2, r)
        e2, _ = krylov.gmres_fixed(lambda v: coarse_apply(self.Dcc, v, mu), c, self.prm.coarse_m,
                                   self.prm.coarse_rtol)
        z = prolong_c(self.P2, e2)
        return self.smooth(r, z, mu)

    def solve(self, b, mu):
        """The level-1 K-cycle: FGMRES on D_c preconditioned by the level-1 cycle, from zero."""
        x, _, _ = krylov.fgmres(lambda v: self.A(v, mu), b, lambda r: self.cycle(r, mu),
                                m=self.prm.k_restart, tol=self.prm.k_rtol, maxiter=self.prm.k_maxiter)
        return x

    def setup(self, v0, mu):
        v = np.array(v0, dtype=np.complex128, copy=True)
        for _ in range(self.prm.n_init):
            for j in range(v.shape[0]):
                x = self.smooth(v[j], np.zeros_like(v[j]), mu)
                v[j] = x / np.sqrt(np.real(np.vdot(x.ravel(), x.ravel())))
        self.set_vectors(v)
        for _ in range(self.prm.n_iter):
            for j in range(v.shape[0]):
                x = self.cycle(v[j], mu)
                v[j] = x / np.sqrt(np.real(np.vdot(x.ravel(), x.ravel())))
            self.set_vectors(v)
        return v


class Hierarchy3(Hierarchy):
    """Three-level DD-alpha-AMG: the coarse solve of Eq. 1 becomes the level-1 K-cycle."""

    def __init__(self, U, p, mg: MGParams, prm3: MGParams3, clover=None):
        super().__init__(U, p, mg, clover)
        self.prm3 = prm3
        self.L1 = None

    def setup3(self, v0, v1):
        self.setup(v0)
        self.L1 = Level1(self.Dc, self.prm3)
        self.L1.setup(v1, self.p.mu)

    def coarse_solve(self, c, mu=None):
        mu = self.p.mu if mu is None else mu
        if self.L1 is None:
            return super().coarse_solve(c, mu)
        return self.L1.solve(c, mu)
