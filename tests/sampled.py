"""Oracle values of an operator at single sites of a lattice too large for the oracle to apply the
operator everywhere (test infrastructure).

(D x)(s) depends on x at s and its 8 neighbours, on the links out of s and into s, and on the clover
term at s, whose leaves reach one site along two directions.  So the oracle's operator is applied,
unchanged, to a periodic 5^4 patch centred on s, copied out of the large fields, and the centre
site of the result is kept: the patch's own wrap-around lies two sites from the centre, beyond
everything the centre reads.  The antiperiodic time boundary of the large lattice is moved into the
patch's copies of the time links that cross it (every closed loop of the clover contains such a
link twice, once conjugated, so only the hops see the sign), and the patch is applied with a
periodic boundary.
"""
from __future__ import annotations

import numpy as np

from oracle import dirac

R = 2


def _axes(dims, site):
    """Index arrays (t, z, y, x) of the patch around site = (x, y, z, t)."""
    lx, ly, lz, lt = dims
    x, y, z, t = site
    return [np.arange(c - R, c + R + 1) % L for c, L in ((t, lt), (z, lz), (y, ly), (x, lx))]


def patch_links(U, dims, site, tbc):
    it, iz, iy, ix = _axes(dims, site)
    Up = U[np.ix_(it, iz, iy, ix)].copy()
    lt = dims[3]
    for k in range(2 * R):
        if it[k] == lt - 1:                    # hop t = T-1 -> 0 lies between patch slices k, k+1
            Up[k, :, :, :, 3] *= tbc
    return Up


def patch_field(psi, dims, site, lead=0):
    it, iz, iy, ix = _axes(dims, site)
    idx = (slice(None),) * lead + np.ix_(it, iz, iy, ix)
    return psi[idx]


def random_sites(dims, n, seed):
    rng = np.random.default_rng(seed)
    return [tuple(int(rng.integers(0, L)) for L in dims) for _ in range(n)]


def site_value(out, dims, site):
    """out[..., T, Z, Y, X, ...] at site = (x, y, z, t), leading axes kept."""
    x, y, z, t = site
    return out[..., t, z, y, x, :, :]


def apply_D_at(U, psi, p: dirac.Params, dims, sites, mu=None):
    """[(D(mu) psi)(s) for s in sites] as an array [n, 4, 3]."""
    q = dirac.Params(kappa=p.kappa, csw=p.csw, mu=p.mu, tbc=1, mubar=p.mubar, epsbar=p.epsbar)
    res = []
    for s in sites:
        Up = patch_links(U, dims, s, p.tbc)
        out = dirac.apply_D(Up, patch_field(psi, dims, s), q, mu)
        res.append(out[R, R, R, R])
    return np.array(res)


def apply_DND_at(U, psi2, p: dirac.Params, dims, sites):
    """[(D_ND psi2)(s) for s in sites] as an array [n, 2, 4, 3] (Eq. 2)."""
    q = dirac.Params(kappa=p.kappa, csw=p.csw, mu=p.mu, tbc=1, mubar=p.mubar, epsbar=p.epsbar)
    res = []
    for s in sites:
        Up = patch_links(U, dims, s, p.tbc)
        out = dirac.apply_DND(Up, patch_field(psi2, dims, s, lead=1), q)
        res.append(out[:, R, R, R, R])
    return np.array(res)


def values_at(field, sites, lead=0):
    """field[..., T, Z, Y, X, 4, 3] at the sites, as [n, ..., 4, 3]."""
    out = []
    for x, y, z, t in sites:
        out.append(field[(slice(None),) * lead + (t, z, y, x)])
    return np.array(out)
