"""Seeded synthetic inputs shared by the FP64 oracle tests, the GPU parity tests and bench.py.

This module holds no arithmetic of the solver: it only draws random numbers and shapes them into
gauge links, spinor fields and point sources. Array conventions used throughout the project:

* lattice dims ``(Lx, Ly, Lz, T)``; direction index mu = 0, 1, 2, 3 = x, y, z, t;
* a field is a C-ordered numpy array with lattice axes ``(T, Z, Y, X)`` so that the lexicographic
  site index is ``x + Lx*(y + Ly*(z + Lz*t))``;
* gauge links: ``U[t, z, y, x, mu, a, b]`` complex128 (SU(3) row a, column b);
* spinors: ``psi[..., t, z, y, x, spin, colour]`` complex128 (4 spins, 3 colours);
* coarse vectors: ``c[..., t, z, y, x, dof]`` complex128.

Gauge recipe: for every link, in site order then mu, draw a traceless Hermitian H with N(0,1)
entries (3 real diagonal values, then Re/Im of H01, H02, H12), set U = exp(i*eps*H) through an
eigendecomposition, then re-unitarise by Gram-Schmidt of rows 0 and 1 with row 2 = conj(r0 x r1).
"""
from __future__ import annotations

import os

import numpy as np


def lattice_shape(dims):
    lx, ly, lz, lt = (int(d) for d in dims)
    return (lt, lz, ly, lx)


def _hermitian_from_normals(z):
    """z[..., 9] N(0,1) -> traceless Hermitian 3x3 matrices."""
    h = np.zeros(z.shape[:-1] + (3, 3), dtype=np.complex128)
    h[..., 0, 0] = z[..., 0]
    h[..., 1, 1] = z[..., 1]
    h[..., 2, 2] = z[..., 2]
    for k, (a, b) in enumerate(((0, 1), (0, 2), (1, 2))):
        h[..., a, b] = z[..., 3 + 2 * k] + 1j * z[..., 4 + 2 * k]
        h[..., b, a] = np.conj(h[..., a, b])
    tr = (h[..., 0, 0] + h[..., 1, 1] + h[..., 2, 2]) / 3.0
    for a in range(3):
        h[..., a, a] -= tr
    return h


def reunitarise(u):
    """Project 3x3 matrices onto SU(3): Gram-Schmidt on rows 0, 1; row 2 = conj(row0 x row1)."""
    u = np.array(u, dtype=np.complex128, copy=True)
    r0 = u[..., 0, :]
    r0 = r0 / np.sqrt(np.sum(np.abs(r0) ** 2, axis=-1, keepdims=True))
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.sqrt(np.sum(np.abs(r1) ** 2, axis=-1, keepdims=True))
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def exp_i_hermitian(h, eps):
    """exp(i*eps*H) for Hermitian H via numpy.linalg.eigh (FP64)."""
    w, v = np.linalg.eigh(h)
    ph = np.exp(1j * eps * w)
    return np.einsum("...ab,...b,...cb->...ac", v, ph, np.conj(v))


def _links(z, eps):
    return reunitarise(exp_i_hermitian(_hermitian_from_normals(z), eps))


def gauge_field(dims, eps, seed):
    """Random SU(3) links U = exp(i eps H), H traceless Hermitian with N(0,1) entries.

    Large lattices are built in chunks of time slices on a thread pool; every link is computed by
    the same per-link arithmetic from the same random numbers, so the result does not depend on the
    chunking."""
    shp = lattice_shape(dims)
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(shp + (4, 9))
    if int(np.prod(shp)) < (1 << 20) or shp[0] < 2:
        return _links(z, eps)
    from concurrent.futures import ThreadPoolExecutor
    out = np.empty(shp + (4, 3, 3), dtype=np.complex128)
    bounds = np.linspace(0, shp[0], min(shp[0], 96) + 1).astype(int)

    def work(i):
        out[bounds[i]:bounds[i + 1]] = _links(z[bounds[i]:bounds[i + 1]], eps)

    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(work, range(len(bounds) - 1)))
    return out


def unit_gauge(dims):
    shp = lattice_shape(dims)
    u = np.zeros(shp + (4, 3, 3), dtype=np.complex128)
    for a in range(3):
        u[..., a, a] = 1.0
    return u


def gauge_transform(dims, seed):
    """Random SU(3) matrix per site (QR of a complex Gaussian matrix, phase-fixed to det 1)."""
    shp = lattice_shape(dims)
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(shp + (3, 3)) + 1j * rng.standard_normal(shp + (3, 3))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(q)
    q = q / (det ** (1.0 / 3.0))[..., None, None]
    return reunitarise(q)


def gaussian_spinor(dims, seed, n=None, flavours=None):
    """Gaussian spinor(s): Re, Im ~ N(0,1) i.i.d. in index order."""
    shp = lattice_shape(dims) + (4, 3)
    lead = ()
    if n is not None:
        lead += (int(n),)
    if flavours is not None:
        lead += (int(flavours),)
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(lead + shp + (2,))
    return z[..., 0] + 1j * z[..., 1]


def gaussian_spinor_columns(dims, seed, n, flavours=None):
    """The n columns of gaussian_spinor(dims, seed, n=n, flavours=...) one at a time (the same
    random stream, drawn column by column), for lattices where all n do not fit in host memory."""
    shp = lattice_shape(dims) + (4, 3)
    lead = () if flavours is None else (int(flavours),)
    rng = np.random.default_rng(seed)
    for _ in range(int(n)):
        z = rng.standard_normal(lead + shp + (2,))
        yield z[..., 0] + 1j * z[..., 1]


def gaussian_coarse(coarse_dims, ndof, seed, n=None):
    shp = lattice_shape(coarse_dims) + (int(ndof),)
    lead = () if n is None else (int(n),)
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(lead + shp + (2,))
    return z[..., 0] + 1j * z[..., 1]


def point_sources(dims, site=(0, 0, 0, 0)):
    """12 point sources delta(x=site) delta(spin s) delta(colour c); column index 3*s + c."""
    shp = lattice_shape(dims)
    b = np.zeros((12,) + shp + (4, 3), dtype=np.complex128)
    x, y, z, t = site
    for s in range(4):
        for c in range(3):
            b[3 * s + c, t, z, y, x, s, c] = 1.0
    return b


def su3_algebra_directions(dims, seed, n):
    """n random directions omega[n, t, z, y, x, mu, 8] with N(0,1) coefficients."""
    shp = lattice_shape(dims)
    rng = np.random.default_rng(seed)
    return rng.standard_normal((int(n),) + shp + (4, 8))


def uniform_abelian_field(dims, plane, n_flux):
    """Diagonal U(1)^2 c SU(3) field with a uniform flux through every plaquette of one plane.

    For plane (mu, nu) and colour phases q = (1, -1, 0) the counter-clockwise (mu -> nu) plaquette
    equals exp(i q_c phi) with phi = 2 pi n_flux / (L_mu L_nu) on every site.  Used only to build
    closed-form expectations for the clover term.
    """
    mu, nu = plane
    shp = lattice_shape(dims)
    l = [int(d) for d in dims]
    u = unit_gauge(dims)
    phi = 2.0 * np.pi * n_flux / (l[mu] * l[nu])
    coords = np.indices(shp)  # (4, T, Z, Y, X) in (t, z, y, x) order
    c = [coords[3], coords[2], coords[1], coords[0]]  # x, y, z, t
    q = np.array([1.0, -1.0, 0.0])
    # U_mu(x) = exp(-i q phi x_nu); U_nu(x) = exp(+i q phi L_nu x_mu) on the last nu slice
    ph_mu = -phi * c[nu]
    ph_nu = np.where(c[nu] == l[nu] - 1, phi * l[nu] * c[mu], 0.0)
    for a in range(3):
        u[..., mu, a, a] = np.exp(1j * q[a] * ph_mu)
        u[..., nu, a, a] = np.exp(1j * q[a] * ph_nu)
    return u, phi, q
