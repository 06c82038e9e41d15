"""Seeded synthetic inputs for the Wilson-clover operator and its solvers.

This module is shared by the FP64 CPU oracle (``oracle/``), the tests and the
benchmark.  It draws random numbers and nothing else: it holds none of the
operator's or the solvers' arithmetic.  Everything is FP64 / complex128 numpy
in the canonical layouts

  gauge  U[t][z][y][x][mu][a][b]      mu = 0..3 for x, y, z, t
  spinor psi[t][z][y][x][spin][colour]

i.e. arrays of shape ``(Lt, Lz, Ly, Lx, 4, 3, 3)`` and ``(Lt, Lz, Ly, Lx, 4, 3)``.
Lattice extents are given as ``dims = (Lx, Ly, Lz, Lt)``.

Generators (the random-number stream is numpy ``Generator(PCG64(seed))``; the
draw order is t, z, y, x with x fastest, then mu, then matrix entries row-major,
real part before imaginary part):

* ``haar_gauge``: Haar-random SU(3) links (complex Gaussian 3x3, Gram-Schmidt
  on the rows, then division by the principal cube root of the determinant).
* ``smooth_gauge``: ``U = exp(i eps H)`` with ``H = sum_a h_a lambda_a / 2``
  (Gell-Mann matrices, ``h_a ~ N(0, 1)``), exponentiated by scaling and
  squaring of the Taylor series (Moler & Van Loan, "Nineteen dubious ways",
  method 3), then re-unitarised.
* ``gaussian_spinor``: complex Gaussian with unit variance (1/2 per real part).
* ``point_source``: delta at one site, spin and colour.
* ``random_gauge_transform``: Haar SU(3) per site, for covariance tests.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "haar_su3", "smooth_su3", "haar_gauge", "smooth_gauge", "unit_gauge",
    "gaussian_spinor", "point_source", "random_gauge_transform",
    "gauge_field", "lattice_shape",
]


def lattice_shape(dims):
    """Canonical site shape (Lt, Lz, Ly, Lx) for dims = (Lx, Ly, Lz, Lt)."""
    lx, ly, lz, lt = (int(d) for d in dims)
    return (lt, lz, ly, lx)


def _complex_normal(rng, shape):
    """Complex Gaussian with variance 1/2 per real component (E|z|^2 = 1)."""
    z = rng.standard_normal(tuple(shape) + (2,)) * np.sqrt(0.5)
    return z[..., 0] + 1j * z[..., 1]


def _project_su3(g):
    """Gram-Schmidt on the rows of each 3x3 matrix, then fix det to +1."""
    g = np.array(g, dtype=np.complex128, copy=True)
    r0 = g[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = g[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = g[..., 2, :]
    r2 = r2 - np.sum(np.conj(r0) * r2, axis=-1, keepdims=True) * r0
    r2 = r2 - np.sum(np.conj(r1) * r2, axis=-1, keepdims=True) * r1
    r2 = r2 / np.linalg.norm(r2, axis=-1, keepdims=True)
    u = np.stack([r0, r1, r2], axis=-2)
    det = np.linalg.det(u)
    # principal cube root of the (unit-modulus) determinant
    root = np.exp(1j * np.angle(det) / 3.0)
    return u / root[..., None, None]


def haar_su3(rng, shape):
    """Haar-random SU(3) matrices of the given leading shape."""
    # a second Gram-Schmidt pass removes the rounding of the first one
    return _project_su3(_project_su3(_complex_normal(rng, tuple(shape) + (3, 3))))


# Gell-Mann matrices lambda_1..lambda_8 (standard normalisation tr l_a l_b = 2 d_ab)
_GELL_MANN = np.zeros((8, 3, 3), dtype=np.complex128)
_GELL_MANN[0][0, 1] = _GELL_MANN[0][1, 0] = 1
_GELL_MANN[1][0, 1] = -1j
_GELL_MANN[1][1, 0] = 1j
_GELL_MANN[2][0, 0] = 1
_GELL_MANN[2][1, 1] = -1
_GELL_MANN[3][0, 2] = _GELL_MANN[3][2, 0] = 1
_GELL_MANN[4][0, 2] = -1j
_GELL_MANN[4][2, 0] = 1j
_GELL_MANN[5][1, 2] = _GELL_MANN[5][2, 1] = 1
_GELL_MANN[6][1, 2] = -1j
_GELL_MANN[6][2, 1] = 1j
_GELL_MANN[7][0, 0] = _GELL_MANN[7][1, 1] = 1 / np.sqrt(3)
_GELL_MANN[7][2, 2] = -2 / np.sqrt(3)


def _expm_taylor(a):
    """exp(a) for a batch of 3x3 matrices by scaling and squaring of Taylor."""
    nrm = np.max(np.sum(np.abs(a), axis=-1), axis=-1)
    s = int(max(0, np.ceil(np.log2(max(float(nrm.max(initial=0.0)), 1e-300) / 0.25))))
    b = a / (2.0 ** s)
    # Horner form of sum_{k<=12} b^k / k!  (|b| <= 1/4: remainder < 1e-17)
    eye = np.broadcast_to(np.eye(3, dtype=np.complex128), b.shape)
    out = eye + b / 12.0
    for k in range(11, 0, -1):
        out = eye + np.matmul(b, out) / k
    for _ in range(s):
        out = np.matmul(out, out)
    return out


def smooth_su3(rng, shape, eps):
    """SU(3) matrices exp(i eps H), H = sum_a h_a lambda_a / 2, h_a ~ N(0,1)."""
    h = rng.standard_normal(tuple(shape) + (8,))
    H = np.einsum("...a,aij->...ij", h, _GELL_MANN) * 0.5
    return _project_su3(_expm_taylor(1j * eps * H))


def _gauge_by_slices(dims, make):
    lt, lz, ly, lx = lattice_shape(dims)
    out = np.empty((lt, lz, ly, lx, 4, 3, 3), dtype=np.complex128)
    for t in range(lt):  # t slowest: same stream as one big draw
        out[t] = make((lz, ly, lx, 4))
    return out


def haar_gauge(dims, seed):
    """Haar-random gauge field, canonical layout."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return _gauge_by_slices(dims, lambda shp: haar_su3(rng, shp))


def smooth_gauge(dims, eps, seed):
    """Gauge field of links exp(i eps H), canonical layout."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return _gauge_by_slices(dims, lambda shp: smooth_su3(rng, shp, eps))


def unit_gauge(dims):
    """Free field: every link is the 3x3 identity."""
    lt, lz, ly, lx = lattice_shape(dims)
    u = np.zeros((lt, lz, ly, lx, 4, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def constant_abelian_gauge(dims, mu, nu, k):
    """U_nu(x) = exp(i theta x_mu T) with T = diag(1, -1, 0) and theta =
    2 pi k / L_mu; every other link is 1 (a constant abelian field strength
    in the mu-nu plane)."""
    lt, lz, ly, lx = lattice_shape(dims)
    u = unit_gauge(dims)
    theta = 2.0 * np.pi * k / dims[mu]
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    ph = np.exp(1j * theta * [x, y, z, t][mu])
    u[..., nu, 0, 0] = ph
    u[..., nu, 1, 1] = ph.conj()
    return u


def gauge_field(dims, kind, seed, eps=None):
    """``kind`` is 'haar', 'smooth' (needs eps) or 'unit'."""
    if kind == "haar":
        return haar_gauge(dims, seed)
    if kind == "smooth":
        return smooth_gauge(dims, eps, seed)
    if kind == "unit":
        return unit_gauge(dims)
    raise ValueError(kind)


def gaussian_spinor(dims, seed, nfields=None):
    """Complex Gaussian spinor field(s), canonical layout."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shp = lattice_shape(dims) + (4, 3)
    if nfields is not None:
        shp = (int(nfields),) + shp
    return _complex_normal(rng, shp)


def point_source(dims, spin, colour, site=(0, 0, 0, 0)):
    """Delta source at site (x, y, z, t), given spin and colour."""
    lt, lz, ly, lx = lattice_shape(dims)
    b = np.zeros((lt, lz, ly, lx, 4, 3), dtype=np.complex128)
    x, y, z, t = site
    b[t, z, y, x, spin, colour] = 1.0
    return b


def random_gauge_transform(dims, seed):
    """Haar SU(3) matrix g(x) per site, shape (Lt, Lz, Ly, Lx, 3, 3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return haar_su3(rng, lattice_shape(dims))
