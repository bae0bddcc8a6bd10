"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This module holds input generation only, none of the method's arithmetic: random gauge
links, random spinors and point sources.  Every array is produced on the host with
numpy's ``Generator(PCG64(seed))`` so both sides of a parity test receive the same bits.

Canonical layouts (complex128, C order; viewed as interleaved re/im float64 at the C-ABI):
  lattice extents ``dims = (T, L1, L2, L3)``, site x = (x0, x1, x2, x3), mu = 0 is time,
  lex(x) = x3 + L3*(x2 + L2*(x1 + L1*x0))   (x3 fastest);
  gauge field   ``U[mu, lex, row, col]``  shape (4, V, 3, 3);
  spinor field  ``psi[lex, spin, colour]`` shape (V, 4, 3).
Links are drawn mu-major, then site, as the array order says.
"""
import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def volume(dims):
    return int(np.prod(dims))


def complex_gaussian(r, shape):
    """Complex Gaussian entries with independent re, im ~ N(0, 1/2) (unit mean modulus squared)."""
    s = np.sqrt(0.5)
    return r.normal(0.0, s, size=shape) + 1j * r.normal(0.0, s, size=shape)


def haar_su3(n, seed):
    """n Haar-random SU(3) matrices: QR of a complex-Gaussian 3x3, column phases of Q fixed by
    the diagonal of R, then the determinant phase removed with the principal cube root."""
    r = rng(seed)
    z = complex_gaussian(r, (n, 3, 3))
    q, rr = np.linalg.qr(z)
    d = np.diagonal(rr, axis1=1, axis2=2)
    ph = d / np.abs(d)
    u = q * ph[:, None, :]
    det = np.linalg.det(u)
    u = u * (det ** (-1.0 / 3.0))[:, None, None]
    return u


def gellmann():
    """The eight Gell-Mann matrices lambda^1..lambda^8 as an (8, 3, 3) array (index a-1)."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0, 0, 1] = l[0, 1, 0] = 1
    l[1, 0, 1], l[1, 1, 0] = -1j, 1j
    l[2, 0, 0], l[2, 1, 1] = 1, -1
    l[3, 0, 2] = l[3, 2, 0] = 1
    l[4, 0, 2], l[4, 2, 0] = -1j, 1j
    l[5, 1, 2] = l[5, 2, 1] = 1
    l[6, 1, 2], l[6, 2, 1] = -1j, 1j
    l[7] = np.diag([1, 1, -2]) / np.sqrt(3.0)
    return l


def near_identity_su3(n, eps, seed):
    """n SU(3) matrices exp(i eps H) with H = sum_a h_a lambda^a / 2, h_a ~ N(0, 1); the
    exponential is taken through the eigendecomposition of the Hermitian H."""
    r = rng(seed)
    h = r.normal(0.0, 1.0, size=(n, 8))
    H = np.einsum("na,aij->nij", h, gellmann()) / 2.0
    w, v = np.linalg.eigh(H)
    return np.einsum("nij,nj,nkj->nik", v, np.exp(1j * eps * w), v.conj())


def gauge_field(dims, kind="haar", seed=0, eps=0.3):
    """Canonical gauge field U[mu, lex, 3, 3] for the lattice ``dims``.

    kind: "haar" (Haar-random SU(3)), "near_identity" (exp(i eps H)), "unit" (free field).
    """
    V = volume(dims)
    if kind == "haar":
        u = haar_su3(4 * V, seed)
    elif kind == "near_identity":
        u = near_identity_su3(4 * V, eps, seed)
    elif kind == "unit":
        u = np.broadcast_to(np.eye(3, dtype=np.complex128), (4 * V, 3, 3)).copy()
    else:
        raise ValueError(kind)
    return np.ascontiguousarray(u.reshape(4, V, 3, 3))


def spinor(dims, seed=1, nrhs=None):
    """Complex-Gaussian spinor field psi[lex, 4, 3] (or [nrhs, lex, 4, 3])."""
    V = volume(dims)
    shape = (V, 4, 3) if nrhs is None else (nrhs, V, 4, 3)
    return np.ascontiguousarray(complex_gaussian(rng(seed), shape))


def point_source(dims, spin, colour, site=0):
    """delta_{x,site} delta_{alpha,spin} delta_{a,colour}."""
    psi = np.zeros((volume(dims), 4, 3), dtype=np.complex128)
    psi[site, spin, colour] = 1.0
    return psi


def gauge_transform(dims, seed):
    """A random site-dependent SU(3) gauge transformation g[lex, 3, 3] (Haar)."""
    return haar_su3(volume(dims), seed).reshape(volume(dims), 3, 3)


def su3_directions(dims, seed):
    """Random su(3) directions: real coefficients omega[mu, lex, a] for T^a = lambda^a / 2."""
    return rng(seed).normal(0.0, 1.0, size=(4, volume(dims), 8))
