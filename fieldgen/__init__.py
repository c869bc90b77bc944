"""Seeded synthetic inputs shared by the oracle-side and GPU-side tests and the bench.

This module holds none of the smearing arithmetic.  It draws random numbers
with numpy's PCG64 (``np.random.default_rng(seed)``) in site-lexicographic
order and builds:

* ``haar_su3``          Haar-random SU(3) links: QR of a complex Gaussian
                        matrix with the phase fix of Mezzadri (Notices AMS 54
                        (2007) 592), then division by a cube root of det.
* ``near_identity_su3`` U = exp(i*eps*H), H = (A + A^dag)/2 - tr(.)/3 with A
                        complex Gaussian (re, im ~ N(0,1)); the exponential of
                        the Hermitian matrix is taken through its
                        eigendecomposition (numpy ``eigh``); the large-lattice
                        variant uses ``torch.linalg.matrix_exp`` on the device
                        (same normals, same field up to rounding).
* ``diagonal_phases``   abelian links diag(e^{ia}, e^{ib}, e^{-i(a+b)}).
* ``gauge_field_g``     a Haar SU(3) matrix per site (gauge transformation).
* ``su3_direction``     a random unit-norm traceless anti-Hermitian matrix.
* ``color_vector``      complex Gaussian colour vectors.

Link fields are complex128 arrays of shape (Lt, Lz, Ly, Lx, 4, 3, 3):
C order = site-major, x fastest, then direction, row, column.
"""
import numpy as np


def _shape(dims):
    lx, ly, lz, lt = dims
    return (lt, lz, ly, lx)


def _complex_gauss(rng, shape):
    z = rng.standard_normal(shape + (2,))
    return z[..., 0] + 1j * z[..., 1]


def _haar_from_gauss(z):
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    ph = d / np.abs(d)
    q = q * ph[..., None, :]                 # Q diag(ph): Haar on U(3)
    det = np.linalg.det(q)
    return q / (det ** (1.0 / 3.0))[..., None, None]   # principal cube root


def haar_su3(dims, seed, ndir=4):
    rng = np.random.default_rng(seed)
    return _haar_from_gauss(_complex_gauss(rng, _shape(dims) + (ndir, 3, 3)))


def gauge_field_g(dims, seed):
    rng = np.random.default_rng(seed)
    return _haar_from_gauss(_complex_gauss(rng, _shape(dims) + (3, 3)))


def _traceless_hermitian(a):
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    t = np.trace(h, axis1=-2, axis2=-1) / 3.0
    return h - t[..., None, None] * np.eye(3)


def near_identity_su3(dims, seed, eps=0.3, ndir=4):
    rng = np.random.default_rng(seed)
    h = _traceless_hermitian(_complex_gauss(rng, _shape(dims) + (ndir, 3, 3)))
    lam, v = np.linalg.eigh(h)
    ph = np.exp(1j * eps * lam)
    return (v * ph[..., None, :]) @ np.conj(np.swapaxes(v, -1, -2))


def near_identity_su3_torch(dims, seed, eps=0.3, ndir=4, device="cuda", chunk=1 << 22):
    """Same recipe for large lattices: normals from PCG64 on the host, the
    exponential by torch.linalg.matrix_exp on `device`.  Returns a complex128
    torch tensor shaped (Lt, Lz, Ly, Lx, ndir, 3, 3) on `device`."""
    import torch
    rng = np.random.default_rng(seed)
    shape = _shape(dims) + (ndir,)
    n = int(np.prod(shape))
    out = torch.empty((n, 3, 3), dtype=torch.complex128, device=device)
    done = 0
    while done < n:
        m = min(chunk, n - done)
        h = _traceless_hermitian(_complex_gauss(rng, (m, 3, 3)))
        ht = torch.from_numpy(h).to(device)
        out[done:done + m] = torch.linalg.matrix_exp((1j * eps) * ht)
        done += m
    return out.reshape(shape + (3, 3))


def diagonal_phases(dims, seed, scale=1.0, ndir=4):
    """Abelian links diag(e^{ia}, e^{ib}, e^{-i(a+b)}); returns (links, angles[...,ndir,3])."""
    rng = np.random.default_rng(seed)
    ab = scale * rng.uniform(-np.pi, np.pi, _shape(dims) + (ndir, 2))
    ang = np.concatenate([ab, -ab.sum(-1, keepdims=True)], axis=-1)
    u = np.zeros(ang.shape + (3,), dtype=np.complex128)
    for k in range(3):
        u[..., k, k] = np.exp(1j * ang[..., k])
    return u, ang


def su3_direction(rng):
    """Random traceless anti-Hermitian X with Re tr(X^dag X) = 1."""
    x = 1j * _traceless_hermitian(_complex_gauss(rng, (3, 3)))
    return x / np.sqrt(np.real(np.trace(np.conj(x.T) @ x)))


def color_vector(dims, seed):
    rng = np.random.default_rng(seed)
    return _complex_gauss(rng, _shape(dims) + (3,))


def unit_links(dims, ndir=4):
    return np.broadcast_to(np.eye(3, dtype=np.complex128), _shape(dims) + (ndir, 3, 3)).copy()


def batch_sizes(seed, n_cfg=64, choices=(8, 12, 16, 20, 24)):
    """L for each of n_cfg lattices L^3 x 2L, drawn uniformly from `choices`."""
    rng = np.random.default_rng(seed)
    return [int(choices[i]) for i in rng.integers(0, len(choices), n_cfg)]
