"""Lattice geometry and the periodic nearest-neighbour shift (oracle; test infrastructure only).

The paper's Listing 1 (Sec. 6) writes the hopping term with
``shift(psi, FORWARD, mu)`` and ``shift(., BACKWARD, mu)``; its operator
K (Sec. 6, definition of K_{x,x'}) couples x to x+mu through U_mu(x) and to
x-mu through U_mu(x-mu)^dagger.  Hence ``shift(f, +1, mu)(x) = f(x + mu)``
and ``shift(f, -1, mu)(x) = f(x - mu)``, with periodic wrap in every
direction.  Lattice shapes are L^3 x 2L with t last (Sec. 7, Table 1).
"""
import numpy as np

# Array axis of direction mu in a field shaped (Lt, Lz, Ly, Lx, ...):
# mu = 0 (x) is the fastest site index, mu = 3 (t) the slowest.
AXIS = (3, 2, 1, 0)
ND = 4


def field_shape(dims):
    """dims = (Lx, Ly, Lz, Lt) -> leading array shape (Lt, Lz, Ly, Lx)."""
    lx, ly, lz, lt = dims
    return (lt, lz, ly, lx)


def dims_of(field):
    """Inverse of field_shape for any field whose first four axes are sites."""
    lt, lz, ly, lx = field.shape[:4]
    return (lx, ly, lz, lt)


def volume(dims):
    return int(np.prod(dims))


def site_index(x, y, z, t, dims):
    """Lexicographic site index, x fastest: s = x + Lx*(y + Ly*(z + Lz*t))."""
    lx, ly, lz, _ = dims
    return x + lx * (y + ly * (z + lz * t))


def shift(f, mu, sign):
    """g(x) = f(x + sign * mu_hat), periodic.  sign=+1 is FORWARD, -1 BACKWARD."""
    if sign not in (1, -1):
        raise ValueError("sign must be +1 or -1")
    return np.roll(f, -sign, axis=AXIS[mu])


def translate(f, offset):
    """g(x) = f(x + offset) for an integer 4-vector offset (x, y, z, t)."""
    g = f
    for mu in range(ND):
        if offset[mu]:
            g = np.roll(g, -offset[mu], axis=AXIS[mu])
    return g


def sub_box(f, center, radius):
    """Periodically wrapped box of side 2*radius+1 centred on site `center`.

    The returned array is again a periodic lattice field (of side
    2*radius+1 in every direction).  A quantity that depends only on sites
    within Chebyshev distance r of x, computed on this machine at its centre,
    equals the full-lattice value whenever r <= radius.
    """
    idx = []
    for mu in (3, 2, 1, 0):  # array axes t, z, y, x
        L = f.shape[AXIS[mu]]
        idx.append((np.arange(-radius, radius + 1) + center[mu]) % L)
    return f[np.ix_(*idx)]
