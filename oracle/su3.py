"""Small complex-matrix helpers on stacks of 3x3 matrices (oracle; test infrastructure only).

``adj`` is the QDP++ ``adj`` of Listing 1 (Sec. 6): the conjugate transpose.
"""
import numpy as np

NC = 3


def adj(a):
    """Conjugate transpose of the last two axes."""
    return np.conj(np.swapaxes(a, -1, -2))


def tr(a):
    """Trace over the last two axes."""
    return np.trace(a, axis1=-2, axis2=-1)


def eye_like(a):
    return np.broadcast_to(np.eye(a.shape[-1], dtype=a.dtype), a.shape).copy()


def ta(m):
    """Traceless anti-Hermitian part: (M - M^dag)/2 - tr(M - M^dag)/(2N) * 1.

    This is the orthogonal projector onto su(N) under <A,B> = Re tr(A^dag B),
    hence self-adjoint under that inner product.
    """
    a = 0.5 * (m - adj(m))
    return a - (tr(a) / m.shape[-1])[..., None, None] * np.eye(m.shape[-1])


def unitarity_violation(u):
    """max |U^dag U - 1| over elements, and max |det U - 1|."""
    d = adj(u) @ u - np.eye(u.shape[-1])
    return float(np.max(np.abs(d))), float(np.max(np.abs(np.linalg.det(u) - 1.0)))
