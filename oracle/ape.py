"""APE link smearing in FP64 (oracle; test infrastructure only).

APE smearing (M. Albanese et al., Phys. Lett. B 192 (1987) 163) mixes each
link with its staples and projects the sum back to SU(3):

  V_mu(x) = (1 - alpha) U_mu(x) + alpha / (2 (d - 1)) * sum_{nu in dirs, nu != mu}
              [ U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) ]
  U'_mu(x) = P(V_mu(x))     for mu in dirs; U'_mu = U_mu otherwise,

d = |dirs| (2 (d - 1) staples per link, so a unit field stays the identity).
Every link of a step is computed from the previous step's field.

Reading of the projection P (the method is not unique; the one taken here is
covariant under V -> g V h^dag for g, h in SU(3)): the unitary polar factor
W = V (V^dag V)^(-1/2), then the determinant phase removed with the principal
cube root,  P(V) = W * exp(-i arg(det W) / 3),  arg in (-pi, pi].
(V^dag V)^(-1/2) comes from numpy's Hermitian eigendecomposition.
"""
import numpy as np

from .stout import staple_sum
from .su3 import adj


def project_su3(v):
    """P(V) = W exp(-i arg det W / 3) with W = V (V^dag V)^(-1/2)."""
    a = adj(v) @ v
    lam, q = np.linalg.eigh(a)
    inv_sqrt = (q * (1.0 / np.sqrt(lam))[..., None, :]) @ adj(q)
    w = v @ inv_sqrt
    phase = np.angle(np.linalg.det(w))
    return w * np.exp(-1j * phase / 3.0)[..., None, None]


def ape_step(U, alpha, dirs):
    out = U.copy()
    n_staples = 2 * (len(dirs) - 1)
    coef = alpha / n_staples if n_staples else 0.0     # one direction: no staples
    for mu in dirs:
        v = (1.0 - alpha) * U[..., mu, :, :] + coef * staple_sum(U, mu, dirs)
        out[..., mu, :, :] = project_su3(v)
    return out


def ape_smear(U, alpha, n_steps, dirs):
    for _ in range(n_steps):
        U = ape_step(U, alpha, dirs)
    return U
