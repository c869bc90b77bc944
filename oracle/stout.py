"""Stout link smearing in FP64 (oracle; test infrastructure only).

Definitions (Morningstar & Peardon, Phys. Rev. D 69 (2004) 054501, Sec. II),
with an isotropic weight rho_{mu nu} = rho for mu, nu in the smeared set
`dirs` and zero otherwise:

  C_mu(x) = rho * sum_{nu in dirs, nu != mu} [ U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
                                             + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) ]
  Omega_mu(x) = C_mu(x) U_mu(x)^dag
  Q_mu(x) = (i/2)(Omega^dag - Omega) - (i/6) tr(Omega^dag - Omega)      (Hermitian, traceless)
  U'_mu(x) = exp(i Q_mu(x)) U_mu(x)     for mu in dirs; U'_mu = U_mu otherwise.

Every link of a step is computed from the previous step's field.

exp(iQ) follows the Cayley-Hamilton construction of the same paper (Sec. III):
exp(iQ) = f0 + f1 Q + f2 Q^2 with

  c0 = det Q = tr(Q^3)/3,   c1 = tr(Q^2)/2,   c0max = 2 (c1/3)^{3/2}
  theta = arccos(|c0| / c0max),   u = sqrt(c1/3) cos(theta/3),   w = sqrt(c1) sin(theta/3)
  xi0(w) = sin(w)/w   (series 1 - w^2/6 (1 - w^2/20 (1 - w^2/42)) for |w| <= 0.05)
  h0 = (u^2 - w^2) e^{2iu} + e^{-iu} [ 8u^2 cos w + 2iu (3u^2 + w^2) xi0 ]
  h1 = 2u e^{2iu} - e^{-iu} [ 2u cos w - i (3u^2 - w^2) xi0 ]
  h2 = e^{2iu} - e^{-iu} [ cos w + 3iu xi0 ]
  f_j = h_j / (9u^2 - w^2);   for c0 < 0:  f_j -> (-1)^j conj(f_j).

Readings where the source is silent: the ratio |c0|/c0max is clamped to
[0, 1]; for c1 below C1_SERIES (where 0/0 would occur, e.g. rho = 0 or a
unit field) the Q -> 0 limits f0 = 1, f1 = i, f2 = -1/2 are used.
"""
import numpy as np

from .lattice import ND, shift
from .su3 import adj, tr

C1_SERIES = 1e-28      # below this c1 the Q -> 0 limit of (f0, f1, f2) is used
XI0_SERIES = 0.05      # |w| at or below this uses the xi0 Taylor series


def dirs_from_mask(mask):
    return tuple(mu for mu in range(ND) if (mask >> mu) & 1)


def staple_sum(U, mu, dirs):
    """sum over nu in dirs, nu != mu, of the upper and lower staples of U_mu (no rho)."""
    Umu = U[..., mu, :, :]
    C = np.zeros_like(Umu)
    for nu in dirs:
        if nu == mu:
            continue
        Unu = U[..., nu, :, :]
        # U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
        C += Unu @ shift(Umu, nu, +1) @ adj(shift(Unu, mu, +1))
        # U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)
        C += adj(shift(Unu, nu, -1)) @ shift(Umu, nu, -1) @ shift(shift(Unu, mu, +1), nu, -1)
    return C


def q_from_omega(Om):
    """Q = (i/2)(Omega^dag - Omega) - (i/6) tr(Omega^dag - Omega) * 1."""
    d = adj(Om) - Om
    return 0.5j * d - (1j / 6.0) * tr(d)[..., None, None] * np.eye(3)


def ch_coefficients(Q):
    """(f0, f1, f2) with exp(iQ) = f0 + f1 Q + f2 Q^2 for Hermitian traceless Q."""
    Q2 = Q @ Q
    c0 = np.real(tr(Q2 @ Q)) / 3.0
    c1 = np.real(tr(Q2)) / 2.0
    small = c1 < C1_SERIES
    neg = c0 < 0
    c1s = np.where(small, 1.0, c1)               # keeps the masked lanes finite
    c0max = 2.0 * (c1s / 3.0) ** 1.5
    theta = np.arccos(np.clip(np.abs(c0) / c0max, 0.0, 1.0))
    u = np.sqrt(c1s / 3.0) * np.cos(theta / 3.0)
    w = np.sqrt(c1s) * np.sin(theta / 3.0)
    w2 = w * w
    u2 = u * u
    xi0 = np.where(np.abs(w) <= XI0_SERIES,
                   1.0 - w2 / 6.0 * (1.0 - w2 / 20.0 * (1.0 - w2 / 42.0)),
                   np.sin(w) / np.where(w == 0, 1.0, w))
    e2iu = np.exp(2j * u)
    emiu = np.exp(-1j * u)
    cw = np.cos(w)
    h0 = (u2 - w2) * e2iu + emiu * (8.0 * u2 * cw + 2j * u * (3.0 * u2 + w2) * xi0)
    h1 = 2.0 * u * e2iu - emiu * (2.0 * u * cw - 1j * (3.0 * u2 - w2) * xi0)
    h2 = e2iu - emiu * (cw + 3j * u * xi0)
    den = 9.0 * u2 - w2
    f = [h0 / den, h1 / den, h2 / den]
    f = [np.where(neg, ((-1) ** j) * np.conj(fj), fj) for j, fj in enumerate(f)]
    limits = (1.0 + 0j, 1j, -0.5 + 0j)
    f = [np.where(small, lim, fj) for fj, lim in zip(f, limits)]
    return f[0], f[1], f[2]


def expiq_ch(Q):
    """exp(iQ) = f0 + f1 Q + f2 Q^2 (Cayley-Hamilton form)."""
    f0, f1, f2 = ch_coefficients(Q)
    eye = np.eye(3)
    return f0[..., None, None] * eye + f1[..., None, None] * Q + f2[..., None, None] * (Q @ Q)


def stout_q(U, mu, rho, dirs):
    """(C, Omega, Q) of link direction mu."""
    C = rho * staple_sum(U, mu, dirs)
    Om = C @ adj(U[..., mu, :, :])
    return C, Om, q_from_omega(Om)


def stout_step(U, rho, dirs):
    """One stout step; all new links are computed from the input field U."""
    out = U.copy()
    for mu in dirs:
        _, _, Q = stout_q(U, mu, rho, dirs)
        out[..., mu, :, :] = expiq_ch(Q) @ U[..., mu, :, :]
    return out


def stout_smear(U, rho, n_steps, dirs):
    for _ in range(n_steps):
        U = stout_step(U, rho, dirs)
    return U


def stout_smear_steps(U, rho, n_steps, dirs):
    """[U^(0), ..., U^(n)]: every step's field (used by the backward pass)."""
    out = [U]
    for _ in range(n_steps):
        out.append(stout_step(out[-1], rho, dirs))
    return out
