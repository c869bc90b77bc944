"""Plaquette, Wilson action, its gradient, and gauge transformations (oracle; test infrastructure only).

P_{mu nu}(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag.
Average plaquette = (1/(18 V)) sum_x sum_{mu<nu} Re tr P_{mu nu}(x)   (unit field -> 1);
spatial = planes with nu < 3, normalised by 1/(9V); temporal = planes with nu = 3.
Wilson action S = beta * sum_x sum_{mu<nu} (1 - Re tr P_{mu nu}(x) / 3).

Gradient convention used by every gradient in this package: for a real S of a
complex matrix U, G_U = dS/dRe U + i dS/dIm U, so that dS = Re tr(G_U^dag dU).
"""
import numpy as np

from .lattice import ND, shift
from .su3 import adj, tr

PLANES = [(mu, nu) for mu in range(ND) for nu in range(mu + 1, ND)]


def plaquette_field(U, mu, nu):
    """Re tr P_{mu nu}(x) at every site."""
    Umu = U[..., mu, :, :]
    Unu = U[..., nu, :, :]
    P = Umu @ shift(Unu, mu, +1) @ adj(shift(Umu, nu, +1)) @ adj(Unu)
    return np.real(tr(P))


def plaquette(U):
    """(average, spatial, temporal) plaquette."""
    V = int(np.prod(U.shape[:4]))
    s = {pl: float(np.sum(plaquette_field(U, *pl))) for pl in PLANES}
    spatial = sum(v for (mu, nu), v in s.items() if nu < 3)
    temporal = sum(v for (mu, nu), v in s.items() if nu == 3)
    return (spatial + temporal) / (18.0 * V), spatial / (9.0 * V), temporal / (9.0 * V)


def local_action(U, beta):
    """s(x) = beta * sum_{mu<nu} (1 - Re tr P_{mu nu}(x)/3); S = sum_x s(x)."""
    return beta * sum(1.0 - plaquette_field(U, mu, nu) / 3.0 for mu, nu in PLANES)


def wilson_action(U, beta):
    return float(np.sum(local_action(U, beta)))


def wilson_action_grad(U, beta):
    """G_U of the Wilson action by the chain rule through each plaquette product.

    For Y = A B: G_A += G_Y B^dag, G_B += A^dag G_Y; for Y = A^dag: G_A += G_Y^dag.
    Re tr P has G_P = 1, so every plaquette contributes with weight -beta/3.
    """
    G = np.zeros_like(U)
    eye = np.eye(3, dtype=np.complex128)
    for mu, nu in PLANES:
        A = U[..., mu, :, :]                 # U_mu(x)
        B = shift(U[..., nu, :, :], mu, +1)  # U_nu(x+mu)
        Cm = shift(U[..., mu, :, :], nu, +1)  # U_mu(x+nu)   (enters as Cm^dag)
        D = U[..., nu, :, :]                 # U_nu(x)      (enters as D^dag)
        GP = -(beta / 3.0) * np.broadcast_to(eye, A.shape)
        # P = A B Cm^dag D^dag
        gA = GP @ adj(B @ adj(Cm) @ adj(D))
        gB = adj(A) @ GP @ adj(adj(Cm) @ adj(D))
        gCd = adj(A @ B) @ GP @ D            # gradient w.r.t. Cm^dag
        gDd = adj(A @ B @ adj(Cm)) @ GP      # gradient w.r.t. D^dag
        G[..., mu, :, :] += gA
        G[..., nu, :, :] += shift(gB, mu, -1)        # B lives at x+mu
        G[..., mu, :, :] += shift(adj(gCd), nu, -1)  # Cm lives at x+nu
        G[..., nu, :, :] += adj(gDd)
    return G


def force_from_grad(G, U):
    """su(3) force F_mu(x) = TA(G_{U_mu(x)} U_mu(x)^dag).

    It satisfies d/de S(exp(e X) U_mu(x))|_0 = Re tr(F^dag X) for every
    traceless anti-Hermitian X.
    """
    from .su3 import ta
    return ta(G @ adj(U))


def gauge_transform(U, g):
    """U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dag for a site field g of SU(3) matrices."""
    out = np.empty_like(U)
    for mu in range(ND):
        out[..., mu, :, :] = g @ U[..., mu, :, :] @ adj(shift(g, mu, +1))
    return out
