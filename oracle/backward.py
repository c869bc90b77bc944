"""Reverse-mode gradient through stout smearing (oracle; test infrastructure only).

Built only from the chain rule, the brute-force exponential and its Frechet
derivative, so that it is independent of the closed-form stout-force
recursion (Morningstar & Peardon 2004, Sec. IV) that the CUDA path uses.

Convention (as in ``gauge``): G_U = dS/dRe U + i dS/dIm U, dS = Re tr(G^dag dU).
Rules used:  Y = A B   -> G_A += G_Y B^dag,  G_B += A^dag G_Y
             Y = A^dag -> G_A += G_Y^dag
             Y = exp(X) -> G_X = L(X^dag, G_Y)   (L = Frechet derivative of exp)
             Y = TA(M)  -> G_M = TA(G_Y)        (TA is an orthogonal projector)
One stout step per link:  C = rho*S(U), Omega = C U^dag, X = TA(Omega) = iQ,
E = exp(X), U' = E U.
"""
import numpy as np

from .expm import expm_frechet, expm_series
from .gauge import force_from_grad, wilson_action_grad
from .lattice import shift
from .stout import staple_sum, stout_smear_steps
from .su3 import adj, ta


def staple_vjp(U, mu, dirs, K, G):
    """Adds to G the gradient through the bare staple sum S_mu of ``staple_sum``,
    given K = G_S (the gradient w.r.t. S_mu at every site)."""
    Umu = U[..., mu, :, :]
    for nu in dirs:
        if nu == mu:
            continue
        Unu = U[..., nu, :, :]
        # upper staple A = P Qm R^dag, P = U_nu(x), Qm = U_mu(x+nu), R = U_nu(x+mu)
        P = Unu
        Qm = shift(Umu, nu, +1)
        R = shift(Unu, mu, +1)
        G[..., nu, :, :] += K @ R @ adj(Qm)
        G[..., mu, :, :] += shift(adj(P) @ K @ R, nu, -1)
        G[..., nu, :, :] += shift(adj(K) @ P @ Qm, mu, -1)
        # lower staple B = P^dag Qm R, P = U_nu(x-nu), Qm = U_mu(x-nu), R = U_nu(x-nu+mu)
        P = shift(Unu, nu, -1)
        Qm = shift(Umu, nu, -1)
        R = shift(shift(Unu, mu, +1), nu, -1)
        G[..., nu, :, :] += shift(Qm @ R @ adj(K), nu, +1)
        G[..., mu, :, :] += shift(P @ K @ adj(R), nu, +1)
        G[..., nu, :, :] += shift(shift(adj(Qm) @ P @ K, nu, +1), mu, -1)


def stout_step_vjp(U, rho, dirs, Gp):
    """Gradient w.r.t. the step input U, given Gp = gradient w.r.t. the step output."""
    G = Gp.copy()                       # links outside `dirs` pass through unchanged
    for mu in dirs:
        G[..., mu, :, :] = 0.0
    for mu in dirs:
        Umu = U[..., mu, :, :]
        C = rho * staple_sum(U, mu, dirs)
        X = ta(C @ adj(Umu))            # = iQ
        E = expm_series(X)
        Gpm = Gp[..., mu, :, :]
        # U' = E U
        G_E = Gpm @ adj(Umu)
        G[..., mu, :, :] += adj(E) @ Gpm
        # E = exp(X); X = TA(Omega); Omega = C U^dag
        G_Om = ta(expm_frechet(adj(X), G_E))
        G[..., mu, :, :] += adj(G_Om) @ C          # via U^dag in Omega
        staple_vjp(U, mu, dirs, rho * (G_Om @ Umu), G)   # K: gradient w.r.t. the bare staple sum
    return G


def stout_backward(U0, rho, n_steps, dirs, G_out):
    """Gradient w.r.t. the thin links U^(0), given G_out w.r.t. U^(n)."""
    fields = stout_smear_steps(U0, rho, n_steps, dirs)
    G = G_out
    for k in range(n_steps - 1, -1, -1):
        G = stout_step_vjp(fields[k], rho, dirs, G)
    return G


def smeared_wilson_force(U0, rho, n_steps, dirs, beta):
    """su(3) force TA(G U^dag) of S_W(stout^n(U0)) w.r.t. the thin links."""
    fields = stout_smear_steps(U0, rho, n_steps, dirs)
    G = wilson_action_grad(fields[-1], beta)
    for k in range(n_steps - 1, -1, -1):
        G = stout_step_vjp(fields[k], rho, dirs, G)
    return force_from_grad(G, U0), G
