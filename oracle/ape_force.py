"""Reverse-mode gradient through APE smearing (oracle; test infrastructure only).

Convention and chain rules as in ``backward``: G_U = dS/dRe U + i dS/dIm U,
dS = Re tr(G^dag dU).  One APE step per smeared link (``ape``):

  V = (1 - alpha) U + c S(U),   S the bare staple sum, c = alpha / (2 (d - 1)),
  U' = P(V) = W z,   W = V X,   X = f(A) = A^(-1/2),   A = V^dag V,
  z = exp(-i phi / 3),   phi = arg det W.

The gradient of P is written from these pieces, each by its own rule:
  U' = W z, with d(phi) = Im tr(W^-1 dW) (Jacobi's formula for the determinant):
      G_W = conj(z) G_P + Im(tr(G_P^dag U')) / 3 * i W^(-dag)
  W = V X:       G_V += G_W X^dag,   G_X = V^dag G_W
  X = f(A):      G_A = L(A, G_X), L the Frechet derivative of f at A.  For
                 Hermitian A = Q diag(lambda) Q^dag the Daleckii-Krein formula
                 gives L(A, E) = Q (Gamma o (Q^dag E Q)) Q^dag with Gamma_ij the
                 divided difference f[lambda_i, lambda_j] (f'(lambda_i) for
                 i = j); N. J. Higham, Functions of Matrices, SIAM 2008,
                 Thm 3.11.  Gamma is real symmetric, so L(A, .) is self-adjoint
                 under Re tr(A^dag B) and serves as its own adjoint.
  A = V^dag V:   G_V += V (G_A + G_A^dag)
and the staple sum as in the stout gradient (``backward.staple_vjp``).
"""
import numpy as np

from .ape import ape_step, project_su3
from .backward import staple_vjp
from .gauge import force_from_grad, wilson_action_grad
from .stout import staple_sum
from .su3 import adj


def inv_sqrt_divided_difference(lam_i, lam_j):
    """f[l_i, l_j] for f(x) = x^(-1/2): -1 / (s_i s_j (s_i + s_j)), s = sqrt(l).

    (1/s_j - 1/s_i) / (s_j^2 - s_i^2) = (s_i - s_j) / (s_i s_j (s_j - s_i)(s_j + s_i));
    at l_i = l_j the same expression is f'(l) = -1/(2 l^(3/2))."""
    si, sj = np.sqrt(lam_i), np.sqrt(lam_j)
    return -1.0 / (si * sj * (si + sj))


def project_su3_vjp(v, g_p):
    """G_V of a scalar through U' = P(V), given G_P = its gradient w.r.t. U'."""
    a = adj(v) @ v
    lam, q = np.linalg.eigh(a)
    x = (q * (1.0 / np.sqrt(lam))[..., None, :]) @ adj(q)
    w = v @ x
    z = np.exp(-1j * np.angle(np.linalg.det(w)) / 3.0)[..., None, None]
    p = w * z
    # U' = W z
    kappa_im = np.imag(np.trace(adj(g_p) @ p, axis1=-2, axis2=-1))[..., None, None]
    g_w = np.conj(z) * g_p + (kappa_im / 3.0) * 1j * adj(np.linalg.inv(w))
    # W = V X
    g_v = g_w @ adj(x)
    g_x = adj(v) @ g_w
    # X = f(A), Daleckii-Krein
    gamma = inv_sqrt_divided_difference(lam[..., :, None], lam[..., None, :])
    g_a = q @ (gamma * (adj(q) @ g_x @ q)) @ adj(q)
    # A = V^dag V
    g_v = g_v + v @ (g_a + adj(g_a))
    return g_v


def ape_step_vjp(U, alpha, dirs, Gp):
    """Gradient w.r.t. the step input U, given Gp = gradient w.r.t. the step output."""
    G = Gp.copy()                       # links outside `dirs` pass through unchanged
    for mu in dirs:
        G[..., mu, :, :] = 0.0
    n_staples = 2 * (len(dirs) - 1)
    coef = alpha / n_staples if n_staples else 0.0
    for mu in dirs:
        v = (1.0 - alpha) * U[..., mu, :, :] + coef * staple_sum(U, mu, dirs)
        g_v = project_su3_vjp(v, Gp[..., mu, :, :])
        G[..., mu, :, :] += (1.0 - alpha) * g_v
        if coef != 0.0:
            staple_vjp(U, mu, dirs, coef * g_v, G)
    return G


def ape_smear_steps(U0, alpha, n_steps, dirs):
    """[U^(0), ..., U^(n)]."""
    fields = [U0]
    for _ in range(n_steps):
        fields.append(ape_step(fields[-1], alpha, dirs))
    return fields


def ape_backward(U0, alpha, n_steps, dirs, G_out):
    """Gradient w.r.t. the thin links U^(0), given G_out w.r.t. U^(n)."""
    fields = ape_smear_steps(U0, alpha, n_steps, dirs)
    G = G_out
    for k in range(n_steps - 1, -1, -1):
        G = ape_step_vjp(fields[k], alpha, dirs, G)
    return G


def smeared_wilson_force(U0, alpha, n_steps, dirs, beta):
    """su(3) force TA(G U^dag) of S_W(ape^n(U0)) w.r.t. the thin links, and G."""
    fields = ape_smear_steps(U0, alpha, n_steps, dirs)
    G = wilson_action_grad(fields[-1], beta)
    for k in range(n_steps - 1, -1, -1):
        G = ape_step_vjp(fields[k], alpha, dirs, G)
    return force_from_grad(G, U0), G


__all__ = ["inv_sqrt_divided_difference", "project_su3_vjp", "ape_step_vjp", "ape_smear_steps",
           "ape_backward", "smeared_wilson_force", "project_su3"]
