"""Reverse-mode gradient through HYP smearing (oracle; test infrastructure only).

Convention and chain rules as in ``backward``; the forward definitions are
those of ``hyp`` (levels 3, 2, 1 with weights a3, a2, a1, each level's sum
projected by P of ``ape``).  The gradient runs the levels backwards:

  level 1  G_V1[mu] = P'(V1[mu])^* G_out[mu];  G_U[mu] += (1 - a1) G_V1[mu];
           through S(Vt[nu][mu], Vt[mu][nu], mu, nu) with K = a1/6 G_V1[mu]
           into G_Vt[nu][mu] (transverse) and G_Vt[mu][nu] (along mu)
  level 2  G_V2[mu][nu] from G_Vt[mu][nu];  G_U[mu] += (1 - a2) G_V2;
           through S(Vb[rho][sigma], Vb[mu][sigma], mu, rho), K = a2/4 G_V2,
           into G_Vb[rho][sigma] and G_Vb[mu][sigma]
  level 3  G_V3[mu][eta] from G_Vb[mu][eta];  G_U[mu] += (1 - a3) G_V3;
           through S(U_eta, U_mu, mu, eta), K = a3/2 G_V3, into G_U[eta] and G_U[mu]

with P'^* the projection's gradient (``ape_force.project_su3_vjp``) and the
staple's gradient written out below for two link fields A (transverse) and
B (along mu).
"""
import numpy as np

from .ape_force import project_su3_vjp
from .gauge import force_from_grad, wilson_action_grad
from .hyp import hyp_step, staples
from .lattice import ND, shift
from .ape import project_su3
from .su3 import adj


def staples_vjp(A_eta, B_mu, mu, eta, K):
    """(G_A, G_B) of Re tr(K^dag S) for S = staples(A_eta, B_mu, mu, eta):
    S(x) = A(x) B(x+eta) A(x+mu)^dag + A(x-eta)^dag B(x-eta) A(x-eta+mu)."""
    # upper staple: P = A(x), Q = B(x+eta), R = A(x+mu); Y = P Q R^dag
    Q = shift(B_mu, eta, +1)
    R = shift(A_eta, mu, +1)
    g_a = K @ R @ adj(Q)
    g_b = shift(adj(A_eta) @ K @ R, eta, -1)
    g_a = g_a + shift(adj(K) @ A_eta @ Q, mu, -1)
    # lower staple: P = A(x-eta), Q = B(x-eta), R = A(x-eta+mu); Y = P^dag Q R
    P = shift(A_eta, eta, -1)
    Q = shift(B_mu, eta, -1)
    R = shift(shift(A_eta, mu, +1), eta, -1)
    g_a = g_a + shift(Q @ R @ adj(K), eta, +1)
    g_b = g_b + shift(P @ K @ adj(R), eta, +1)
    g_a = g_a + shift(shift(adj(Q) @ P @ K, eta, +1), mu, -1)
    return g_a, g_b


def _decorated(U, a2, a3):
    """Vb, Vt and the sums V2 of the forward step (V3 and V1 are formed in the gradient)."""
    link = [U[..., mu, :, :] for mu in range(ND)]
    Vb = {}
    for mu in range(ND):
        for eta in range(ND):
            if eta != mu:
                Vb[mu, eta] = project_su3((1 - a3) * link[mu] + (a3 / 2) * staples(link[eta], link[mu], mu, eta))
    Vt, V2 = {}, {}
    for mu in range(ND):
        for nu in range(ND):
            if nu == mu:
                continue
            acc = np.zeros_like(link[mu])
            for rho in range(ND):
                if rho in (mu, nu):
                    continue
                sigma = ({0, 1, 2, 3} - {mu, nu, rho}).pop()
                acc = acc + staples(Vb[rho, sigma], Vb[mu, sigma], mu, rho)
            V2[mu, nu] = (1 - a2) * link[mu] + (a2 / 4) * acc
            Vt[mu, nu] = project_su3(V2[mu, nu])
    return link, Vb, Vt, V2


def hyp_step_vjp(U, a1, a2, a3, Gp):
    """Gradient w.r.t. the step input U, given Gp = gradient w.r.t. the step output."""
    link, Vb, Vt, V2 = _decorated(U, a2, a3)
    G = np.zeros_like(U)
    # level 1
    G_Vt = {k: np.zeros_like(link[0]) for k in Vt}
    for mu in range(ND):
        acc = np.zeros_like(link[mu])
        for nu in range(ND):
            if nu != mu:
                acc = acc + staples(Vt[nu, mu], Vt[mu, nu], mu, nu)
        g_v = project_su3_vjp((1 - a1) * link[mu] + (a1 / 6) * acc, Gp[..., mu, :, :])
        G[..., mu, :, :] += (1 - a1) * g_v
        for nu in range(ND):
            if nu != mu:
                ga, gb = staples_vjp(Vt[nu, mu], Vt[mu, nu], mu, nu, (a1 / 6) * g_v)
                G_Vt[nu, mu] += ga
                G_Vt[mu, nu] += gb
    # level 2
    G_Vb = {k: np.zeros_like(link[0]) for k in Vb}
    for (mu, nu), v in V2.items():
        g_v = project_su3_vjp(v, G_Vt[mu, nu])
        G[..., mu, :, :] += (1 - a2) * g_v
        for rho in range(ND):
            if rho in (mu, nu):
                continue
            sigma = ({0, 1, 2, 3} - {mu, nu, rho}).pop()
            ga, gb = staples_vjp(Vb[rho, sigma], Vb[mu, sigma], mu, rho, (a2 / 4) * g_v)
            G_Vb[rho, sigma] += ga
            G_Vb[mu, sigma] += gb
    # level 3
    for (mu, eta), g_vb in G_Vb.items():
        v = (1 - a3) * link[mu] + (a3 / 2) * staples(link[eta], link[mu], mu, eta)
        g_v = project_su3_vjp(v, g_vb)
        G[..., mu, :, :] += (1 - a3) * g_v
        ga, gb = staples_vjp(link[eta], link[mu], mu, eta, (a3 / 2) * g_v)
        G[..., eta, :, :] += ga
        G[..., mu, :, :] += gb
    return G


def hyp_smear_steps(U0, a1, a2, a3, n_steps):
    """[U^(0), ..., U^(n)]."""
    fields = [U0]
    for _ in range(n_steps):
        fields.append(hyp_step(fields[-1], a1, a2, a3))
    return fields


def hyp_backward(U0, a1, a2, a3, n_steps, G_out):
    """Gradient w.r.t. the thin links U^(0), given G_out w.r.t. U^(n)."""
    fields = hyp_smear_steps(U0, a1, a2, a3, n_steps)
    G = G_out
    for k in range(n_steps - 1, -1, -1):
        G = hyp_step_vjp(fields[k], a1, a2, a3, G)
    return G


def smeared_wilson_force(U0, a1, a2, a3, n_steps, beta):
    """su(3) force TA(G U^dag) of S_W(hyp^n(U0)) w.r.t. the thin links, and G."""
    fields = hyp_smear_steps(U0, a1, a2, a3, n_steps)
    G = wilson_action_grad(fields[-1], beta)
    for k in range(n_steps - 1, -1, -1):
        G = hyp_step_vjp(fields[k], a1, a2, a3, G)
    return force_from_grad(G, U0), G
