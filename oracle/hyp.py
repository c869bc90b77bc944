"""HYP link smearing in FP64 (oracle; test infrastructure only).

Hypercubic blocking (A. Hasenfratz and F. Knechtli, Phys. Rev. D 64 (2001)
034504): three nested APE-type levels whose staples stay inside the
hypercubes attached to the link.  For a 4D lattice, with P the SU(3)
projection of oracle/ape.py and S(A, B)_mu(x) the sum of the forward and
backward staples of direction pair (mu, eta) built from link fields A (the
transverse links) and B (the links along mu):

  S(A, B, mu, eta)(x) = A_eta(x) B_mu(x+eta) A_eta(x+mu)^dag
                      + A_eta(x-eta)^dag B_mu(x-eta) A_eta(x-eta+mu)

  level 3, mu with one remaining direction eta (the decorated link is
  "not smeared in" the other two directions):
    Vb[mu][eta] = P((1 - a3) U_mu + a3/2 * S(U, U, mu, eta))
  level 2, mu not smeared in nu; rho runs over the two directions outside
  {mu, nu} and sigma is the fourth direction:
    Vt[mu][nu]  = P((1 - a2) U_mu + a2/4 * sum_rho S(Vb[.][sigma], Vb[.][sigma], mu, rho))
    (transverse links Vb[rho][sigma], links along mu Vb[mu][sigma])
  level 1:
    V_mu        = P((1 - a1) U_mu + a1/6 * sum_{nu != mu} S(Vt[.][mu], Vt[mu][.], mu, nu))
    (transverse links Vt[nu][mu], links along mu Vt[mu][nu])

All four directions are smeared; every link of a step comes from the
previous step's field.  The usual weights are (a1, a2, a3) = (0.75, 0.6, 0.3).
"""
import numpy as np

from .ape import project_su3
from .lattice import ND, shift
from .su3 import adj


def staples(A_eta, B_mu, mu, eta):
    """Forward + backward staple of (mu, eta) from the eta links A_eta and the mu links B_mu."""
    fwd = A_eta @ shift(B_mu, eta, +1) @ adj(shift(A_eta, mu, +1))
    Am = shift(A_eta, eta, -1)
    bwd = adj(Am) @ shift(B_mu, eta, -1) @ shift(Am, mu, +1)
    return fwd + bwd


def hyp_step(U, a1, a2, a3):
    link = [U[..., mu, :, :] for mu in range(ND)]
    # level 3: Vb[mu][eta], eta != mu
    Vb = {}
    for mu in range(ND):
        for eta in range(ND):
            if eta != mu:
                v = (1 - a3) * link[mu] + (a3 / 2) * staples(link[eta], link[mu], mu, eta)
                Vb[mu, eta] = project_su3(v)
    # level 2: Vt[mu][nu], nu != mu
    Vt = {}
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
            Vt[mu, nu] = project_su3((1 - a2) * link[mu] + (a2 / 4) * acc)
    # level 1
    out = np.empty_like(U)
    for mu in range(ND):
        acc = np.zeros_like(link[mu])
        for nu in range(ND):
            if nu != mu:
                acc = acc + staples(Vt[nu, mu], Vt[mu, nu], mu, nu)
        out[..., mu, :, :] = project_su3((1 - a1) * link[mu] + (a1 / 6) * acc)
    return out


def hyp_smear(U, a1, a2, a3, n_steps):
    for _ in range(n_steps):
        U = hyp_step(U, a1, a2, a3)
    return U
