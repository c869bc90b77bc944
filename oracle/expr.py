"""Reference semantics of fused per-site expressions and of Jacobi smearing
(oracle; test infrastructure only).

An expression program is a list of ops over a small register file of per-site
3x3 complex matrices, evaluated here with whole-lattice numpy operations (the
paper evaluates one expression per kernel over all sites, Sec. 4; its
operations are shift, adj, products, sums and scalar multiples, Listing 1).
Op tuples (register indices r*, operand index k):

  ("load",  rd, k, mu, sign)  rd = shift(operand[k], sign, mu)   (sign 0: no shift)
  ("loadl", rd, k, dir, mu, sign)  rd = shift(links[k][dir], sign, mu)
  ("adj",   rd, ra)           rd = ra^dag
  ("mul",   rd, ra, rb)       rd = ra @ rb
  ("add",   rd, ra, rb)       rd = ra + rb
  ("sub",   rd, ra, rb)       rd = ra - rb
  ("scale", rd, ra, re, im)   rd = (re + i im) * ra
  ("shift", rd, ra, mu, sign) rd = shift(ra, sign, mu)   (shift of a computed value)
  ("trace", rd, ra)           rd = tr(ra) * 1  (complex trace on the diagonal)
  ("retr",  rd, ra)           rd = Re tr(ra) * 1
  ("store", ra)               result = ra
The optional reduction returns sum_x tr(result(x)) as a complex number.

Registers hold 3x3 matrices: an operand that is a colour vector (trailing
shape (3,)) is loaded into column 0 with the other columns zero, a complex or
real scalar field (no trailing axes) as scalar * identity; ``as_vector`` and
``as_scalar`` read a result back the way a vector / scalar output stores it
(column 0, entry (0,0)).  This is the register machine of the expression
programs (the flattened expressions of Sec. 4.2).
"""
import numpy as np

from .lattice import ND, shift
from .su3 import adj, tr


def as_matrix(f):
    """Promote a site field to 3x3 matrices (vector -> column 0, scalar -> s * 1)."""
    f = np.asarray(f)
    if f.ndim == 4:                                   # scalar per site
        return f[..., None, None] * np.eye(3)
    if f.shape[-1] == 3 and (f.ndim == 5 or f.shape[-2] != 3):
        m = np.zeros(f.shape + (3,), dtype=np.complex128)
        m[..., :, 0] = f
        return m
    return f


def as_vector(m):
    return m[..., :, 0]


def as_scalar(m):
    return m[..., 0, 0]


def eval_program(prog, operands, nreg=8):
    regs = [None] * nreg
    result = None
    for op in prog:
        kind = op[0]
        if kind == "load":
            _, rd, k, mu, sign = op
            f = as_matrix(operands[k])
            regs[rd] = f if sign == 0 else shift(f, mu, sign)
        elif kind == "loadl":
            _, rd, k, d, mu, sign = op
            f = operands[k][..., d, :, :]
            regs[rd] = f if sign == 0 else shift(f, mu, sign)
        elif kind == "adj":
            regs[op[1]] = adj(regs[op[2]])
        elif kind == "mul":
            regs[op[1]] = regs[op[2]] @ regs[op[3]]
        elif kind == "add":
            regs[op[1]] = regs[op[2]] + regs[op[3]]
        elif kind == "sub":
            regs[op[1]] = regs[op[2]] - regs[op[3]]
        elif kind == "scale":
            regs[op[1]] = (op[3] + 1j * op[4]) * regs[op[2]]
        elif kind == "shift":
            regs[op[1]] = shift(regs[op[2]], op[3], op[4])
        elif kind == "trace":
            regs[op[1]] = tr(regs[op[2]])[..., None, None] * np.eye(3)
        elif kind == "retr":
            regs[op[1]] = np.real(tr(regs[op[2]]))[..., None, None] * np.eye(3) + 0j
        elif kind == "store":
            result = regs[op[1]]
        else:
            raise ValueError(kind)
    return result


def trace_sum(field):
    """sum_x tr(field(x)) (complex)."""
    return complex(np.sum(tr(field)))


def jacobi_smear(U, chi, kappa, n_iter, norm, dirs=(0, 1, 2, 3)):
    """Listing 1 (Sec. 6): chi <- s0 + kappa * sum_mu [U_mu(x) psi(x+mu) + U_mu(x-mu)^dag psi(x-mu)],
    iterated n_iter times from s0 = chi, then chi /= norm.  chi: (Lt,Lz,Ly,Lx,3), or
    (Lt,Lz,Ly,Lx,4,3) for a fermion (the links act on colour, every spin alike)."""
    if chi.ndim == 6:
        return np.stack([jacobi_smear(U, chi[..., sp, :], kappa, n_iter, norm, dirs)
                         for sp in range(chi.shape[-2])], axis=-2)
    s0 = chi.copy()
    for _ in range(n_iter):
        psi = chi.copy()
        h = np.zeros_like(psi)
        for mu in dirs:
            Umu = U[..., mu, :, :]
            h += (Umu @ shift(psi, mu, +1)[..., None])[..., 0]
            h += shift((adj(Umu) @ psi[..., None])[..., 0], mu, -1)
        chi = s0 + kappa * h
    return chi / norm
