"""Pins of the oracle's expression programs and Jacobi smearing (Listing 1, Sec. 6).

* shift(shift(f, +, mu), -, mu) = f;  sum_x of a shifted field = sum_x of the field
* sum_x tr(A(x) B(x)) = sum_x tr(B(x) A(x))
* a program forming U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag and
  summing Re tr reproduces the (separately pinned) plaquette
* Jacobi smearing with unit links on a plane wave: the hopping term is
  2 sum_mu cos(p_mu) times the wave, so chi_n is a geometric series
* Jacobi smearing is gauge covariant: chi -> g chi under U -> U^g
"""
import numpy as np

import fieldgen
from oracle import expr, gauge, lattice


def test_shift_roundtrip_and_sum():
    dims = (3, 4, 2, 5)
    U = fieldgen.haar_su3(dims, 40)
    for mu in range(4):
        prog = [("loadl", 0, 0, 1, mu, +1), ("shift", 1, 0, mu, -1), ("store", 1)]
        assert np.array_equal(expr.eval_program(prog, [U]), U[..., 1, :, :])
        prog = [("loadl", 0, 0, 2, mu, -1), ("store", 0)]
        assert abs(expr.trace_sum(expr.eval_program(prog, [U])) - expr.trace_sum(U[..., 2, :, :])) < 1e-12


def test_trace_cyclic():
    dims = (3, 3, 2, 2)
    U = fieldgen.haar_su3(dims, 41)
    ab = [("loadl", 0, 0, 0, 0, 0), ("loadl", 1, 0, 1, 0, 0), ("mul", 2, 0, 1), ("store", 2)]
    ba = [("loadl", 0, 0, 0, 0, 0), ("loadl", 1, 0, 1, 0, 0), ("mul", 2, 1, 0), ("store", 2)]
    a = expr.trace_sum(expr.eval_program(ab, [U]))
    b = expr.trace_sum(expr.eval_program(ba, [U]))
    assert abs(a - b) < 1e-12


def test_plaquette_program():
    dims = (3, 2, 4, 3)
    U = fieldgen.near_identity_su3(dims, 42)
    tot = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            prog = [("loadl", 0, 0, mu, 0, 0), ("loadl", 1, 0, nu, mu, +1),
                    ("loadl", 2, 0, mu, nu, +1), ("loadl", 3, 0, nu, 0, 0),
                    ("mul", 4, 0, 1), ("adj", 5, 2), ("mul", 4, 4, 5), ("adj", 6, 3),
                    ("mul", 4, 4, 6), ("retr", 7, 4), ("store", 7)]
            tot += expr.trace_sum(expr.eval_program(prog, [U])).real / 3.0
    V = lattice.volume(dims)
    assert abs(tot / (18 * V) - gauge.plaquette(U)[0]) < 1e-14


def test_jacobi_unit_links_plane_wave():
    dims = (4, 4, 4, 8)
    U = fieldgen.unit_links(dims)
    n = np.array([1, 3, 2, 5])
    p = 2 * np.pi * n / np.array(dims)
    lt, lz, ly, lx = lattice.field_shape(dims)
    t, z, y, x = np.meshgrid(range(lt), range(lz), range(ly), range(lx), indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    v = np.array([0.3 + 0.1j, -1.0 + 0.0j, 0.5j])
    chi = phase[..., None] * v
    kappa, n_iter, norm = 0.21, 5, 1.7
    lam = 2 * np.sum(np.cos(p))
    coef = sum((kappa * lam) ** k for k in range(n_iter + 1)) / norm
    got = expr.jacobi_smear(U, chi, kappa, n_iter, norm)
    assert np.max(np.abs(got - coef * chi)) < 1e-12


def test_jacobi_gauge_covariant():
    dims = (3, 4, 3, 2)
    U = fieldgen.haar_su3(dims, 43)
    g = fieldgen.gauge_field_g(dims, 44)
    chi = fieldgen.color_vector(dims, 45)
    a = expr.jacobi_smear(gauge.gauge_transform(U, g), (g @ chi[..., None])[..., 0], 0.2, 3, 1.0)
    b = (g @ expr.jacobi_smear(U, chi, 0.2, 3, 1.0)[..., None])[..., 0]
    assert np.max(np.abs(a - b)) < 1e-12


def test_jacobi_subset_of_directions_and_fermion():
    """With unit links a plane wave is an eigenvector of the hopping term summed
    over `dirs` with eigenvalue 2 sum_{mu in dirs} cos p_mu; a fermion is smeared
    spin by spin (the links act on colour only)."""
    dims = (4, 4, 4, 8)
    U = fieldgen.unit_links(dims)
    n = np.array([1, 3, 2, 5])
    p = 2 * np.pi * n / np.array(dims)
    lt, lz, ly, lx = lattice.field_shape(dims)
    t, z, y, x = np.meshgrid(range(lt), range(lz), range(ly), range(lx), indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    spins = np.array([[0.3, -1.0, 0.5j], [1j, 0.2, 0.0], [0.0, 0.0, 1.0], [-0.5, 0.25j, 2.0]])
    chi = phase[..., None, None] * spins
    kappa, n_iter, norm, dirs = 0.17, 4, 2.0, (0, 1, 2)
    lam = 2 * np.sum(np.cos(p[list(dirs)]))
    coef = sum((kappa * lam) ** k for k in range(n_iter + 1)) / norm
    got = expr.jacobi_smear(U, chi, kappa, n_iter, norm, dirs)
    assert np.max(np.abs(got - coef * chi)) < 1e-12
    Uh = fieldgen.haar_su3(dims, 46)
    f = fieldgen.color_vector(dims, 47)
    ferm = np.stack([f, 2 * f, -f, 1j * f], axis=-2)
    one = expr.jacobi_smear(Uh, f, kappa, 2, norm, dirs)
    both = expr.jacobi_smear(Uh, ferm, kappa, 2, norm, dirs)
    for sp, c in enumerate((1, 2, -1, 1j)):
        assert np.max(np.abs(both[..., sp, :] - c * one)) < 1e-12


def test_program_operand_promotion():
    """A colour vector v loads as the matrix [v 0 0] and a scalar s as s * 1, so
    (U v)(x) of a program equals the matrix-vector product, and s * U scales."""
    dims = (3, 2, 2, 3)
    U = fieldgen.haar_su3(dims, 48)
    v = fieldgen.color_vector(dims, 49)
    s = np.random.default_rng(50).standard_normal(lattice.field_shape(dims)) + 0.5j
    prog = [("loadl", 0, 0, 2, 1, -1), ("load", 1, 1, 1, -1), ("mul", 2, 0, 1), ("store", 2)]
    got = expr.as_vector(expr.eval_program(prog, [U, v]))
    ref = lattice.shift((U[..., 2, :, :] @ v[..., None])[..., 0], 1, -1)
    assert np.max(np.abs(got - ref)) < 1e-14
    prog = [("load", 0, 1, 0, 0), ("loadl", 1, 0, 3, 0, 0), ("mul", 2, 0, 1), ("store", 2)]
    got = expr.eval_program(prog, [U, s])
    assert np.max(np.abs(got - s[..., None, None] * U[..., 3, :, :])) < 1e-14
    assert np.array_equal(expr.as_scalar(expr.as_matrix(s)), s)
