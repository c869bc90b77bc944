"""Pins of the oracle's stout smearing (Morningstar & Peardon 2004, Secs. II-III).

* unit field and constant fields are fixed points; rho = 0 is the identity (bitwise)
* smeared links stay in SU(3) (U^dag U = 1, det U = 1 to 1e-13)
* gauge covariance per link: stout(U^g) = stout(U)^g
* translation invariance
* abelian (diagonal) links: closed form from scalar phase arithmetic, written
  as an explicit site loop
* the generator iQ = TA(rho * staples * U^dag) is -(3 rho / beta) times the
  Wilson-action force, whose finite differences are pinned separately
* small-rho limit (U'(rho) - U)/rho -> i Q_1 U
* the 2^4 lattice, where x + mu and x - mu coincide
"""
import itertools

import numpy as np
import pytest

import fieldgen
from oracle import gauge, lattice, stout
from oracle.su3 import adj, ta, unitarity_violation

ALL = (0, 1, 2, 3)
SPATIAL = (0, 1, 2)


def test_unit_field_fixed_point():
    U = fieldgen.unit_links((3, 2, 2, 4))
    for dirs in (ALL, SPATIAL):
        out = stout.stout_smear(U, 0.3, 3, dirs)
        assert np.array_equal(out, U)


def test_rho_zero_identity_bitwise():
    U = fieldgen.haar_su3((3, 3, 2, 2), 3)
    out = stout.stout_smear(U, 0.0, 2, ALL)
    assert np.array_equal(out, U)


def test_constant_field_fixed_point():
    V = fieldgen.haar_su3((1, 1, 1, 1), 6)[0, 0, 0, 0, 0]
    U = np.broadcast_to(V, (2, 3, 2, 3, 4, 3, 3)).copy()
    out = stout.stout_step(U, 0.2, ALL)
    assert np.max(np.abs(out - U)) < 1e-14


@pytest.mark.parametrize("gen", ["haar", "near"])
@pytest.mark.parametrize("dirs", [ALL, SPATIAL])
def test_unitarity(gen, dirs):
    dims = (4, 4, 4, 4)
    U = fieldgen.haar_su3(dims, 0) if gen == "haar" else fieldgen.near_identity_su3(dims, 1)
    for _ in range(3):
        U = stout.stout_step(U, 0.125, dirs)
        du, dd = unitarity_violation(U)
        assert du < 1e-13 and dd < 1e-13, (du, dd)


@pytest.mark.parametrize("dirs", [ALL, SPATIAL])
@pytest.mark.parametrize("dims", [(3, 4, 2, 3), (2, 2, 2, 2)])
def test_gauge_covariance(dirs, dims):
    U = fieldgen.haar_su3(dims, 10)
    g = fieldgen.gauge_field_g(dims, 11)
    a = stout.stout_smear(gauge.gauge_transform(U, g), 0.1, 2, dirs)
    b = gauge.gauge_transform(stout.stout_smear(U, 0.1, 2, dirs), g)
    assert np.max(np.abs(a - b)) < 1e-13
    # the plaquette of the smeared field is gauge invariant too
    assert abs(gauge.plaquette(a)[0] - gauge.plaquette(b)[0]) < 1e-14


def test_translation_invariance():
    dims = (4, 3, 3, 4)
    U = fieldgen.near_identity_su3(dims, 12)
    off = (1, 2, 0, 3)
    a = stout.stout_smear(lattice.translate(U, off), 0.1, 2, ALL)
    b = lattice.translate(stout.stout_smear(U, 0.1, 2, ALL), off)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("dirs", [ALL, SPATIAL])
def test_abelian_closed_form(dirs):
    dims = (3, 2, 4, 3)
    rho = 0.17
    U, ang = fieldgen.diagonal_phases(dims, 21, scale=0.8)
    out = stout.stout_step(U, rho, dirs)
    L = dims

    def a(x, mu):
        return ang[x[3] % L[3], x[2] % L[2], x[1] % L[1], x[0] % L[0], mu]

    def mv(x, mu, d):
        y = list(x)
        y[mu] += d
        return y

    for x in itertools.product(*[range(n) for n in dims]):
        for mu in range(4):
            if mu not in dirs:
                ref = np.exp(1j * a(x, mu))
            else:
                # Omega_kk = rho * sum_nu (e^{i phi_up} + e^{i phi_dn}) e^{-i a_mu(x)}
                im = np.zeros(3)
                for nu in dirs:
                    if nu == mu:
                        continue
                    up = a(x, nu) + a(mv(x, nu, 1), mu) - a(mv(x, mu, 1), nu) - a(x, mu)
                    xm = mv(x, nu, -1)
                    dn = -a(xm, nu) + a(xm, mu) + a(mv(xm, mu, 1), nu) - a(x, mu)
                    im += rho * (np.sin(up) + np.sin(dn))
                # Q_kk = Im Omega_kk - mean; U'_kk = exp(i (Q_kk + a_k))
                q = im - im.mean()
                ref = np.exp(1j * (q + a(x, mu)))
            got = out[x[3], x[2], x[1], x[0], mu]
            assert np.max(np.abs(got - np.diag(ref))) < 1e-14


def test_generator_is_wilson_flow_direction():
    # iQ = TA(rho S U^dag) and the Wilson force is TA(-(beta/3) S U^dag)
    dims = (3, 3, 2, 3)
    beta, rho = 6.0, 0.11
    U = fieldgen.haar_su3(dims, 13)
    F = gauge.force_from_grad(gauge.wilson_action_grad(U, beta), U)
    for mu in ALL:
        _, _, Q = stout.stout_q(U, mu, rho, ALL)
        assert np.max(np.abs(1j * Q + (3 * rho / beta) * F[..., mu, :, :])) < 1e-14


def test_small_rho_linear_order():
    dims = (3, 3, 3, 3)
    U = fieldgen.haar_su3(dims, 14)
    _, _, Q1 = stout.stout_q(U, 2, 1.0, ALL)
    lin = 1j * Q1 @ U[..., 2, :, :]
    errs = []
    for rho in (1e-3, 5e-4):
        d = (stout.stout_step(U, rho, ALL)[..., 2, :, :] - U[..., 2, :, :]) / rho
        errs.append(np.max(np.abs(d - lin)))
    assert errs[1] < 0.6 * errs[0] and errs[0] < 1e-1


def test_spatial_smearing_leaves_time_links():
    U = fieldgen.haar_su3((3, 3, 2, 2), 15)
    out = stout.stout_smear(U, 0.1, 2, SPATIAL)
    assert np.array_equal(out[..., 3, :, :], U[..., 3, :, :])
    assert np.max(np.abs(out[..., 0, :, :] - U[..., 0, :, :])) > 1e-3


def test_smearing_raises_plaquette():
    U = fieldgen.near_identity_su3((4, 4, 4, 4), 16)
    p0 = gauge.plaquette(U)[0]
    p1 = gauge.plaquette(stout.stout_smear(U, 0.1, 2, ALL))[0]
    assert p1 > p0 + 0.05
