"""Pins of the APE oracle (oracle/ape.py) against what the definition fixes:
the projection returns U for V = r U and for V = U H (H Hermitian positive
definite: the polar factor), lands in SU(3), unit fields and alpha = 0 are
fixed points, the step is gauge covariant and translation invariant, and on
diagonal (abelian) fields it reduces to scalar phase arithmetic, checked
against an explicit site loop."""
import itertools

import numpy as np
import pytest

import fieldgen
from oracle import ape, gauge, lattice
from oracle.su3 import adj, unitarity_violation

ALL, SPATIAL = (0, 1, 2, 3), (0, 1, 2)


def test_projection_of_scaled_su3_is_itself():
    U = fieldgen.haar_su3((3, 2, 2, 3), 40)
    r = np.random.default_rng(41).uniform(0.2, 3.0, size=U.shape[:-2])
    assert np.max(np.abs(ape.project_su3(r[..., None, None] * U) - U)) < 1e-14


def test_projection_is_the_polar_factor():
    rng = np.random.default_rng(42)
    U = fieldgen.haar_su3((2, 2, 2, 2), 43)
    # H = Q diag(positive) Q^dag, Hermitian positive definite
    Q = fieldgen.haar_su3((2, 2, 2, 2), 44)
    d = rng.uniform(0.1, 2.0, size=Q.shape[:-1])
    H = (Q * d[..., None, :]) @ adj(Q)
    assert np.max(np.abs(ape.project_su3(U @ H) - U)) < 1e-13


def test_projection_lands_in_su3():
    rng = np.random.default_rng(45)
    shape = (50, 3, 3)
    V = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    du, dd = unitarity_violation(ape.project_su3(V))
    assert du < 1e-13 and dd < 1e-13


@pytest.mark.parametrize("dirs", [ALL, SPATIAL])
def test_unit_field_and_alpha_zero(dirs):
    dims = (3, 2, 3, 4)
    one = fieldgen.unit_links(dims)
    assert np.max(np.abs(ape.ape_smear(one, 0.6, 2, dirs) - one)) < 1e-15
    U = fieldgen.haar_su3(dims, 46)
    assert np.max(np.abs(ape.ape_step(U, 0.0, dirs) - U)) < 1e-14


@pytest.mark.parametrize("dirs", [ALL, (0, 3)])
def test_gauge_covariance(dirs):
    dims = (3, 4, 2, 3)
    U = fieldgen.near_identity_su3(dims, 47)
    g = fieldgen.gauge_field_g(dims, 48)
    a = ape.ape_step(gauge.gauge_transform(U, g), 0.45, dirs)
    b = gauge.gauge_transform(ape.ape_step(U, 0.45, dirs), g)
    assert np.max(np.abs(a - b)) < 1e-13


def test_translation_invariance():
    dims = (4, 3, 2, 5)
    U = fieldgen.haar_su3(dims, 49)
    off = (1, 2, 0, 3)
    a = ape.ape_step(lattice.translate(U, off), 0.3, ALL)
    b = lattice.translate(ape.ape_step(U, 0.3, ALL), off)
    assert np.max(np.abs(a - b)) < 1e-14


def test_steps_stay_in_su3():
    U = fieldgen.haar_su3((3, 3, 3, 3), 50)
    du, dd = unitarity_violation(ape.ape_smear(U, 0.5, 3, ALL))
    assert du < 1e-13 and dd < 1e-13


@pytest.mark.parametrize("dirs", [ALL, SPATIAL])
def test_abelian_closed_form(dirs):
    """Diagonal links diag(e^{i a_k}): staples are diagonal phases, V is
    diagonal with entries v_k, the polar factor is v_k/|v_k| and the
    determinant fix subtracts the mean phase."""
    dims = (3, 2, 4, 3)
    alpha = 0.37
    U, ang = fieldgen.diagonal_phases(dims, 51, scale=0.9)
    out = ape.ape_step(U, alpha, dirs)
    L = dims

    def a(x, mu):
        return ang[x[3] % L[3], x[2] % L[2], x[1] % L[1], x[0] % L[0], mu]

    def mv(x, mu, d):
        y = list(x)
        y[mu] += d
        return y

    n_staples = 2 * (len(dirs) - 1)
    for x in itertools.product(*[range(n) for n in dims]):
        for mu in range(4):
            if mu not in dirs:
                ref = np.exp(1j * a(x, mu))
            else:
                v = (1 - alpha) * np.exp(1j * a(x, mu))
                for nu in dirs:
                    if nu == mu:
                        continue
                    up = a(x, nu) + a(mv(x, nu, 1), mu) - a(mv(x, mu, 1), nu)
                    xm = mv(x, nu, -1)
                    dn = -a(xm, nu) + a(xm, mu) + a(mv(xm, mu, 1), nu)
                    v = v + alpha / n_staples * (np.exp(1j * up) + np.exp(1j * dn))
                ph = np.angle(v)
                tot = np.angle(np.exp(1j * ph.sum()))          # arg(det W) in (-pi, pi]
                ref = np.exp(1j * (ph - tot / 3.0))
            got = out[x[3], x[2], x[1], x[0], mu]
            assert np.max(np.abs(got - np.diag(ref))) < 1e-14
