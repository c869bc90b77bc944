"""Pins of the APE-force oracle (oracle/ape_force.py).

The projection's gradient against central differences of Re tr(R^dag P(V))
(Richardson-extrapolated, so the differencing error is far below the pin);
the force of S_W(ape^n(U)) against central differences of the per-site
action along random su(3) directions, in 4 and 3 smeared directions and on
Haar-random links; the closed-form divided difference of x^(-1/2) against
the plain quotient and the derivative; and the special cases the definition
fixes: alpha = 0 and a single smeared direction leave every link in place
(P(r U) = U), so the force is the thin field's Wilson force; n = 0 is the
Wilson gradient itself; the force is gauge covariant.
"""
import numpy as np
import pytest
from scipy.linalg import expm

import fieldgen
from oracle import ape, ape_force, gauge
from oracle.su3 import adj

ALL, SPATIAL = (0, 1, 2, 3), (0, 1, 2)


def test_divided_difference_closed_form():
    rng = np.random.default_rng(70)
    a = rng.uniform(0.05, 5.0, size=200)
    b = rng.uniform(0.05, 5.0, size=200)
    quotient = (a ** -0.5 - b ** -0.5) / (a - b)
    assert np.max(np.abs(ape_force.inv_sqrt_divided_difference(a, b) / quotient - 1.0)) < 1e-10
    assert np.max(np.abs(ape_force.inv_sqrt_divided_difference(a, a) / (-0.5 * a ** -1.5) - 1.0)) < 1e-15


def _richardson(f, h):
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(2 * h) - f(-2 * h)) / (4 * h)
    return (4 * d1 - d2) / 3


@pytest.mark.parametrize("kind", ["gaussian", "near_unitary", "scaled_su3"])
def test_projection_gradient_matches_fd(kind):
    rng = np.random.default_rng({"gaussian": 71, "near_unitary": 72, "scaled_su3": 73}[kind])
    for _ in range(6):
        if kind == "gaussian":
            V = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
        else:
            U = fieldgen.haar_su3((1, 1, 1, 1), int(rng.integers(1 << 30)))[0, 0, 0, 0, 0]
            E = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
            V = 0.7 * U + (0.1 * E if kind == "near_unitary" else 0.0)
        R = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
        D = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
        fd = _richardson(lambda t: float(np.real(np.trace(adj(R) @ ape.project_su3(V + t * D)))), 1e-3)
        an = float(np.real(np.trace(adj(ape_force.project_su3_vjp(V, R)) @ D)))
        assert abs(fd - an) < 1e-9 * max(1.0, abs(an)), (fd, an)


def _fd_force(U, mu, x, X, alpha, n, dirs, beta, h=1e-3):
    def s(t):
        P = U.copy()
        P[x + (mu,)] = expm(t * X) @ U[x + (mu,)]
        return float(np.sum(gauge.local_action(ape.ape_smear(P, alpha, n, dirs), beta)))
    base = float(np.sum(gauge.local_action(ape.ape_smear(U, alpha, n, dirs), beta)))
    return _richardson(lambda t: s(t) - base, h)


@pytest.mark.parametrize("dirs,n,field", [(ALL, 2, "near"), (SPATIAL, 2, "near"), (ALL, 1, "haar")])
def test_force_matches_fd(dirs, n, field):
    dims = (3, 3, 3, 3)
    U = fieldgen.near_identity_su3(dims, 74) if field == "near" else fieldgen.haar_su3(dims, 75)
    F, _ = ape_force.smeared_wilson_force(U, 0.6, n, dirs, 6.0)
    rng = np.random.default_rng(76)
    for _ in range(4):
        mu = int(rng.integers(4))
        x = tuple(int(rng.integers(k)) for k in U.shape[:4])
        X = fieldgen.su3_direction(rng)
        fd = _fd_force(U, mu, x, X, 0.6, n, dirs, 6.0)
        an = float(np.real(np.trace(adj(F[x + (mu,)]) @ X)))
        assert abs(fd - an) < 2e-9 * max(1.0, abs(an)), (mu, x, fd, an)


@pytest.mark.parametrize("alpha,dirs", [(0.0, ALL), (0.6, (2,))])
def test_links_left_in_place_give_the_wilson_force(alpha, dirs):
    dims = (3, 2, 3, 2)
    U = fieldgen.haar_su3(dims, 77)
    F, _ = ape_force.smeared_wilson_force(U, alpha, 2, dirs, 6.0)
    F0 = gauge.force_from_grad(gauge.wilson_action_grad(U, 6.0), U)
    assert np.max(np.abs(F - F0)) < 1e-13


def test_zero_steps_is_the_wilson_gradient():
    U = fieldgen.haar_su3((2, 3, 2, 3), 78)
    _, G = ape_force.smeared_wilson_force(U, 0.6, 0, ALL, 6.0)
    assert np.array_equal(G, gauge.wilson_action_grad(U, 6.0))


def test_force_is_gauge_covariant():
    dims = (3, 3, 2, 3)
    U = fieldgen.near_identity_su3(dims, 79)
    g = fieldgen.gauge_field_g(dims, 80)
    Fa, _ = ape_force.smeared_wilson_force(gauge.gauge_transform(U, g), 0.5, 2, ALL, 6.0)
    Fb, _ = ape_force.smeared_wilson_force(U, 0.5, 2, ALL, 6.0)
    # F_mu(x) = TA(G U^dag) transforms with g(x) on both sides
    Fb = g[..., None, :, :] @ Fb @ adj(g)[..., None, :, :]
    assert np.max(np.abs(Fa - Fb)) < 1e-12
