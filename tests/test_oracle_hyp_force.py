"""Pins of the HYP-force oracle (oracle/hyp_force.py).

The two-field staple gradient against central differences of Re tr(K^dag S)
(S is cubic in the links, so the Richardson-extrapolated difference is exact
up to rounding); the force of S_W(hyp^n(U)) against central differences of
the per-site action along random su(3) directions; with a2 = a3 = 0 the
inner levels return the thin links (P(U) = U on SU(3)) and the force equals
the APE force of weight a1 (pinned on its own); zero weights give the thin
field's Wilson force, n = 0 the Wilson gradient bitwise; the force is gauge
covariant.
"""
import numpy as np
import pytest
from scipy.linalg import expm

import fieldgen
from oracle import ape_force, gauge, hyp, hyp_force, lattice
from oracle.su3 import adj

W = (0.75, 0.6, 0.3)


def _richardson(f, h):
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(2 * h) - f(-2 * h)) / (4 * h)
    return (4 * d1 - d2) / 3


@pytest.mark.parametrize("mu,eta", [(0, 1), (3, 2), (1, 3)])
def test_staple_gradient_matches_fd(mu, eta):
    dims = (3, 4, 3, 2)
    rng = np.random.default_rng(90 + 4 * mu + eta)
    shape = lattice.field_shape(dims) + (3, 3)
    A, B, K, dA, dB = (rng.normal(size=shape) + 1j * rng.normal(size=shape) for _ in range(5))
    ga, gb = hyp_force.staples_vjp(A, B, mu, eta, K)
    f = lambda t: float(np.sum(np.real(np.conj(K) * hyp.staples(A + t * dA, B + t * dB, mu, eta))))
    fd = _richardson(f, 1e-2)
    an = float(np.sum(np.real(np.conj(ga) * dA)) + np.sum(np.real(np.conj(gb) * dB)))
    assert abs(fd - an) < 1e-11 * abs(an)


def _fd_force(U, mu, x, X, n, weights, h=1e-3):
    def s(t):
        P = U.copy()
        P[x + (mu,)] = expm(t * X) @ U[x + (mu,)]
        return float(np.sum(gauge.local_action(hyp.hyp_smear(P, *weights, n), 6.0)))
    base = float(np.sum(gauge.local_action(hyp.hyp_smear(U, *weights, n), 6.0)))
    return _richardson(lambda t: s(t) - base, h)


@pytest.mark.parametrize("n,field", [(1, "near"), (2, "near"), (1, "haar")])
def test_force_matches_fd(n, field):
    dims = (3, 3, 3, 3)
    U = fieldgen.near_identity_su3(dims, 92) if field == "near" else fieldgen.haar_su3(dims, 93)
    F, _ = hyp_force.smeared_wilson_force(U, *W, n, 6.0)
    rng = np.random.default_rng(94)
    for _ in range(3):
        mu = int(rng.integers(4))
        x = tuple(int(rng.integers(k)) for k in U.shape[:4])
        X = fieldgen.su3_direction(rng)
        fd = _fd_force(U, mu, x, X, n, W)
        an = float(np.real(np.trace(adj(F[x + (mu,)]) @ X)))
        assert abs(fd - an) < 2e-9 * max(1.0, abs(an)), (mu, x, fd, an)


@pytest.mark.parametrize("field", ["near", "haar"])
def test_outer_level_alone_is_the_ape_force(field):
    dims = (3, 2, 3, 3)
    U = fieldgen.near_identity_su3(dims, 95) if field == "near" else fieldgen.haar_su3(dims, 95)
    Fh, _ = hyp_force.smeared_wilson_force(U, 0.7, 0.0, 0.0, 2, 6.0)
    Fa, _ = ape_force.smeared_wilson_force(U, 0.7, 2, (0, 1, 2, 3), 6.0)
    assert np.max(np.abs(Fh - Fa)) < (1e-13 if field == "near" else 1e-10)


def test_zero_weights_give_the_wilson_force():
    U = fieldgen.haar_su3((2, 3, 2, 3), 96)
    F, _ = hyp_force.smeared_wilson_force(U, 0.0, 0.0, 0.0, 1, 6.0)
    F0 = gauge.force_from_grad(gauge.wilson_action_grad(U, 6.0), U)
    assert np.max(np.abs(F - F0)) < 1e-13


def test_zero_steps_is_the_wilson_gradient():
    U = fieldgen.haar_su3((2, 2, 3, 2), 97)
    _, G = hyp_force.smeared_wilson_force(U, *W, 0, 6.0)
    assert np.array_equal(G, gauge.wilson_action_grad(U, 6.0))


def test_force_is_gauge_covariant():
    dims = (3, 3, 2, 3)
    U = fieldgen.near_identity_su3(dims, 98)
    g = fieldgen.gauge_field_g(dims, 99)
    Fa, _ = hyp_force.smeared_wilson_force(gauge.gauge_transform(U, g), *W, 1, 6.0)
    Fb, _ = hyp_force.smeared_wilson_force(U, *W, 1, 6.0)
    Fb = g[..., None, :, :] @ Fb @ adj(g)[..., None, :, :]
    assert np.max(np.abs(Fa - Fb)) < 1e-12
