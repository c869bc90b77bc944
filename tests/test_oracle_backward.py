"""Pins of the oracle's reverse-mode gradient through stout smearing.

Central finite differences along random unit su(3) directions (per-site
differencing of the local action) of S_W(stout^n(U)) against the oracle's
force, in 4 and 3 smeared directions, and the n = 0 closed form.  Step 1e-4
balances truncation (~eps^2) against rounding (~1e-16 * |S_local| / eps) and
pins to 5e-9; the step 1e-6 of the differentiation workload is rounding-limited
and is held to 1e-7.
"""
import numpy as np
import pytest

import fieldgen
from oracle import backward, gauge, stout
from oracle.su3 import adj


def _fd(U, mu, x, X, rho, n, dirs, beta, eps=1e-4):
    from scipy.linalg import expm
    up, dn = U.copy(), U.copy()
    up[x + (mu,)] = expm(eps * X) @ U[x + (mu,)]
    dn[x + (mu,)] = expm(-eps * X) @ U[x + (mu,)]
    su = gauge.local_action(stout.stout_smear(up, rho, n, dirs), beta)
    sd = gauge.local_action(stout.stout_smear(dn, rho, n, dirs), beta)
    return float(np.sum(su - sd)) / (2 * eps)


@pytest.mark.parametrize("dirs,n", [((0, 1, 2, 3), 2), ((0, 1, 2), 2), ((0, 1, 2, 3), 1)])
def test_backward_matches_fd(dirs, n):
    dims = (3, 3, 3, 3)
    beta, rho = 6.0, 0.1
    U = fieldgen.near_identity_su3(dims, 31)
    F, _ = backward.smeared_wilson_force(U, rho, n, dirs, beta)
    rng = np.random.default_rng(32)
    for _ in range(5):
        mu = int(rng.integers(4))
        x = tuple(int(rng.integers(k)) for k in U.shape[:4])
        X = fieldgen.su3_direction(rng)
        fd = _fd(U, mu, x, X, rho, n, dirs, beta)
        an = float(np.real(np.trace(adj(F[x + (mu,)]) @ X)))
        assert abs(fd - an) < 5e-9 * max(1.0, abs(an)), (mu, x, fd, an)
        fd6 = _fd(U, mu, x, X, rho, n, dirs, beta, eps=1e-6)
        assert abs(fd6 - an) < 1e-7 * max(1.0, abs(an)), (mu, x, fd6, an)


def test_backward_haar_fd():
    dims = (3, 3, 2, 3)
    U = fieldgen.haar_su3(dims, 33)
    F, _ = backward.smeared_wilson_force(U, 0.1, 1, (0, 1, 2, 3), 6.0)
    rng = np.random.default_rng(34)
    for _ in range(4):
        mu = int(rng.integers(4))
        x = tuple(int(rng.integers(k)) for k in U.shape[:4])
        X = fieldgen.su3_direction(rng)
        fd = _fd(U, mu, x, X, 0.1, 1, (0, 1, 2, 3), 6.0)
        an = float(np.real(np.trace(adj(F[x + (mu,)]) @ X)))
        assert abs(fd - an) < 5e-9 * max(1.0, abs(an))


def test_backward_zero_steps_is_wilson_force():
    dims = (3, 2, 3, 2)
    U = fieldgen.haar_su3(dims, 35)
    F, G = backward.smeared_wilson_force(U, 0.1, 0, (0, 1, 2, 3), 6.0)
    assert np.array_equal(G, gauge.wilson_action_grad(U, 6.0))


def test_backward_rho_zero_is_pass_through():
    dims = (3, 2, 2, 3)
    U = fieldgen.haar_su3(dims, 36)
    Gout = gauge.wilson_action_grad(U, 6.0)
    G = backward.stout_backward(U, 0.0, 2, (0, 1, 2, 3), Gout)
    assert np.max(np.abs(G - Gout)) < 1e-14
