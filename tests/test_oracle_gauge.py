"""Pins of the oracle's plaquette, Wilson action and Wilson-action gradient.

* unit field: plaquette exactly 1, action exactly 0
* abelian (diagonal) links: plaquette from scalar phase sums, written as an
  explicit site loop with its own index arithmetic
* invariance of the plaquette under a random gauge transformation
* Haar-random links: plaquette consistent with 0
* gradient: central differences of the action (per-site differencing) along
  random su(3) directions, and the closed form -beta/3 * staple sum
"""
import itertools

import numpy as np
import pytest

import fieldgen
from oracle import gauge, lattice, stout
from oracle.su3 import adj


def test_unit_field_plaquette_is_one():
    for dims in [(2, 2, 2, 2), (3, 4, 2, 5)]:
        U = fieldgen.unit_links(dims)
        assert gauge.plaquette(U) == (1.0, 1.0, 1.0)
        assert gauge.wilson_action(U, 6.0) == 0.0


def test_abelian_plaquette_closed_form():
    dims = (3, 2, 4, 3)
    U, ang = fieldgen.diagonal_phases(dims, 5)
    lx, ly, lz, lt = dims
    L = dims

    def a(x, mu):  # angle triple of U_mu at coordinate x (x,y,z,t), periodic
        xx = [x[i] % L[i] for i in range(4)]
        return ang[xx[3], xx[2], xx[1], xx[0], mu]

    def step(x, mu):
        y = list(x)
        y[mu] += 1
        return y

    tot, sp, tm = 0.0, 0.0, 0.0
    for x in itertools.product(range(lx), range(ly), range(lz), range(lt)):
        for mu, nu in itertools.combinations(range(4), 2):
            phi = a(x, mu) + a(step(x, mu), nu) - a(step(x, nu), mu) - a(x, nu)
            v = float(np.sum(np.cos(phi)))
            tot += v
            if nu < 3:
                sp += v
            else:
                tm += v
    V = lx * ly * lz * lt
    ref = (tot / (18 * V), sp / (9 * V), tm / (9 * V))
    assert np.allclose(gauge.plaquette(U), ref, rtol=0, atol=1e-14)


@pytest.mark.parametrize("gen", ["haar", "near"])
def test_plaquette_gauge_invariant(gen):
    dims = (4, 3, 2, 4)
    U = fieldgen.haar_su3(dims, 1) if gen == "haar" else fieldgen.near_identity_su3(dims, 1)
    g = fieldgen.gauge_field_g(dims, 2)
    Ug = gauge.gauge_transform(U, g)
    assert np.max(np.abs(Ug - U)) > 0.1
    p, pg = gauge.plaquette(U), gauge.plaquette(Ug)
    assert np.allclose(p, pg, rtol=0, atol=1e-14)
    s, sg = gauge.local_action(U, 6.0), gauge.local_action(Ug, 6.0)
    assert np.max(np.abs(s - sg)) < 1e-13


def test_haar_plaquette_near_zero_and_near_identity_near_06():
    dims = (4, 4, 4, 4)
    p = gauge.plaquette(fieldgen.haar_su3(dims, 0))[0]
    # <Re tr P>/3 = 0 for Haar links; std of the lattice mean ~ 1/sqrt(18 V * 3)
    assert abs(p) < 5.0 / np.sqrt(18 * 256 * 3)
    q = gauge.plaquette(fieldgen.near_identity_su3((6, 6, 6, 6), 1))[0]
    assert 0.45 < q < 0.7


def _fd_force(U, mu, x, X, f_local, eps=1e-6):
    """central difference of sum_x f_local(U) along U_mu(x) -> exp(eps X) U_mu(x)."""
    from scipy.linalg import expm
    t, z, y, xx = x
    up, dn = U.copy(), U.copy()
    up[t, z, y, xx, mu] = expm(eps * X) @ U[t, z, y, xx, mu]
    dn[t, z, y, xx, mu] = expm(-eps * X) @ U[t, z, y, xx, mu]
    return float(np.sum(f_local(up) - f_local(dn))) / (2 * eps)


@pytest.mark.parametrize("gen", ["haar", "near"])
def test_wilson_gradient_fd(gen):
    dims = (3, 3, 3, 4)
    beta = 6.0
    U = fieldgen.haar_su3(dims, 4) if gen == "haar" else fieldgen.near_identity_su3(dims, 4)
    G = gauge.wilson_action_grad(U, beta)
    F = gauge.force_from_grad(G, U)
    rng = np.random.default_rng(9)
    for _ in range(6):
        mu = int(rng.integers(4))
        x = tuple(int(rng.integers(n)) for n in U.shape[:4])
        X = fieldgen.su3_direction(rng)
        fd = _fd_force(U, mu, x, X, lambda V: gauge.local_action(V, beta))
        an = float(np.real(np.trace(adj(F[x + (mu,)]) @ X)))
        assert abs(fd - an) < 1e-7 * max(1.0, abs(an)), (fd, an)


def test_wilson_gradient_is_minus_beta_third_staples():
    dims = (3, 2, 3, 2)
    U = fieldgen.haar_su3(dims, 8)
    G = gauge.wilson_action_grad(U, 6.0)
    for mu in range(4):
        S = stout.staple_sum(U, mu, (0, 1, 2, 3))
        assert np.max(np.abs(G[..., mu, :, :] + 2.0 * S)) < 1e-13


def test_shift_conventions():
    dims = (3, 4, 2, 5)
    f = np.arange(lattice.volume(dims)).reshape(lattice.field_shape(dims))
    for mu in range(4):
        g = lattice.shift(f, mu, +1)
        h = lattice.shift(f, mu, -1)
        for x in [(0, 0, 0, 0), (2, 3, 1, 4), (1, 2, 0, 3)]:
            xp = list(x)
            xp[mu] = (xp[mu] + 1) % dims[mu]
            xm = list(x)
            xm[mu] = (xm[mu] - 1) % dims[mu]
            s = lattice.site_index(*x, dims)
            assert g[x[3], x[2], x[1], x[0]] == s - x[mu] * _stride(dims, mu) + xp[mu] * _stride(dims, mu)
            assert h[x[3], x[2], x[1], x[0]] == s - x[mu] * _stride(dims, mu) + xm[mu] * _stride(dims, mu)


def _stride(dims, mu):
    return int(np.prod(dims[:mu]))
