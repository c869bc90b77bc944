"""Pins of the oracle's matrix exponentials against library routines and closed forms.

* brute-force series exp  vs  scipy.linalg.expm (Pade; Al-Mohy & Higham 2009)
* Frechet derivative      vs  scipy.linalg.expm_frechet and a central difference
* Cayley-Hamilton exp(iQ) (Morningstar & Peardon 2004, Sec. III) vs the series,
  over c1 = tr(Q^2)/2 from 0 to 10, both signs of c0 = det Q, the
  degenerate-eigenvalue case and every link of a 2^4 lattice.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import fieldgen
from oracle import expm as oexp
from oracle import stout as ost


def _rand_herm_traceless(rng, n=3):
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    h = 0.5 * (a + a.conj().T)
    return h - np.trace(h) / n * np.eye(n)


def _with_c1(h, c1):
    cur = 0.5 * np.real(np.trace(h @ h))
    return h * np.sqrt(c1 / cur) if c1 > 0 else 0 * h


def test_series_exp_matches_scipy():
    rng = np.random.default_rng(11)
    for scale in (1e-8, 0.1, 1.0, 5.0, 20.0):
        x = scale * (rng.standard_normal((20, 3, 3)) + 1j * rng.standard_normal((20, 3, 3)))
        ours = oexp.expm_series(x)
        ref = np.stack([sla.expm(m) for m in x])
        err = np.max(np.abs(ours - ref)) / max(1.0, np.max(np.abs(ref)))
        assert err < 1e-12, (scale, err)


def test_series_exp_closed_form_diagonal():
    # exp of a diagonal matrix is the elementwise exp of its diagonal
    d = np.array([0.3 + 2.0j, -1.2 + 0.1j, 4.0 - 7.0j])
    assert np.allclose(oexp.expm_series(np.diag(d)), np.diag(np.exp(d)), rtol=1e-14, atol=1e-14)


def test_frechet_matches_scipy_and_fd():
    rng = np.random.default_rng(12)
    for _ in range(5):
        x = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        e = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        ours = oexp.expm_frechet(x, e)
        _, ref = sla.expm_frechet(x, e)
        assert np.max(np.abs(ours - ref)) < 1e-11 * max(1, np.max(np.abs(ref)))
        h = 1e-6
        fd = (sla.expm(x + h * e) - sla.expm(x - h * e)) / (2 * h)
        assert np.max(np.abs(ours - fd)) < 1e-7 * max(1, np.max(np.abs(ref)))


@pytest.mark.parametrize("c1", [0.0, 1e-30, 1e-20, 1e-12, 1e-6, 1e-2, 0.5, 1.0, 10.0])
def test_ch_exp_matches_series_c1_sweep(c1):
    rng = np.random.default_rng(int(1e3 * c1) + 5 if c1 < 1e6 else 5)
    qs = []
    for _ in range(40):
        h = _with_c1(_rand_herm_traceless(rng), c1)
        qs.append(h)
        qs.append(-h)        # flips the sign of c0
    q = np.stack(qs)
    c0 = np.real(np.linalg.det(q))
    if c1 > 0:
        assert (c0 > 0).any() and (c0 < 0).any()
    ours = ost.expiq_ch(q)
    ref = oexp.expm_series(1j * q)
    assert np.max(np.abs(ours - ref)) < 1e-14 * max(1.0, 10 * np.sqrt(c1))


@pytest.mark.parametrize("a", [1e-9, 1e-3, 0.2, 1.0, -0.7])
def test_ch_exp_degenerate_eigenvalues(a):
    # Q = diag(a, a, -2a): w = 0, |c0| = c0max (theta = 0)
    q = np.diag([a, a, -2 * a]).astype(np.complex128)
    v = np.linalg.qr(np.random.default_rng(3).standard_normal((3, 3)) + 0j)[0]
    q = v @ q @ v.conj().T
    ours = ost.expiq_ch(q[None])[0]
    ref = v @ np.diag(np.exp(1j * np.array([a, a, -2 * a]))) @ v.conj().T
    assert np.max(np.abs(ours - ref)) < 1e-14


def test_ch_exp_zero_is_identity():
    q = np.zeros((4, 3, 3), dtype=np.complex128)
    assert np.array_equal(ost.expiq_ch(q), np.broadcast_to(np.eye(3), q.shape))


@pytest.mark.parametrize("gen", ["haar", "near"])
def test_ch_exp_on_2_4_lattice_links(gen):
    dims = (2, 2, 2, 2)
    U = fieldgen.haar_su3(dims, 7) if gen == "haar" else fieldgen.near_identity_su3(dims, 7)
    for rho in (0.1, 0.25):
        dirs = (0, 1, 2, 3)
        for mu in dirs:
            _, _, Q = ost.stout_q(U, mu, rho, dirs)
            err = np.max(np.abs(ost.expiq_ch(Q) - oexp.expm_series(1j * Q)))
            assert err < 1e-14, (gen, rho, mu, err)
