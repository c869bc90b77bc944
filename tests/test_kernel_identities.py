"""CPU checks of the algebraic identities the CUDA kernels are built on,
restated in numpy (FP64): a mistake in a kernel's derivation shows here
without a GPU; the kernels themselves are checked on the GPU against the
oracle.

* The closed-form Lyapunov solve of the projection's gradient (APE/HYP
  forces): for Hermitian positive definite Z with elementary symmetric
  functions p1, p2, p3 of its eigenvalues, Y = A C + C A - Z C Z
  - p1 (Z C - C Z) + p2 C with A = Z^2 and C = H (p1 A + p3)^-1 / 2 solves
  Z Y + Y Z = H.
* The gradient of the projection assembled from it,
  G_V = (G_W - 2 W Y) Z^-1 with G_W = conj(z) G_P + (i/3) Im tr(G_P^dag P) W,
  against the oracle's Daleckii-Krein form.
* The FP32-link re-projection's split: with d0 = |u0|^2 - 1, p = u0^dag u1,
  e0 = (1 + d0)^-1/2 - 1, c = (1 + e0)^2 p, d1 = |u1|^2 - 1 - (1 + e0)^2 |p|^2,
  e1 = (1 + d1)^-1/2 - 1, a1 = e1 u1 - c (1 + e1) u0, the rows u0 + e0 u0,
  u1 + a1 and conj(u0 x u1 + e0 (u0 x u1) + (1 + e0) (u0 x a1)) are the
  Gram-Schmidt rows.
"""
import numpy as np
import pytest

import fieldgen
from oracle import ape, ape_force
from oracle.su3 import adj


def _herm(m):
    return 0.5 * (m + adj(m))


def _lyapunov_closed_form(Z, H):
    lam = np.linalg.eigvalsh(Z)
    p1, p2, p3 = lam.sum(), lam[0] * lam[1] + lam[1] * lam[2] + lam[0] * lam[2], lam.prod()
    A = Z @ Z
    C = H @ np.linalg.inv(p1 * A + p3 * np.eye(3)) / 2.0
    return A @ C + C @ A - Z @ C @ Z - p1 * (Z @ C - C @ Z) + p2 * C


@pytest.mark.parametrize("spread", [1.0, 1e-6, 10.0])
def test_lyapunov_closed_form(spread):
    rng = np.random.default_rng(11)
    for _ in range(20):
        Q = fieldgen.haar_su3((1, 1, 1, 1), int(rng.integers(1 << 30)))[0, 0, 0, 0, 0]
        s = 1.0 + spread * rng.uniform(0.0, 1.0, 3)
        Z = (Q * s) @ adj(Q)
        H = _herm(rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3)))
        Y = _lyapunov_closed_form(Z, H)
        assert np.max(np.abs(Z @ Y + Y @ Z - H)) < 1e-12 * max(1.0, spread)


def test_projection_gradient_assembly_matches_daleckii_krein():
    rng = np.random.default_rng(12)
    for _ in range(20):
        V = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
        if np.linalg.cond(V) > 10:
            continue
        G_P = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
        P = ape.project_su3(V)
        A = adj(V) @ V
        lam, q = np.linalg.eigh(A)
        Z = (q * np.sqrt(lam)) @ adj(q)
        X = np.linalg.inv(Z)
        W = V @ X
        z = np.exp(-1j * np.angle(np.linalg.det(W)) / 3.0)
        G_W = np.conj(z) * G_P + (1j / 3.0) * np.imag(np.trace(adj(G_P) @ P)) * W
        Y = _lyapunov_closed_form(Z, _herm(adj(V) @ G_W))
        G_V = (G_W - 2.0 * W @ Y) @ X
        ref = ape_force.project_su3_vjp(V, G_P)
        assert np.max(np.abs(G_V - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_reprojection_split_is_gram_schmidt():
    rng = np.random.default_rng(13)
    U = fieldgen.haar_su3((2, 2, 2, 2), 14).reshape(-1, 3, 3)
    for u in U:
        u = u + 1e-6 * (rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3)))
        u0, u1 = u[0], u[1]
        # Gram-Schmidt, written out
        r0 = u0 / np.linalg.norm(u0)
        r1 = u1 - np.vdot(r0, u1) * r0
        r1 = r1 / np.linalg.norm(r1)
        r2 = np.conj(np.cross(r0, r1))
        # the split
        d0 = np.vdot(u0, u0).real - 1.0
        p = np.vdot(u0, u1)
        e0 = (1.0 + d0) ** -0.5 - 1.0
        c = (1.0 + e0) ** 2 * p
        d1 = np.vdot(u1, u1).real - 1.0 - (1.0 + e0) ** 2 * abs(p) ** 2
        e1 = (1.0 + d1) ** -0.5 - 1.0
        a1 = e1 * u1 - c * (1.0 + e1) * u0
        x = np.cross(u0, u1)
        s0, s1 = u0 + e0 * u0, u1 + a1
        s2 = np.conj(x + e0 * x + (1.0 + e0) * np.cross(u0, a1))
        assert np.max(np.abs(s0 - r0)) < 1e-15
        assert np.max(np.abs(s1 - r1)) < 1e-15
        assert np.max(np.abs(s2 - r2)) < 1e-15


def _series_deriv(c0, c1, K):
    """numpy restatement of the kernels' differentiated Horner series of
    exp(iQ) reduced by Q^3 = c1 Q + c0 (degree 2K+1), with the c1 derivative
    carried as X1 = dx/dc1 + z: returns f_j, df_j/dc1, df_j/dc0."""
    from math import factorial
    x = y = z = x0 = y0 = z0 = X1 = y1 = z1 = 0j
    for n in range(2 * K + 1, -1, -1):
        a = (1j ** n) / factorial(n)
        x, x0, X1, y, y0, y1, z, z0, z1 = (c0 * z + a, c0 * z0 + z, c0 * z1 + y, c1 * z + x, c1 * z0 + x0,
                                           c1 * z1 + X1, y, y0, y1)
    return np.array([x, y, z]), np.array([X1 - z, y1, z1]), np.array([x0, y0, z0])


def _diag_q(c0, c1):
    """Diagonal traceless Hermitian Q with det Q = c0 and tr(Q^2)/2 = c1 (the
    roots of l^3 - c1 l - c0)."""
    lam = np.sort(np.real(np.roots([1.0, 0.0, -c1, -c0])))
    return np.diag(lam).astype(np.complex128)


@pytest.mark.parametrize("c1,frac", [(0.02, 0.3), (0.3, -0.7), (0.74, 0.95), (0.01, -0.1)])
def test_series_derivative_recurrence(c1, frac):
    """f_j of the series equal the oracle's Cayley-Hamilton coefficients, and
    its c1 and c0 derivatives equal central differences of the oracle's f_j
    (spectra with the prescribed c0, c1 from the characteristic cubic)."""
    from oracle import stout
    c0 = frac * 2.0 * (c1 / 3.0) ** 1.5
    f, b1, b2 = _series_deriv(c0, c1, 10)
    ref = np.array(stout.ch_coefficients(_diag_q(c0, c1)))
    # f_j multiplies Q^j ~ c1^(j/2) (the closed form loses eps/c1^(j/2) on f_j as Q -> 0)
    scale = np.sqrt(c1) ** np.arange(3)
    assert np.max(np.abs(f - ref) * scale) <= 1e-14
    h1 = 1e-5 * c1
    d1 = (np.array(stout.ch_coefficients(_diag_q(c0, c1 + h1))) -
          np.array(stout.ch_coefficients(_diag_q(c0, c1 - h1)))) / (2 * h1)
    c0max = 2.0 * (c1 / 3.0) ** 1.5
    h0 = 1e-5 * c0max
    d0 = (np.array(stout.ch_coefficients(_diag_q(c0 + h0, c1))) -
          np.array(stout.ch_coefficients(_diag_q(c0 - h0, c1)))) / (2 * h0)
    assert np.max(np.abs(b1 - d1)) <= 1e-6 * max(1.0, np.max(np.abs(d1)))
    assert np.max(np.abs(b2 - d0)) <= 1e-6 * max(1.0, np.max(np.abs(d0)))


def test_fp32_derivative_series_order_is_enough():
    """FP32 links differentiate the series at one order more than the f_j's
    (FP32 table, tol 1e-10): over the whole series domain the truncated
    b1_j = df_j/dc1 and b2_j = df_j/dc0 enter d exp(iQ) = sum_j (b1_j dc1 +
    b2_j dc0) Q^j + ... with an error <= 2.4e-12 per unit |dQ| (dc1 ~ 2|Q||dQ|,
    dc0 ~ 3|Q|^2 |dQ|), far below the FP32 rounding of the gradient (6e-8);
    checked against the series taken to order 12."""
    th = [3.67423461e-05, 0.00312012573, 0.0336079014, 0.153820376, 0.451978133]
    worst = 0.0
    for c1 in np.geomspace(1e-12, 0.75, 300):
        K = 2 + sum(c1 > t for t in th)
        q = np.sqrt(4.0 * c1 / 3.0)
        for frac in (-0.99, -0.5, 0.0, 0.5, 0.99):
            c0 = frac * 2.0 * (c1 / 3.0) ** 1.5
            _, b1, b2 = _series_deriv(c0, c1, K)
            _, B1, B2 = _series_deriv(c0, c1, 12)
            e1 = max(abs(b1[j] - B1[j]) * q ** j for j in range(3)) * 2.0 * q
            e2 = max(abs(b2[j] - B2[j]) * q ** j for j in range(3)) * 3.0 * q * q
            worst = max(worst, e1, e2)
    assert worst <= 2.4e-12, worst


def test_fp32_forward_series_order_is_enough():
    """The f_j of FP32 links come from the series at the order of the FP32
    table (tol 1e-10: K = 1 + the number of thresholds below c1, at most 6):
    over the whole series domain (c1 <= 3/4, every c0 of the cubic's range)
    the truncated f_j, weighted by |Q|^j <= (4 c1 / 3)^(j/2), stay within
    1e-10 of the series taken to order 14, 600x below the FP32 rounding of
    the f_j; the thresholds are (3/4)(tol (2K+2)!)^(1/(K+1))."""
    from math import factorial
    th = [3.67423461e-05, 0.00312012573, 0.0336079014, 0.153820376, 0.451978133]
    for K, t in enumerate(th, start=1):
        assert abs(t - 0.75 * (1e-10 * factorial(2 * K + 2)) ** (1.0 / (K + 1))) <= 1e-8 * t
    assert 0.75 * (1e-10 * factorial(14)) ** (1.0 / 7) > 0.75     # K = 6 covers the series domain
    worst = 0.0
    for c1 in np.geomspace(1e-12, 0.75, 400):
        K = 1 + sum(c1 > t for t in th)
        q = np.sqrt(4.0 * c1 / 3.0)
        for frac in (-0.99, -0.5, 0.0, 0.5, 0.99):
            c0 = frac * 2.0 * (c1 / 3.0) ** 1.5
            f, _, _ = _series_deriv(c0, c1, K)
            F, _, _ = _series_deriv(c0, c1, 14)
            worst = max(worst, max(abs(f[j] - F[j]) * q ** j for j in range(3)))
    assert worst <= 1e-10, worst


def _d2f_bits(d):
    """numpy restatement of the kernels' integer-pipe double -> float
    conversion (IEEE-754 bit fields, round to nearest even; signed zero
    below the FP32 normal range, infinity above it, NaN kept)."""
    b = np.asarray(d, dtype=np.float64).view(np.uint64)
    hi = (b >> np.uint64(32)).astype(np.uint64)
    lo = (b & np.uint64(0xffffffff)).astype(np.uint64)
    sign = hi & np.uint64(0x80000000)
    mag = hi & np.uint64(0x7fffffff)
    e = (mag >> np.uint64(20)).astype(np.int64) - 896
    f = sign | (np.clip(e, 0, 255).astype(np.uint64) << np.uint64(23)) | ((hi & np.uint64(0xfffff)) << np.uint64(3)) \
        | (lo >> np.uint64(29))
    rest = lo & np.uint64(0x1fffffff)
    f = f + np.where(rest > 0x10000000, 1, np.where(rest == 0x10000000, f & np.uint64(1), 0)).astype(np.uint64)
    nan = (mag > 0x7ff00000) | ((mag == 0x7ff00000) & (lo != 0))
    f = np.where(e <= 0, sign, np.where(e >= 255, sign | np.uint64(0x7f800000) | np.where(nan, 0x400000, 0).astype(np.uint64), f))
    return (f & np.uint64(0xffffffff)).astype(np.uint32).view(np.float32)


def test_integer_double_to_float_conversion():
    """The conversion equals numpy's (IEEE round to nearest even) over the
    FP32 normal range, including exact ties and carries into the exponent,
    and gives zero / infinity / NaN outside it."""
    rng = np.random.default_rng(77)
    d = np.concatenate([rng.standard_normal(200000) * 10.0 ** rng.integers(-30, 30, 200000),
                        rng.standard_normal(1000)])
    # exact ties between two floats, both parities, and values that round up to the next binade
    f = rng.standard_normal(1000).astype(np.float32)
    up = np.nextafter(f, np.float32(np.inf))
    d = np.concatenate([d, 0.5 * (f.astype(np.float64) + up.astype(np.float64)),
                        [np.float64(np.nextafter(np.float32(2.0), np.float32(0))) + 2.0 ** -26,
                         1.0, -1.0, 3.4028234663852886e38, 1.1754943508222875e-38]])
    assert np.array_equal(_d2f_bits(d).view(np.uint32), d.astype(np.float32).view(np.uint32))
    special = np.array([0.0, -0.0, 1e-39, -1e-45, 1e-300, 4e38, -1e300, np.inf, -np.inf, np.nan])
    got = _d2f_bits(special)
    assert np.array_equal(got[:5].view(np.uint32), np.array([0, 0x80000000, 0, 0x80000000, 0], dtype=np.uint32))
    assert got[5] == np.inf and got[6] == -np.inf and got[7] == np.inf and got[8] == -np.inf
    assert np.isnan(got[9])
