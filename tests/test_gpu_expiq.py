"""GPU exp(iQ) (lq_expiq, the stout step's Cayley-Hamilton exponential) in
each regime of the Morningstar-Peardon formulas, against the matrix
exponential by scaled Taylor series (oracle/expm.py) and the oracle's own
Cayley-Hamilton form (oracle/stout.py).

Regimes: generic spectra of several scales, exactly degenerate spectra
(a, a, -2a) of both signs of c0 = det Q (theta = 0), near-degenerate spectra
(w -> 0, the xi0 series), c0 = 0 (theta = pi/2), Q = 0, eigenvalues of ~100
(argument reduction of the FP64 sine and cosine), and c1 = tr(Q^2)/2 on
either side of 3/4, where the library switches from the reduced Taylor
series of exp(iQ) to the closed form, and of each series-order threshold.

Tolerances (max abs over all entries): FP64, 1e-15 * max(4, lambda_max^2):
the rounding of u, w and the h_j grows with |Q|^2 (the oracle's own CH form
meets 1.2e-15 at lambda ~ 1 and 1.4e-12 at lambda ~ 250 against the series).
FP32: the oracle is evaluated on the FP32-rounded Q; 2e-6 * max(1, lambda_max / 4)
covers the FP32 square Q^2 and the FP32-rounded f_j.
"""
import math

import numpy as np
import pytest

import fieldgen
import paper_1105_2279_gb300 as lq
from oracle import expm as oexp
from oracle import stout as ost

pytestmark = pytest.mark.gpu

DIMS = (5, 4, 3, 7)   # 420 sites: a ragged last block of 128 threads


def _hermitian(lam, seed):
    V = fieldgen.gauge_field_g(DIMS, seed)
    Q = V @ (lam[..., :, None] * np.conj(np.swapaxes(V, -1, -2)))
    return 0.5 * (Q + np.conj(np.swapaxes(Q, -1, -2)))


def _spectrum(regime, rng):
    shape = tuple(reversed(DIMS)) + (3,)
    if regime.startswith("scale"):
        lam = rng.normal(size=shape) * float(regime[5:])
    elif regime == "degenerate_pos":        # (a, a, -2a), a > 0: c0 < 0
        a = rng.uniform(0.1, 3.0, size=shape[:-1])
        lam = np.stack([a, a, -2 * a], axis=-1)
    elif regime == "degenerate_neg":        # a < 0: c0 > 0
        a = -rng.uniform(0.1, 3.0, size=shape[:-1])
        lam = np.stack([a, a, -2 * a], axis=-1)
    elif regime == "near_degenerate":       # w ~ 1e-7 .. 1e-2: xi0 series branch
        a = rng.uniform(-2.0, 2.0, size=shape[:-1])
        eps = 10.0 ** rng.uniform(-7, -2, size=shape[:-1])
        lam = np.stack([a + eps, a - eps, -2 * a], axis=-1)
    elif regime == "c0_zero":               # (a, 0, -a): theta = pi/2
        a = rng.uniform(0.1, 3.0, size=shape[:-1])
        lam = np.stack([a, np.zeros_like(a), -a], axis=-1)
    elif regime == "zero":
        lam = np.zeros(shape)
    elif regime.startswith("c1="):            # generic directions, c1 fixed per site
        lam = rng.normal(size=shape)
        lam -= lam.mean(axis=-1, keepdims=True)
        c1 = 0.5 * np.sum(lam * lam, axis=-1, keepdims=True)
        return lam * np.sqrt(float(regime[3:]) / c1)
    else:
        raise ValueError(regime)
    return lam - lam.mean(axis=-1, keepdims=True)


# series-order thresholds (3/4)(tol (2K+2)!)^(1/(K+1)) of the FP32 (1e-13) and
# FP64 (1e-17) paths, each straddled
_EDGES = [0.75 * (tol * math.factorial(2 * K + 2)) ** (1.0 / (K + 1))
          for tol, kmax in ((1e-13, 6), (1e-17, 8)) for K in range(1, kmax + 1)]
REGIMES = (["scale1e-15", "scale1e-14", "scale1e-3", "scale0.3", "scale1", "scale3", "scale30",
            "degenerate_pos", "degenerate_neg", "near_degenerate", "c0_zero", "zero",
            "c1=0.7499", "c1=0.7501", "c1=0.3", "c1=2.0"]
           + [f"c1={c * f:.9g}" for c in _EDGES for f in (0.999, 1.001)])


def _run(Q, prec):
    g = lq.Geometry(DIMS)
    fq = lq.Field.from_host(g, lq.LQ_COLOR_MATRIX, prec, Q)
    fe = lq.Field(g, lq.LQ_COLOR_MATRIX, prec)
    lq.expiq(fe, fq)
    return fe.download().astype(np.complex128), fq.download().astype(np.complex128)


@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
@pytest.mark.parametrize("regime", REGIMES)
def test_expiq_regimes(gpu, regime, prec):
    rng = np.random.default_rng(100 + REGIMES.index(regime))
    lam = _spectrum(regime, rng)
    Q = _hermitian(lam, 7)
    got, Qd = _run(Q, prec)
    lmax = float(np.max(np.abs(lam)))
    if prec == lq.LQ_F64:
        # the library exponentiates the traceless part; V diag(lambda) V^dag
        # carries a trace of up to ~1e-14 from the rounding of V
        Qt = Q - (np.trace(Q, axis1=-2, axis2=-1) / 3.0)[..., None, None] * np.eye(3)
        tol = 1e-15 * max(4.0, lmax ** 2)
        assert np.max(np.abs(got - oexp.expm_series(1j * Qt))) <= tol
        assert np.max(np.abs(got - ost.expiq_ch(Qt))) <= tol
        eye = np.eye(3)
        assert np.max(np.abs(got @ np.conj(np.swapaxes(got, -1, -2)) - eye)) <= tol
    else:
        # the FP32 input as the kernel saw it, made exactly Hermitian traceless
        Qh = 0.5 * (Qd + np.conj(np.swapaxes(Qd, -1, -2)))
        Qh = Qh - (np.trace(Qh, axis1=-2, axis2=-1) / 3.0)[..., None, None] * np.eye(3)
        tol = 2e-6 * max(1.0, lmax / 4.0)
        assert np.max(np.abs(got - oexp.expm_series(1j * Qh))) <= tol


def test_expiq_zero_is_identity_bitwise(gpu):
    got, _ = _run(np.zeros(tuple(reversed(DIMS)) + (3, 3), np.complex128), lq.LQ_F64)
    assert np.array_equal(got, np.broadcast_to(np.eye(3), got.shape))


@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
def test_expiq_reads_hermitian_traceless_part(gpu, prec):
    """Only the upper triangle and the real diagonal are read, and a trace
    is removed: exp(i Q) of Q + t*1 + (noise below the diagonal and in the
    imaginary diagonal) equals exp(i Q)."""
    rng = np.random.default_rng(11)
    Q = _hermitian(_spectrum("scale1", rng), 8)
    shape = Q.shape
    noise = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    lower = np.tril(np.ones((3, 3)), -1)
    P = Q + noise * lower + 1j * np.eye(3) * rng.normal(size=shape[:-2] + (1, 1))
    P = P + rng.normal(size=shape[:-2])[..., None, None] * np.eye(3)
    got_p, _ = _run(P, prec)
    got_q, _ = _run(Q, prec)
    tol = 1e-14 if prec == lq.LQ_F64 else 2e-6
    assert np.max(np.abs(got_p - got_q)) <= tol
    Qt = Q - (np.trace(Q, axis1=-2, axis2=-1) / 3.0)[..., None, None] * np.eye(3)
    assert np.max(np.abs(got_q - oexp.expm_series(1j * Qt))) <= (1e-14 if prec == lq.LQ_F64 else 3e-6)


def test_expiq_rejects_bad_arguments(gpu):
    g = lq.Geometry(DIMS)
    q = lq.Field(g, lq.LQ_COLOR_MATRIX, lq.LQ_F64)
    with pytest.raises(lq.LqError):
        lq.expiq(q, q)
    with pytest.raises(lq.LqError):
        lq.expiq(lq.Field(g, lq.LQ_COLOR_MATRIX, lq.LQ_F32), q)
    with pytest.raises(lq.LqError):
        lq.expiq(lq.Field(g, lq.LQ_LINKS, lq.LQ_F64), q)
    with pytest.raises(lq.LqError):
        lq.expiq(lq.Field(lq.Geometry((4, 4, 3, 7)), lq.LQ_COLOR_MATRIX, lq.LQ_F64), q)
