"""lq_stout_ch_stats (instrumentation of the coefficient stage): its counts of
links on the Taylor-series branch and of their series orders K against c1 =
tr(Q^2)/2 of every link computed by the oracle, step by step.

The branch rule follows from the truncation bound of the series
(|lambda|_max^2 <= 4 c1 / 3, error <= rho^(2K+2) / (2K+2)!): the series is
used for c1 <= 3/4, with the smallest K >= 1 whose threshold
(3/4)(tol (2K+2)!)^(1/(K+1)) is >= c1, tol = 1e-17 for FP64 links.
"""
import math

import numpy as np
import pytest

import fieldgen
import paper_1105_2279_gb300 as lq
from oracle import stout
from tests.gpu_util import upload_links

pytestmark = pytest.mark.gpu


def _expected(U, rho, n, dirs, tol, kmax):
    thr = [0.75 * (tol * math.factorial(2 * K + 2)) ** (1.0 / (K + 1)) for K in range(1, kmax)]
    n_links = n_series = sum_k = 0
    near = 0
    for _ in range(n):
        for mu in dirs:
            _, _, Q = stout.stout_q(U, mu, rho, dirs)
            c1 = np.real(np.trace(Q @ Q, axis1=-2, axis2=-1)).ravel() / 2
            n_links += c1.size
            ser = c1 <= 0.75
            n_series += int(ser.sum())
            sum_k += int(np.sum(1 + np.sum(c1[ser, None] > np.array(thr)[None, :], axis=1)))
            edges = np.array(thr + [0.75])
            near += int(np.sum(np.min(np.abs(c1[:, None] / edges[None, :] - 1), axis=1) < 1e-9))
        U = stout.stout_step(U, rho, dirs)
    return (n_links, n_series, sum_k), near


@pytest.mark.parametrize("rho,gen", [(0.4, "haar"), (0.125, "near"), (0.0, "haar")])
def test_ch_stats_match_oracle_c1(gpu, rho, gen):
    dims = (4, 4, 4, 6)
    U = fieldgen.haar_su3(dims, 300) if gen == "haar" else fieldgen.near_identity_su3(dims, 300)
    f = upload_links(U, lq.LQ_F64)
    got = lq.stout_ch_stats(f, rho, 2, (0, 1, 2, 3))
    exp, near = _expected(U, rho, 2, (0, 1, 2, 3), 1e-17, 9)
    assert near == 0      # no c1 within rounding of a branch edge: counts must agree exactly
    assert got == exp, (got, exp)
    assert np.array_equal(f.download(), U)   # the input field is not modified


def test_ch_stats_f32_counts(gpu):
    dims = (4, 4, 4, 6)
    U = fieldgen.near_identity_su3(dims, 301)
    f = upload_links(U, lq.LQ_F32)
    n, n_series, sum_k = lq.stout_ch_stats(f, 0.125, 3, (0, 1, 2))
    assert n == 3 * 3 * int(np.prod(dims))
    assert n_series == n                      # exp(i 0.3 H) fields: every |lambda| < 1
    assert n_series <= sum_k <= 7 * n_series


def test_ch_stats_unit_links(gpu):
    dims = (3, 3, 3, 3)
    f = upload_links(fieldgen.unit_links(dims), lq.LQ_F64)
    assert lq.stout_ch_stats(f, 0.1, 2, (0, 1, 2, 3)) == (2 * 4 * 81, 2 * 4 * 81, 2 * 4 * 81)  # Q = 0: K = 1
    assert lq.stout_ch_stats(f, 0.1, 0, (0, 1, 2, 3)) == (0, 0, 0)
