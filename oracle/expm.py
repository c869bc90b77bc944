"""Brute-force matrix exponential and its Frechet derivative (oracle; test infrastructure only).

``expm_series`` is the textbook scaling-and-squaring method (Moler & Van
Loan, "Nineteen dubious ways to compute the exponential of a matrix",
SIAM Rev. 20 (1978), method 3 + squaring): scale X by 2^-s until its
1-norm is at most 1/2, sum 30 Taylor terms, square s times.  With
||X/2^s|| <= 1/2 the truncation error is below 0.5^31/31! ~ 1e-43.

``expm_frechet`` returns L(X, E) = d/dt exp(X + tE)|_{t=0} as the upper-right
block of exp([[X, E], [0, X]]) (Mathias, SIAM J. Matrix Anal. Appl. 17
(1996) 610; Higham, "Functions of Matrices" (2008) Thm. 3.6).
"""
import numpy as np

TAYLOR_TERMS = 30


def expm_series(x, terms=TAYLOR_TERMS):
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    norm1 = np.max(np.sum(np.abs(x), axis=-2), axis=-1)  # max column sum
    s = np.maximum(0, np.ceil(np.log2(np.maximum(norm1, 1e-300) / 0.5))).astype(int)
    y = x / (2.0 ** s)[..., None, None]
    eye = np.eye(n, dtype=np.complex128)
    acc = np.broadcast_to(eye, x.shape).copy()
    term = acc.copy()
    for k in range(1, terms + 1):
        term = (term @ y) / k
        acc = acc + term
    for k in range(int(s.max(initial=0))):
        sq = acc @ acc
        acc = np.where((k < s)[..., None, None], sq, acc)
    return acc


def expm_frechet(x, e):
    """L(X, E): derivative of exp at X in direction E (block-matrix identity)."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    big = np.zeros(x.shape[:-2] + (2 * n, 2 * n), dtype=np.complex128)
    big[..., :n, :n] = x
    big[..., n:, n:] = x
    big[..., :n, n:] = e
    return expm_series(big)[..., :n, n:]
