"""GPU HYP smearing (lq_hyp_smear) against the oracle (oracle/hyp.py).

FP64 on near-identity fields: 1e-12 per step.  Three nested SU(3)
projections amplify rounding by the condition number of each level's mixed
matrix, which on Haar-random fields can be large: there 1e-9.  FP32 (FP32
staples and mixing, FP64 projections): 1e-5 per step.
"""
import numpy as np
import pytest

import fieldgen
import paper_1105_2279_gb300 as lq
from oracle import ape, hyp
from oracle.su3 import unitarity_violation
from tests.gpu_util import upload_links

pytestmark = pytest.mark.gpu
W = (0.75, 0.6, 0.3)


def _run(U, prec, w, n):
    f = upload_links(U, prec)
    lq.hyp_smear(f, *w, n_steps=n)
    return f.download().astype(np.complex128)


@pytest.mark.parametrize("dims,gen,w,n", [
    ((4, 4, 4, 4), "near", W, 1),
    ((3, 4, 5, 6), "near", W, 2),
    ((2, 2, 2, 2), "near", W, 2),
    ((4, 3, 2, 5), "near", (0.5, 0.4, 0.2), 3),
    ((4, 4, 4, 4), "haar", W, 1),
])
@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
def test_hyp_matches_oracle(gpu, prec, dims, gen, w, n):
    U = fieldgen.haar_su3(dims, 140) if gen == "haar" else fieldgen.near_identity_su3(dims, 140)
    ref = hyp.hyp_smear(U, *w, n)
    got = _run(U, prec, w, n)
    if prec == lq.LQ_F64:
        tol = (1e-12 if gen == "near" else 1e-9) * n
    else:
        tol = 1e-5 * n
    assert np.max(np.abs(got - ref)) <= tol
    du, dd = unitarity_violation(got)
    assert du < (1e-13 if prec == lq.LQ_F64 else 5e-7) and dd < (1e-13 if prec == lq.LQ_F64 else 5e-7)


def test_hyp_reductions(gpu):
    """Unit fields stay fixed; zero weights change nothing; with a2 = a3 = 0
    one step is an APE step of weight a1."""
    dims = (3, 4, 3, 4)
    one = fieldgen.unit_links(dims)
    assert np.max(np.abs(_run(one, lq.LQ_F64, W, 2) - one)) <= 1e-15
    U = fieldgen.near_identity_su3(dims, 141)
    assert np.max(np.abs(_run(U, lq.LQ_F64, (0.0, 0.0, 0.0), 1) - U)) <= 1e-14
    assert np.max(np.abs(_run(U, lq.LQ_F64, (0.7, 0.0, 0.0), 1) - ape.ape_step(U, 0.7, (0, 1, 2, 3)))) <= 1e-13


def test_hyp_rejects_bad_arguments(gpu):
    f = upload_links(fieldgen.unit_links((2, 2, 2, 2)), lq.LQ_F64)
    with pytest.raises(lq.LqError):
        lq.hyp_smear(f, float("inf"), 0.6, 0.3)
    with pytest.raises(lq.LqError):
        lq.hyp_smear(f, n_steps=-1)
