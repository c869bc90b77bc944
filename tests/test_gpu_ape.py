"""GPU APE smearing (lq_ape_smear) against the oracle (oracle/ape.py).

FP64: max |U_gpu - U_oracle| <= 1e-12 (the projection's eigenvalues and the
inverse square root are FP64 throughout).  FP32 (FP32 mixing, FP64
projection): <= 2e-6 per step, as for the stout step.
"""
import numpy as np
import pytest

import fieldgen
import paper_1105_2279_gb300 as lq
from oracle import ape
from oracle.su3 import unitarity_violation
from tests.gpu_util import upload_links

pytestmark = pytest.mark.gpu
ALL, SPATIAL = (0, 1, 2, 3), (0, 1, 2)


def _run(U, prec, alpha, n, dirs):
    f = upload_links(U, prec)
    lq.ape_smear(f, alpha, n, dirs)
    return f.download().astype(np.complex128)


@pytest.mark.parametrize("dims,gen,alpha,n,dirs", [
    ((4, 4, 4, 4), "haar", 0.5, 1, ALL),
    ((3, 4, 5, 6), "near", 0.6, 3, ALL),
    ((3, 4, 5, 6), "near", 0.45, 2, SPATIAL),
    ((5, 3, 2, 7), "haar", 0.3, 2, (1, 3)),
    ((2, 2, 2, 2), "haar", 0.5, 2, ALL),
    ((4, 3, 4, 2), "near", 0.7, 1, (2,)),
])
@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
def test_ape_matches_oracle(gpu, prec, dims, gen, alpha, n, dirs):
    U = fieldgen.haar_su3(dims, 130) if gen == "haar" else fieldgen.near_identity_su3(dims, 130)
    ref = ape.ape_smear(U, alpha, n, dirs)
    got = _run(U, prec, alpha, n, dirs)
    tol = 1e-12 if prec == lq.LQ_F64 else 2e-6 * n
    assert np.max(np.abs(got - ref)) <= tol
    du, dd = unitarity_violation(got)
    assert du < (1e-13 if prec == lq.LQ_F64 else 5e-7) and dd < (1e-13 if prec == lq.LQ_F64 else 5e-7)
    for mu in range(4):
        if mu not in dirs:
            assert np.array_equal(got[..., mu, :, :], U[..., mu, :, :].astype(got.dtype) if prec == lq.LQ_F64
                                  else U[..., mu, :, :].astype(np.complex64).astype(np.complex128))


def test_ape_fixed_points(gpu):
    dims = (3, 4, 3, 4)
    one = fieldgen.unit_links(dims)
    assert np.max(np.abs(_run(one, lq.LQ_F64, 0.6, 3, ALL) - one)) <= 1e-15
    U = fieldgen.haar_su3(dims, 131)
    assert np.max(np.abs(_run(U, lq.LQ_F64, 0.0, 2, ALL) - U)) <= 1e-14


def test_ape_rejects_bad_arguments(gpu):
    f = upload_links(fieldgen.unit_links((2, 2, 2, 2)), lq.LQ_F64)
    with pytest.raises(lq.LqError):
        lq.ape_smear(f, float("nan"), 1)
    with pytest.raises(lq.LqError):
        lq.ape_smear(f, 0.5, -1)
    with pytest.raises(lq.LqError):
        lq.ape_smear(f, 0.5, 1, dirs=())
