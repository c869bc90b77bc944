"""GPU Jacobi smearing (lq_jacobi_smear, Listing 1) vs the oracle.

FP64: max |chi_gpu - chi_oracle| <= 1e-12 * max |chi_oracle|; FP32: 1e-5 relative
per iteration (products of ~50 FP32 operations per component and iteration).
"""
import numpy as np
import pytest

import fieldgen
import paper_1105_2279_gb300 as lq
from oracle import expr
from tests.gpu_util import upload_links

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["vector", "fermion"])
@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
@pytest.mark.parametrize("dims,n_iter,dirs", [((4, 4, 4, 8), 5, (0, 1, 2, 3)), ((3, 5, 2, 7), 3, (0, 1, 2)),
                                              ((2, 2, 2, 2), 2, (0, 1, 2, 3)), ((6, 4, 5, 3), 1, (3,)),
                                              ((4, 3, 4, 5), 0, (0, 1, 2, 3))])
def test_jacobi_matches_oracle(gpu, kind, prec, dims, n_iter, dirs):
    U = fieldgen.haar_su3(dims, 600)
    v = fieldgen.color_vector(dims, 601)
    chi = v if kind == "vector" else np.stack([v, 0.5 * v[::-1], 1j * v, -v], axis=-2)
    kappa, norm = 0.21, 1.7
    ref = expr.jacobi_smear(U, chi, kappa, n_iter, norm, dirs)
    fU = upload_links(U, prec)
    fchi = lq.Field.from_host(fU.geom, lq.LQ_COLOR_VECTOR if kind == "vector" else lq.LQ_FERMION, prec, chi)
    lq.jacobi_smear(fU, fchi, kappa, n_iter, norm, dirs)
    got = fchi.download().astype(np.complex128)
    tol = 1e-12 if prec == lq.LQ_F64 else 1e-5 * max(1, n_iter)
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))


def test_jacobi_rejects_bad_arguments(gpu):
    dims = (2, 2, 2, 2)
    fU = upload_links(fieldgen.unit_links(dims), lq.LQ_F64)
    v = lq.Field.from_host(fU.geom, lq.LQ_COLOR_VECTOR, lq.LQ_F64, fieldgen.color_vector(dims, 1))
    m = lq.Field(fU.geom, lq.LQ_COLOR_MATRIX, lq.LQ_F64)
    for args, status in [((fU, m, 0.1, 1, 1.0), -2), ((fU, v, 0.1, 1, 0.0), -1), ((fU, v, 0.1, -1, 1.0), -1)]:
        with pytest.raises(lq.LqError) as e:
            lq.jacobi_smear(*args)
        assert e.value.status == status


@pytest.mark.parametrize("kind", ["vector", "fermion"])
@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
@pytest.mark.parametrize("dims,n_iter,dirs", [((4, 4, 4, 8), 5, (0, 1, 2, 3)), ((3, 5, 2, 7), 3, (0, 1, 2)),
                                              ((2, 2, 2, 2), 2, (0, 1, 2, 3))])
def test_jacobi_compressed_links(gpu, kind, prec, dims, n_iter, dirs):
    """Links read as rows 0 and 1 with row 2 rebuilt as conj(row0 x row1):
    exact for SU(3), so the result meets the oracle at the same tolerance."""
    U = fieldgen.haar_su3(dims, 610)
    v = fieldgen.color_vector(dims, 611)
    chi = v if kind == "vector" else np.stack([v, 0.5 * v[::-1], 1j * v, -v], axis=-2)
    ref = expr.jacobi_smear(U, chi, 0.21, n_iter, 1.7, dirs)
    fU = upload_links(U, prec)
    k = lq.LQ_COLOR_VECTOR if kind == "vector" else lq.LQ_FERMION
    fchi = lq.Field.from_host(fU.geom, k, prec, chi)
    lq.jacobi_smear(fU, fchi, 0.21, n_iter, 1.7, dirs, compress_links=True)
    got = fchi.download().astype(np.complex128)
    tol = 1e-12 if prec == lq.LQ_F64 else 1e-5 * max(1, n_iter)
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    plain = lq.Field.from_host(fU.geom, k, prec, chi)
    lq.jacobi_smear(fU, plain, 0.21, n_iter, 1.7, dirs)
    assert np.max(np.abs(got - plain.download().astype(np.complex128))) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("kind", ["vector", "fermion"])
@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
def test_jacobi_thread_geometry_bitwise(gpu, kind, prec):
    """Every (N_threads, N_site) of the tuner's search space gives the default
    launch's result bit for bit; the volume (5*3*7*9 = 945 sites) is a
    multiple of no block size, so every shape has a ragged last block."""
    dims = (5, 3, 7, 9)
    U = fieldgen.haar_su3(dims, 620)
    v = fieldgen.color_vector(dims, 621)
    chi = v if kind == "vector" else np.stack([v, 0.5 * v[::-1], 1j * v, -v], axis=-2)
    fU = upload_links(U, prec)
    k = lq.LQ_COLOR_VECTOR if kind == "vector" else lq.LQ_FERMION
    ref = lq.Field.from_host(fU.geom, k, prec, chi)
    lq.jacobi_smear(fU, ref, 0.21, 3, 1.7)
    want = ref.download()
    for block in (32, 64, 128, 256):
        for nsite in (1, 2, 4, 8):
            f = lq.Field.from_host(fU.geom, k, prec, chi)
            lq.jacobi_smear(fU, f, 0.21, 3, 1.7, block=block, sites_per_thread=nsite)
            assert np.array_equal(f.download(), want), (block, nsite)


def test_jacobi_tuner_picks_a_shape_and_keeps_results(gpu, tmp_path):
    dims = (6, 6, 6, 12)
    U = fieldgen.haar_su3(dims, 630)
    v = fieldgen.color_vector(dims, 631)
    fU = upload_links(U, lq.LQ_F32)
    a = lq.Field.from_host(fU.geom, lq.LQ_COLOR_VECTOR, lq.LQ_F32, v)
    lq.jacobi_smear(fU, a, 0.21, 4, 1.7)
    cache = tmp_path / "tune.txt"
    lq.tune(str(cache))
    b = lq.Field.from_host(fU.geom, lq.LQ_COLOR_VECTOR, lq.LQ_F32, v)
    lq.jacobi_smear(fU, b, 0.21, 4, 1.7)           # tunes, then smears with the chosen shape
    assert np.array_equal(a.download(), b.download())
    entries = [ln.split() for ln in cache.read_text().splitlines() if ln.startswith("jacobi_vector ")]
    assert len(entries) == 1
    block, nsite = int(entries[0][-3]), int(entries[0][-2])
    assert block in (32, 64, 128, 256) and nsite in (1, 2, 4, 8)
