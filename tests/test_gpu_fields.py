"""GPU reductions, shift, expression programs and transfers through the C ABI
vs the oracle.

Reductions accumulate in FP64: FP64 fields agree with the oracle to 1e-13
relative (different summation order); FP32 fields to 1e-6 relative.  Shift
and upload/download are bit exact.  Reductions are bit-identical run to run.
"""
import numpy as np
import pytest

import fieldgen
import paper_1105_2279_gb300 as lq
from oracle import expr, gauge, lattice
from tests.gpu_util import upload_links

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
def test_upload_download_roundtrip(gpu, prec):
    dims = (3, 5, 2, 7)
    U = fieldgen.haar_su3(dims, 200)
    f = upload_links(U, prec)
    back = f.download()
    want = U if prec == lq.LQ_F64 else U.astype(np.complex64)
    assert np.array_equal(back, want)
    # device layout is [dir][comp][site] (re, im)
    t = f.tensor.cpu().numpy()
    s = lattice.site_index(1, 3, 1, 4, dims)
    assert t[2, 5, s, 0] == want[4, 1, 3, 1, 2, 1, 2].real
    assert t[2, 5, s, 1] == want[4, 1, 3, 1, 2, 1, 2].imag


@pytest.mark.parametrize("kind,prec", [(lq.LQ_LINKS, lq.LQ_F64), (lq.LQ_LINKS, lq.LQ_F32),
                                       (lq.LQ_FERMION, lq.LQ_F32), (lq.LQ_REAL, lq.LQ_F64)])
def test_pinned_upload_download_equal_pageable(gpu, kind, prec):
    """From page-locked host memory the transposes read and write the host
    buffer themselves (no staging copy): the same bytes as the pageable path
    (staging copy, then transpose); ragged volume, several field kinds."""
    import torch
    dims = (3, 5, 7, 11)
    g = lq.Geometry(dims)
    a = lq.Field(g, kind, prec)
    rng = np.random.default_rng(210)
    real = np.float64 if prec == lq.LQ_F64 else np.float32
    host = rng.standard_normal(a.nbytes // np.dtype(real).itemsize).astype(real)
    pinned = torch.from_numpy(host.copy()).pin_memory()
    a.upload_ptr(host.ctypes.data)
    b = lq.Field(g, kind, prec)
    b.upload_ptr(pinned.data_ptr())
    assert torch.equal(a.tensor, b.tensor)
    out = torch.zeros_like(pinned).pin_memory()
    b.download_ptr(out.data_ptr())
    assert np.array_equal(out.numpy(), host)


@pytest.mark.parametrize("dims,gen", [((4, 4, 4, 4), "haar"), ((2, 2, 2, 2), "near"),
                                      ((3, 4, 5, 6), "near"), ((8, 8, 8, 16), "near")])
def test_plaquette(gpu, dims, gen):
    U = fieldgen.haar_su3(dims, 201) if gen == "haar" else fieldgen.near_identity_su3(dims, 201)
    ref = gauge.plaquette(U)
    f64 = upload_links(U, lq.LQ_F64)
    got = lq.plaquette(f64)
    assert np.allclose(got, ref, rtol=0, atol=1e-14)
    assert lq.plaquette(f64) == got          # deterministic
    f32 = upload_links(U, lq.LQ_F32)
    assert np.allclose(lq.plaquette(f32), ref, rtol=0, atol=2e-6)
    S = lq.wilson_action(f64, 6.0)
    assert abs(S - gauge.wilson_action(U, 6.0)) < 1e-12 * max(1.0, abs(S))


def test_unit_plaquette_exact(gpu):
    f = upload_links(fieldgen.unit_links((3, 4, 5, 2)), lq.LQ_F64)
    assert lq.plaquette(f) == (1.0, 1.0, 1.0)
    assert lq.wilson_action(f, 6.0) == 0.0


@pytest.mark.parametrize("kind", [lq.LQ_LINKS, lq.LQ_COLOR_MATRIX, lq.LQ_COLOR_VECTOR, lq.LQ_COMPLEX, lq.LQ_REAL])
@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
def test_shift_all_kinds(gpu, kind, prec):
    dims = (3, 4, 5, 2)
    g = lq.Geometry(dims)
    rng = np.random.default_rng(202)
    shape = lattice.field_shape(dims) + lq.SITE_SHAPE[kind]
    a = rng.standard_normal(shape) + (0 if kind == lq.LQ_REAL else 1j * rng.standard_normal(shape))
    fin = lq.Field.from_host(g, kind, prec, a)
    fout = lq.Field(g, kind, prec)
    host = a.astype(fin.host_dtype())
    for mu in range(4):
        for sign in (1, -1):
            lq.shift(fout, fin, mu, sign)
            assert np.array_equal(fout.download(), lattice.shift(host, mu, sign))


@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
def test_reduce_sum_and_trace(gpu, prec):
    dims = (5, 3, 4, 3)
    U = fieldgen.haar_su3(dims, 203)
    f = upload_links(U, prec)
    tol = 1e-12 if prec == lq.LQ_F64 else 1e-5
    ref_sum = complex(np.sum(U.astype(f.host_dtype()).astype(np.complex128)))
    assert abs(lq.reduce_sum(f) - ref_sum) < tol * max(1, abs(ref_sum))
    ref_tr = complex(np.sum(np.trace(U.astype(f.host_dtype()).astype(np.complex128), axis1=-2, axis2=-1)))
    assert abs(lq.reduce_trace(f) - ref_tr) < tol * max(1, abs(ref_tr))
    g = lq.Geometry(dims)
    r = np.random.default_rng(204).standard_normal(lattice.field_shape(dims))
    fr = lq.Field.from_host(g, lq.LQ_REAL, prec, r)
    assert abs(lq.reduce_sum(fr).real - r.astype(fr.host_dtype()).astype(np.float64).sum()) < tol * 100


def micro_suite_programs():
    """Programs of the micro-suite on a links operand (index 0)."""
    # sum_mu tr(U_mu(x) U_mu(x+mu))
    p_tr = []
    for mu in range(4):
        p_tr += [("loadl", 0, 0, mu, 0, 0), ("loadl", 1, 0, mu, mu, +1), ("mul", 2, 0, 1)]
        p_tr += [("add", 3, 3, 2)] if mu else [("add", 3, 2, 2), ("sub", 3, 3, 2)]
    p_tr += [("store", 3)]
    # U_mu(x) U_nu(x+mu)^dag for (mu, nu) = (0, 1) and (2, 3)
    p_adj = [[("loadl", 0, 0, mu, 0, 0), ("loadl", 1, 0, nu, mu, +1), ("adj", 2, 1), ("mul", 3, 0, 2), ("store", 3)]
             for mu, nu in [(0, 1), (2, 3)]]
    return p_tr, p_adj


@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
def test_micro_suite_expressions(gpu, prec):
    dims = (6, 4, 5, 8)
    U = fieldgen.near_identity_su3(dims, 205)
    g = lq.Geometry(dims)
    fU = upload_links(U, prec)
    p_tr, p_adj = micro_suite_programs()
    tol = 1e-12 if prec == lq.LQ_F64 else 2e-5
    got = lq.expr_eval(p_tr, [fU], reduce=True)
    ref = expr.trace_sum(expr.eval_program(p_tr, [U]))
    assert abs(got - ref) < tol * max(1.0, abs(ref))
    for p in p_adj:
        out = lq.Field(g, lq.LQ_COLOR_MATRIX, prec)
        red = lq.expr_eval(p, [fU], out=out, reduce=True)
        ref_field = expr.eval_program(p, [U])
        assert np.max(np.abs(out.download() - ref_field)) < (1e-14 if prec == lq.LQ_F64 else 1e-6)
        assert abs(red - expr.trace_sum(ref_field)) < tol * max(1.0, abs(red))


def test_plaquette_program_matches_plaquette(gpu):
    dims = (4, 3, 4, 5)
    U = fieldgen.near_identity_su3(dims, 206)
    fU = upload_links(U, lq.LQ_F64)
    tot = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            prog = [("loadl", 0, 0, mu, 0, 0), ("loadl", 1, 0, nu, mu, +1), ("loadl", 2, 0, mu, nu, +1),
                    ("loadl", 3, 0, nu, 0, 0), ("mul", 4, 0, 1), ("adj", 5, 2), ("mul", 4, 4, 5), ("adj", 6, 3),
                    ("mul", 4, 4, 6), ("retr", 7, 4), ("store", 7)]
            tot += lq.expr_eval(prog, [fU], reduce=True).real / 3.0
    assert abs(tot / (18 * lattice.volume(dims)) - lq.plaquette(fU)[0]) < 1e-13


def test_jacobi_hopping_term_program(gpu):
    """One Jacobi iteration of Listing 1 built from C-ABI expression programs
    (colour-vector operand, shifts pushed to the loads) vs the oracle."""
    dims = (4, 3, 4, 6)
    U = fieldgen.haar_su3(dims, 207)
    chi = fieldgen.color_vector(dims, 208)
    g = lq.Geometry(dims)
    fU = upload_links(U, lq.LQ_F64)
    fchi = lq.Field.from_host(g, lq.LQ_COLOR_VECTOR, lq.LQ_F64, chi)
    kappa = 0.21
    prog = []
    for mu in range(4):
        # U_mu(x) chi(x+mu) + U_mu(x-mu)^dag chi(x-mu)
        prog += [("loadl", 0, 0, mu, 0, 0), ("load", 1, 1, mu, +1), ("mul", 2, 0, 1),
                 ("loadl", 3, 0, mu, mu, -1), ("adj", 3, 3), ("load", 4, 1, mu, -1), ("mul", 5, 3, 4),
                 ("add", 2, 2, 5)]
        prog += [("add", 6, 6, 2)] if mu else [("add", 6, 2, 2), ("sub", 6, 6, 2)]
    prog += [("scale", 6, 6, kappa, 0.0), ("load", 7, 1, 0, 0), ("add", 6, 6, 7), ("store", 6)]
    out = lq.Field(g, lq.LQ_COLOR_VECTOR, lq.LQ_F64)
    lq.expr_eval(prog, [fU, fchi], out=out)
    ref = expr.jacobi_smear(U, chi, kappa, 1, 1.0)
    assert np.max(np.abs(out.download() - ref)) < 1e-13


@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
def test_jit_programs_bit_identical_to_interpreter(gpu, prec):
    """NVRTC-compiled programs (lq_expr_eval_jit) give bit-identical fields and
    reductions to the interpreted ones, for every output kind."""
    dims = (5, 4, 3, 6)
    U = fieldgen.near_identity_su3(dims, 209)
    chi = fieldgen.color_vector(dims, 210)
    g = lq.Geometry(dims)
    fU = upload_links(U, prec)
    fchi = lq.Field.from_host(g, lq.LQ_COLOR_VECTOR, prec, chi)
    p_tr, p_adj = micro_suite_programs()
    assert lq.expr_eval_jit(p_tr, [fU], reduce=True) == lq.expr_eval(p_tr, [fU], reduce=True)
    for p in p_adj:
        a, b = lq.Field(g, lq.LQ_COLOR_MATRIX, prec), lq.Field(g, lq.LQ_COLOR_MATRIX, prec)
        ra = lq.expr_eval_jit(p, [fU], out=a, reduce=True)
        rb = lq.expr_eval(p, [fU], out=b, reduce=True)
        assert ra == rb and np.array_equal(a.download(), b.download())
    hop = [("loadl", 0, 0, 2, 0, 0), ("load", 1, 1, 2, +1), ("mul", 2, 0, 1), ("loadl", 3, 0, 2, 2, -1),
           ("adj", 3, 3), ("load", 4, 1, 2, -1), ("mul", 5, 3, 4), ("add", 2, 2, 5),
           ("scale", 2, 2, 0.21, 0.0), ("load", 6, 1, 0, 0), ("add", 2, 2, 6), ("store", 2)]
    a, b = lq.Field(g, lq.LQ_COLOR_VECTOR, prec), lq.Field(g, lq.LQ_COLOR_VECTOR, prec)
    lq.expr_eval_jit(hop, [fU, fchi], out=a)
    lq.expr_eval(hop, [fU, fchi], out=b)
    assert np.array_equal(a.download(), b.download())
    for kind, prog in ((lq.LQ_COMPLEX, [("loadl", 0, 0, 1, 3, -1), ("trace", 1, 0), ("store", 1)]),
                       (lq.LQ_REAL, [("loadl", 0, 0, 0, 0, 0), ("loadl", 1, 0, 3, 0, +1), ("mul", 2, 0, 1),
                                     ("retr", 3, 2), ("store", 3)])):
        a, b = lq.Field(g, kind, prec), lq.Field(g, kind, prec)
        lq.expr_eval_jit(prog, [fU], out=a)
        lq.expr_eval(prog, [fU], out=b)
        assert np.array_equal(a.download(), b.download())
    before = lq.jit_stats()
    lq.expr_eval_jit(p_tr, [fU], reduce=True)          # cached: no new compilation or module load
    after = lq.jit_stats()
    assert after[0] == before[0] and after[3] == before[3] and after[1] == before[1] + 1


def test_library_owned_fields(gpu):
    """lq_field_alloc / lq_field_device_ptr / lq_field_free through the C ABI:
    a library-owned field uploads, smears and downloads like a wrapped one."""
    import ctypes
    lib = lq.capi()
    dims = (4, 3, 4, 5)
    U = fieldgen.near_identity_su3(dims, 211)
    g = lq.Geometry(dims)
    h = ctypes.c_void_p()
    assert lib.lq_field_alloc(g.handle, lq.LQ_LINKS, lq.LQ_F64, None, ctypes.byref(h)) == 0
    p = ctypes.c_void_p()
    assert lib.lq_field_device_ptr(h, ctypes.byref(p)) == 0 and p.value
    host = np.ascontiguousarray(U)
    assert lib.lq_field_upload(h, ctypes.c_void_p(host.ctypes.data), None) == 0
    assert lib.lq_stout_smear(h, 0.1, 2, 15, None, None) == 0
    back = np.empty_like(host)
    assert lib.lq_field_download(h, ctypes.c_void_p(back.ctypes.data), None) == 0
    ref = upload_links(U, lq.LQ_F64)
    lq.stout_smear(ref, 0.1, 2, (0, 1, 2, 3), stream=0)
    assert np.array_equal(back, ref.download())
    assert lib.lq_field_free(h) == 0


@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
def test_programs_with_vector_and_scalar_operands(gpu, prec):
    """Colour-vector, complex and real operands and outputs (register-machine
    promotion) vs the oracle, interpreted and compiled."""
    dims = (4, 3, 5, 2)
    U = fieldgen.haar_su3(dims, 212)
    v = fieldgen.color_vector(dims, 213)
    rng = np.random.default_rng(214)
    z = rng.standard_normal(lattice.field_shape(dims)) + 1j * rng.standard_normal(lattice.field_shape(dims))
    r = rng.standard_normal(lattice.field_shape(dims))
    g = lq.Geometry(dims)
    fU = upload_links(U, prec)
    fv = lq.Field.from_host(g, lq.LQ_COLOR_VECTOR, prec, v)
    fz = lq.Field.from_host(g, lq.LQ_COMPLEX, prec, z)
    fr = lq.Field.from_host(g, lq.LQ_REAL, prec, r)
    host = [U, v, z, r]
    if prec == lq.LQ_F32:
        host = [U.astype(np.complex64), v.astype(np.complex64), z.astype(np.complex64), r.astype(np.float32)]
    tol = 1e-13 if prec == lq.LQ_F64 else 2e-6
    # z(x) * U_1(x-mu_3)^dag v(x-mu_3) + r(x+mu_0) v(x)  -> colour vector
    prog = [("load", 0, 2, 0, 0), ("loadl", 1, 0, 1, 3, -1), ("adj", 1, 1), ("load", 2, 1, 3, -1),
            ("mul", 3, 1, 2), ("mul", 3, 0, 3), ("load", 4, 3, 0, +1), ("load", 5, 1, 0, 0), ("mul", 4, 4, 5),
            ("add", 3, 3, 4), ("store", 3)]
    ref = expr.as_vector(expr.eval_program(prog, host))
    for ev in (lq.expr_eval, lq.expr_eval_jit):
        out = lq.Field(g, lq.LQ_COLOR_VECTOR, prec)
        ev(prog, [fU, fv, fz, fr], out=out)
        assert np.max(np.abs(out.download() - ref)) <= tol * max(1.0, np.max(np.abs(ref)))
    # tr(U_0(x) U_2(x+mu_1)) * r(x) -> complex and real outputs
    prog = [("loadl", 0, 0, 0, 0, 0), ("loadl", 1, 0, 2, 1, +1), ("mul", 2, 0, 1), ("trace", 3, 2),
            ("load", 4, 3, 0, 0), ("mul", 3, 3, 4), ("store", 3)]
    ref = expr.as_scalar(expr.eval_program(prog, host))
    for kind, want in ((lq.LQ_COMPLEX, ref), (lq.LQ_REAL, ref.real)):
        out = lq.Field(g, kind, prec)
        lq.expr_eval(prog, [fU, fv, fz, fr], out=out)
        assert np.max(np.abs(out.download() - want)) <= tol * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
def test_field_checkpoint_roundtrip(gpu, prec, tmp_path):
    """A smeared field saved with lq_field_save and loaded into a fresh field is
    bit-identical, and smearing the loaded field continues the sequence exactly."""
    dims = (4, 4, 3, 6)
    U = fieldgen.near_identity_su3(dims, 215)
    a = upload_links(U, prec)
    lq.stout_smear(a, 0.1, 2, (0, 1, 2, 3))
    path = tmp_path / "links.lqf"
    a.save(path)
    b = lq.Field(a.geom, lq.LQ_LINKS, prec)
    b.load(path)
    assert np.array_equal(a.download(), b.download())
    lq.stout_smear(a, 0.1, 1, (0, 1, 2, 3))
    lq.stout_smear(b, 0.1, 1, (0, 1, 2, 3))
    assert np.array_equal(a.download(), b.download())
    c = lq.Field(a.geom, lq.LQ_COLOR_MATRIX, prec)
    with pytest.raises(lq.LqError) as e:
        c.load(path)
    assert e.value.status == -2
