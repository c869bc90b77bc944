"""The C-ABI library loads, exports every entry point include/lqcd.h declares,
and validates arguments on the host (no device work is launched here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "lqcd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lq_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lqlib):
    lib = lqlib.capi()
    names = header_functions()
    assert len(names) >= 24
    for n in names:
        assert hasattr(lib, n), n


def test_binding_declares_every_symbol(lqlib):
    from paper_1105_2279_gb300 import _lib
    assert set(header_functions()) == set(_lib.SIGNATURES)


def test_abi_version_and_geometry(lqlib):
    lib = lqlib.capi()
    assert lib.lq_abi_version() == 1
    g = lqlib.Geometry((3, 4, 5, 6))
    dims, vol = lqlib.geom_info(g)
    assert dims == (3, 4, 5, 6) and vol == 360
    assert lqlib.field_bytes(g, lqlib.LQ_LINKS, lqlib.LQ_F64) == 360 * 36 * 16
    assert lqlib.field_bytes(g, lqlib.LQ_REAL, lqlib.LQ_F32) == 360 * 4
    assert lqlib.field_bytes(g, lqlib.LQ_COLOR_VECTOR, lqlib.LQ_F32) == 360 * 3 * 8


@pytest.mark.parametrize("dims", [(0, 4, 4, 4), (4, -1, 4, 4), (2048, 2048, 1024, 1)])
def test_bad_geometry_rejected(lqlib, dims):
    with pytest.raises(lqlib.LqError) as e:
        lqlib.Geometry(dims)
    assert e.value.status == -1
    assert "lq_geom_create" in str(e.value)


def test_wrap_validation(lqlib):
    lib = lqlib.capi()
    g = lqlib.Geometry((2, 2, 2, 2))
    h = ctypes.c_void_p()
    need = lqlib.field_bytes(g, lqlib.LQ_LINKS, lqlib.LQ_F64)
    # misaligned pointer, too few bytes, bad kind
    assert lib.lq_field_wrap(g.handle, 0, 1, ctypes.c_void_p(0x1008), need, ctypes.byref(h)) == -1
    assert b"aligned" in lib.lq_last_error()
    assert lib.lq_field_wrap(g.handle, 0, 1, ctypes.c_void_p(0x1000), need - 1, ctypes.byref(h)) == -1
    assert lib.lq_field_wrap(g.handle, 9, 1, ctypes.c_void_p(0x1000), need, ctypes.byref(h)) == -1
    assert lib.lq_field_wrap(g.handle, 0, 1, ctypes.c_void_p(0x1000), need, ctypes.byref(h)) == 0
    f = h
    # stout argument checks happen before any device work
    assert lib.lq_stout_smear(f, 0.1, 1, 0, None, None) == -1
    assert lib.lq_stout_smear(f, 0.1, 1, 16, None, None) == -1
    assert lib.lq_stout_smear(f, -0.1, 1, 15, None, None) == -1
    assert lib.lq_stout_smear(f, float("nan"), 1, 15, None, None) == -1
    assert lib.lq_stout_smear(f, 0.1, -1, 15, None, None) == -1
    assert lib.lq_stout_smear(f, 0.1, 0, 15, None, None) == 0      # zero steps: nothing to do
    assert lib.lq_stout_smear(None, 0.1, 1, 15, None, None) == -1
    # shift of a field onto itself, bad direction
    assert lib.lq_shift(f, f, 0, 1, None) == -1
    assert lib.lq_shift(f, f, 4, 1, None) == -1
    assert lib.lq_plaquette(None, None, None) == -1
    assert lib.lq_field_free(f) == 0


def test_kind_mismatch_is_geom_error(lqlib):
    lib = lqlib.capi()
    g = lqlib.Geometry((2, 2, 2, 2))
    h = ctypes.c_void_p()
    assert lib.lq_field_wrap(g.handle, 1, 1, ctypes.c_void_p(0x1000), 1 << 20, ctypes.byref(h)) == 0
    assert lib.lq_stout_smear(h, 0.1, 1, 15, None, None) == -2
    out = (ctypes.c_double * 3)()
    assert lib.lq_plaquette(h, out, None) == -2
    lib.lq_field_free(h)


def test_expr_program_validation(lqlib):
    lib = lqlib.capi()
    g = lqlib.Geometry((2, 2, 2, 2))
    h = ctypes.c_void_p()
    assert lib.lq_field_wrap(g.handle, 0, 1, ctypes.c_void_p(0x1000), 1 << 20, ctypes.byref(h)) == 0
    red = (ctypes.c_double * 2)()
    ops = (ctypes.c_void_p * 1)(h)
    # program without a final STORE, register out of range, operand out of range
    for prog in ([("loadl", 0, 0, 0, 0, 0)],
                 [("loadl", 9, 0, 0, 0, 0), ("store", 9)],
                 [("loadl", 0, 3, 0, 0, 0), ("store", 0)],
                 [("loadl", 0, 0, 5, 0, 0), ("store", 0)]):
        arr, n = lqlib.compile_program(prog)
        assert lib.lq_expr_eval(None, arr, n, ops, 1, red, None) == -1
    lib.lq_field_free(h)


def test_injected_allocation_failure_is_reported(lqlib, monkeypatch):
    """LQ_FAULT_INJECT=alloc makes the library's scratch allocations fail on the
    host: calls return LQ_ERR_OOM with a message and launch nothing (the fake
    device pointer below is never dereferenced)."""
    lib = lqlib.capi()
    g = lqlib.Geometry((4, 4, 4, 4))
    h = ctypes.c_void_p()
    need = lqlib.field_bytes(g, lqlib.LQ_LINKS, lqlib.LQ_F64)
    assert lib.lq_field_wrap(g.handle, 0, 1, ctypes.c_void_p(0x1000), need, ctypes.byref(h)) == 0
    monkeypatch.setenv("LQ_FAULT_INJECT", "alloc")
    assert lib.lq_stout_smear(h, 0.1, 2, 15, None, None) == -3
    assert b"fault injected" in lib.lq_last_error()
    out = (ctypes.c_double * 3)()
    assert lib.lq_plaquette(h, out, None) == -3
    assert lib.lq_stout_backward(h, 0.1, 1, 15, None, 6.0, h, None, None, None) in (-1, -3)
    # the APE and HYP smearings and forces allocate their scratch before any launch
    f = ctypes.c_void_p()
    assert lib.lq_field_wrap(g.handle, 0, 1, ctypes.c_void_p(0x2000), need, ctypes.byref(f)) == 0
    assert lib.lq_ape_smear(h, 0.5, 1, 15, None) == -3
    assert lib.lq_hyp_smear(h, 0.75, 0.6, 0.3, 1, None) == -3
    for call in (lambda: lib.lq_stout_backward(h, 0.1, 1, 15, None, 6.0, f, None, None, None),
                 lambda: lib.lq_ape_backward(h, 0.6, 1, 15, None, 6.0, f, None, None, None),
                 lambda: lib.lq_hyp_backward(h, 0.75, 0.6, 0.3, 1, None, 6.0, f, None, None, None)):
        assert call() == -3
        assert b"fault injected" in lib.lq_last_error()
    monkeypatch.delenv("LQ_FAULT_INJECT")
    lib.lq_field_free(f)
    lib.lq_field_free(h)


def test_jit_compiles_and_caches_without_a_gpu(lqlib, tmp_path):
    """lq_expr_jit_prepare generates and NVRTC-compiles a program's kernel on the
    host (no device needed); the second request hits the in-memory cache; after
    lq_free_all drops that cache, the cubin comes back from the disk cache."""
    lib = lqlib.capi()
    g = lqlib.Geometry((4, 3, 4, 5))
    h = ctypes.c_void_p()
    assert lib.lq_field_wrap(g.handle, 0, 0, ctypes.c_void_p(0x1000), 1 << 26, ctypes.byref(h)) == 0

    class _F:
        handle = h
    prog = [("loadl", 0, 0, 3, 0, 0), ("loadl", 1, 0, 0, 3, -1), ("mul", 2, 0, 1), ("trace", 3, 2),
            ("scale", 3, 3, 0.375, -1.25), ("store", 3)]
    lqlib.jit_cache_dir(str(tmp_path))
    c0 = lqlib.jit_stats()
    lqlib.expr_jit_prepare(prog, [_F], reduce=True)
    c1 = lqlib.jit_stats()
    assert c1[0] == c0[0] + 1
    lqlib.expr_jit_prepare(prog, [_F], reduce=True)
    assert lqlib.jit_stats()[1] == c1[1] + 1
    assert any(p.suffix == ".cubin" for p in tmp_path.iterdir())
    lqlib.free_all()
    lqlib.expr_jit_prepare(prog, [_F], reduce=True)
    c3 = lqlib.jit_stats()
    assert c3[2] == c1[2] + 1 and c3[0] == c1[0]
    lqlib.jit_cache_dir(None)
    # malformed programs are refused before any code generation
    bad, n = lqlib.compile_program([("loadl", 0, 0, 9, 0, 0), ("store", 0)])
    ops = (ctypes.c_void_p * 1)(h)
    assert lib.lq_expr_jit_prepare(None, bad, n, ops, 1, 1) == -1
    lib.lq_field_free(h)


def test_tuner_cache_file_is_read_back(lqlib, tmp_path):
    """lq_tune(path) loads a cache written earlier; lq_tune_lookup returns the
    stored launch shape for its key (kernel, device, precision, dims, dirs).
    Without a device the device name reads 'unknown'.  Runs in a child process
    because lq_tune switches the tuner on for the whole process."""
    import subprocess
    import sys
    path = tmp_path / "tune.txt"
    path.write_text("stout unknown 1 4 4 4 8 15 64 2 1\nstout unknown 0 6 6 6 12 7 256 8 2\n")
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import paper_1105_2279_gb300 as lq\n"
        "lq.tune(%r)\n"
        "assert lq.tune_lookup(lq.LQ_F64, (4, 4, 4, 8), 15) == (64, 2, 1)\n"
        "assert lq.tune_lookup(lq.LQ_F32, (6, 6, 6, 12), (0, 1, 2)) == (256, 8, 2)\n"
        "assert lq.tune_lookup(lq.LQ_F32, (4, 4, 4, 8), 15) is None\n"
        "print('ok')\n" % (ROOT, str(path)))
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120, env=env)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr


def test_field_checkpoint_header_checks(lqlib, tmp_path):
    """lq_field_load validates the file before touching the device: a foreign
    file is LQ_ERR_ARG, a checkpoint of another geometry / kind is LQ_ERR_GEOM."""
    import struct
    lib = lqlib.capi()
    g = lqlib.Geometry((2, 2, 2, 4))
    h = ctypes.c_void_p()
    need = lqlib.field_bytes(g, lqlib.LQ_LINKS, lqlib.LQ_F64)
    assert lib.lq_field_wrap(g.handle, 0, 1, ctypes.c_void_p(0x1000), need, ctypes.byref(h)) == 0
    junk = tmp_path / "junk.bin"
    junk.write_bytes(b"not a field" * 10)
    assert lib.lq_field_load(h, str(junk).encode(), None) == -1
    other = tmp_path / "other.lqf"
    hdr = b"LQFIELD1" + struct.pack("<iii4iiq", 1, 0, 1, 2, 2, 2, 2, 0, need // 2)
    assert len(hdr) == 48
    other.write_bytes(hdr + bytes(need // 2))
    assert lib.lq_field_load(h, str(other).encode(), None) == -2
    assert b"differs" in lib.lq_last_error()
    assert lib.lq_field_load(h, str(tmp_path / "missing.lqf").encode(), None) == -1
    lib.lq_field_free(h)


def test_jacobi_launch_shape_checked_before_device_work(lqlib):
    """A thread geometry outside the tuner's range is refused with LQ_ERR_ARG
    before any CUDA call (the fields point at unmapped addresses), and the
    options struct of the previous, smaller layout is still accepted."""
    from paper_1105_2279_gb300 import LqJacobiOpts
    lib = lqlib.capi()
    g = lqlib.Geometry((2, 2, 2, 2))
    U, v = ctypes.c_void_p(), ctypes.c_void_p()
    nU = lqlib.field_bytes(g, lqlib.LQ_LINKS, lqlib.LQ_F32)
    nv = lqlib.field_bytes(g, lqlib.LQ_COLOR_VECTOR, lqlib.LQ_F32)
    assert lib.lq_field_wrap(g.handle, lqlib.LQ_LINKS, lqlib.LQ_F32, ctypes.c_void_p(0x1000), nU, ctypes.byref(U)) == 0
    assert lib.lq_field_wrap(g.handle, lqlib.LQ_COLOR_VECTOR, lqlib.LQ_F32, ctypes.c_void_p(0x100000), nv,
                             ctypes.byref(v)) == 0
    for block, nsite in ((48, 1), (512, 1), (-32, 1), (64, -1), (64, 65)):
        o = LqJacobiOpts(ctypes.sizeof(LqJacobiOpts), 0, block, nsite)
        assert lib.lq_jacobi_smear_ex(U, v, 0.1, 1, 1.0, 15, ctypes.byref(o), None) == -1, (block, nsite)
        assert b"block" in lib.lq_last_error()
    o = LqJacobiOpts(4, 0, 0, 0)       # struct_size below the first option
    assert lib.lq_jacobi_smear_ex(U, v, 0.1, 1, 1.0, 15, ctypes.byref(o), None) == -1
    assert lib.lq_field_free(U) == 0 and lib.lq_field_free(v) == 0


def test_backward_step_arguments_checked_before_device_work(lqlib):
    """lq_stout_backward_step refuses, before any CUDA call (the fields point
    at unmapped addresses), a gather without K of the next step, a link stage
    without both outputs, an output that aliases an input, a site range past
    the volume, an unknown source and fields of another geometry."""
    lib = lqlib.capi()
    g = lqlib.Geometry((2, 2, 2, 2))
    g2 = lqlib.Geometry((2, 2, 2, 4))

    def wrap(geom, addr):
        h = ctypes.c_void_p()
        nb = lqlib.field_bytes(geom, lqlib.LQ_LINKS, lqlib.LQ_F64)
        assert lib.lq_field_wrap(geom.handle, lqlib.LQ_LINKS, lqlib.LQ_F64, ctypes.c_void_p(addr), nb,
                                 ctypes.byref(h)) == 0
        return h
    u, kn, gi, go, ko, other = (wrap(g, 0x100000 * (i + 1)) for i in range(6))
    far = wrap(g2, 0x1000000)
    V = 16
    W, GIVEN, GATHER = lqlib.LQ_BWD_SOURCE_WILSON, lqlib.LQ_BWD_SOURCE_GIVEN, lqlib.LQ_BWD_SOURCE_GATHER
    cases = [
        ((u, None, gi, u, go, ko, None, GATHER, 0, V), b"source needs"),
        ((None, None, None, u, go, ko, None, GIVEN, 0, V), b"source needs"),
        ((u, None, None, u, None, ko, None, W, 0, V), b"k_out"),
        ((u, None, None, u, go, ko, other, W, 0, V), b"k_out"),
        ((u, None, None, u, u, ko, None, W, 0, V), b"alias"),
        ((u, None, None, u, go, go, None, W, 0, V), b"alias"),
        ((u, None, None, u, go, ko, None, W, 0, V + 1), b"s_begin"),
        ((u, None, None, u, go, ko, None, W, 5, 4), b"s_begin"),
        ((u, None, None, u, go, ko, None, 7, 0, V), b"source must"),
        ((far, None, None, u, go, ko, None, W, 0, V), b"geometry"),
    ]
    for (un, kk, gg, uc, g_o, k_o, f_o, src, s0, s1), msg in cases:
        st = lib.lq_stout_backward_step(un, kk, gg, uc, g_o, k_o, f_o, src, 0.1, 6.0, 15, s0, s1, None)
        assert st < 0, msg
        assert msg in lib.lq_last_error(), (msg, lib.lq_last_error())
    for h in (u, kn, gi, go, ko, other, far):
        assert lib.lq_field_free(h) == 0
