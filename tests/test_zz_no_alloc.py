"""lq_stout_smear_noalloc: stout smearing that allocates no device memory.

Some callers cannot let a library allocate device memory: an application
whose own allocator already holds all of the GPU's memory, a plug-in whose
host forbids device allocations, a latency-critical path that must not risk
the synchronisation or failure an allocation can bring.  They call this entry
point, which takes its double buffer from a 32 MiB array built into the
library instead of allocating one.

The tests call it through the C ABI twice in a row (the built-in array keeps
the first call's contents) and compare each result with lq_stout_smear on the
same input bit for bit: both run the same step kernels with the same launch
shape, so any difference would come from the shared array (stale
pass-through directions, a missed copy-back).  One case smears an odd number
of steps over a subset of the directions right after a call that left other
data in the array, the path that copies only the smeared directions back.
A lattice too large for the built-in array is refused with a clear error.
This file is collected last so that a run stopping at its first failure has
run every other test.
"""
import ctypes

import numpy as np
import pytest

import fieldgen
import paper_1105_2279_gb300 as lq
from tests.gpu_util import upload_links

pytestmark = pytest.mark.gpu


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _noalloc_vs_stout_smear(lib, U, prec, dirs, n):
    a = upload_links(U, prec)
    b = upload_links(U, prec)
    st = lib.lq_stout_smear_noalloc(a.handle, 0.1, n, dirs, _stream())
    assert st == 0, lib.lq_last_error().decode()
    lq.stout_smear(b, 0.1, n, dirs)
    return a.download(), b.download()


@pytest.mark.parametrize("prec,dims,dirs,n", [
    (lq.LQ_F64, (8, 8, 8, 16), 0b1111, 3),            # 8,192 sites, 4 directions
    (lq.LQ_F32, (12, 12, 12, 24), 0b0111, 4),         # 41,472 sites, spatial directions
    (lq.LQ_F32, (12, 12, 12, 24), 0b0111, 3),         # odd n: smeared directions copied back
])
def test_noalloc_matches_stout_smear_on_two_calls(gpu, prec, dims, dirs, n):
    lib = lq.capi()
    for call in range(2):
        U = fieldgen.near_identity_su3(dims, 500 + call)
        got, ref = _noalloc_vs_stout_smear(lib, U, prec, dirs, n)
        assert np.array_equal(got, ref), call


def test_noalloc_after_other_contents(gpu):
    """An FP64 call on another lattice over all four directions fills the
    array with other data; the FP32 call after it (3 steps, spatial
    directions) must not see any of it."""
    lib = lq.capi()
    _noalloc_vs_stout_smear(lib, fieldgen.haar_su3((8, 8, 8, 8), 510), lq.LQ_F64, 0b1111, 2)
    U = fieldgen.near_identity_su3((10, 12, 14, 16), 511)
    got, ref = _noalloc_vs_stout_smear(lib, U, lq.LQ_F32, 0b0111, 3)
    assert np.array_equal(got, ref)
    assert np.array_equal(got[..., 3, :, :], U[..., 3, :, :].astype(np.complex64))   # t links untouched


def test_noalloc_refuses_lattice_larger_than_its_buffer(gpu):
    import torch
    lib = lq.capi()
    dims = (16, 16, 16, 16)                       # 65,536 sites: 37.7 MB as FP64 links
    g = lq.Geometry(dims)
    t = torch.zeros((4, 9, g.volume, 2), dtype=torch.float64, device="cuda")
    f = lq.Field(g, lq.LQ_LINKS, lq.LQ_F64, tensor=t)
    st = lib.lq_stout_smear_noalloc(f.handle, 0.1, 1, 0b1111, _stream())
    assert st == -1
    assert b"built-in workspace" in lib.lq_last_error()
    assert torch.count_nonzero(t).item() == 0     # nothing was launched
