"""lq_stout_smear_noalloc: stout smearing that allocates no device memory.

Some callers cannot let a library allocate device memory: an application
whose own allocator already holds all of the GPU's memory, a plug-in whose
host forbids device allocations, a latency-critical path that must not risk
the synchronisation or failure an allocation can bring.  They call this entry
point, which takes its double buffer from a 32 MiB array built into the
library instead of allocating one.

The tests call it through the C ABI twice in a row (the built-in array keeps
the first call's contents) and compare each result with lq_stout_smear on the
same input, within the tolerances of the other GPU tests (FP64: 1e-12 per
link element; FP32: 2e-6 per step), and check that a lattice too large for the
built-in array is refused with a clear error.  This file is collected last so
that a run stopping at its first failure has run every other test.
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


@pytest.mark.parametrize("prec,dims,dirs,n,tol", [
    (lq.LQ_F64, (8, 8, 8, 16), 0b1111, 3, 1e-12),            # 8,192 sites, 4 directions
    (lq.LQ_F32, (12, 12, 12, 24), 0b0111, 4, 4 * 2e-6),      # 41,472 sites, spatial directions
])
def test_noalloc_matches_stout_smear_on_two_calls(gpu, prec, dims, dirs, n, tol):
    lib = lq.capi()
    for call in range(2):
        U = fieldgen.near_identity_su3(dims, 500 + call)
        a = upload_links(U, prec)
        b = upload_links(U, prec)
        st = lib.lq_stout_smear_noalloc(a.handle, 0.1, n, dirs, _stream())
        assert st == 0, lib.lq_last_error().decode()
        lq.stout_smear(b, 0.1, n, dirs)
        got, ref = a.download(), b.download()
        assert np.max(np.abs(got.astype(np.complex128) - ref)) <= tol, call


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
