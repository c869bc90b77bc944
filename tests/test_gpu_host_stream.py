"""lq_stout_smear_host (host buffers in, host buffers out, transfers
overlapped with the smearing slab by slab) against lq_field_upload +
lq_stout_smear + lq_plaquette + lq_field_download: bit-identical links and
plaquette for every slab count, including one slab, one t-slice per slab,
and slab counts that do not divide the t extent."""
import numpy as np
import pytest

import fieldgen
import paper_1105_2279_gb300 as lq
from tests.gpu_util import upload_links

pytestmark = pytest.mark.gpu
ALL, SPATIAL = (0, 1, 2, 3), (0, 1, 2)


def _reference(U, prec, rho, n, dirs):
    f = upload_links(U, prec)
    lq.stout_smear(f, rho, n, dirs)
    return f.download(), lq.plaquette(f)


def _host(U, prec):
    return np.ascontiguousarray(U.astype(np.complex64 if prec == lq.LQ_F32 else np.complex128))


@pytest.mark.parametrize("prec", [lq.LQ_F32, lq.LQ_F64])
@pytest.mark.parametrize("dims,n,dirs,chunks", [
    ((4, 4, 4, 8), 3, ALL, 0),
    ((4, 4, 4, 8), 2, ALL, 8),          # one t-slice per slab
    ((3, 4, 5, 7), 3, ALL, 3),          # 7 t-slices in 3 slabs
    ((3, 4, 5, 7), 1, SPATIAL, 4),      # t links pass through both fields
    ((4, 3, 2, 5), 2, (1, 3), 2),
    ((4, 4, 4, 2), 3, ALL, 0),          # fewer slices than the default slab count
    ((4, 4, 3, 1), 2, ALL, 1),          # one slab: its own neighbour
    ((4, 4, 4, 6), 0, ALL, 3),          # no steps: a round trip
    ((2, 3, 4, 32), 6, ALL, 0),         # 16 slabs, wavefront over 6 steps
    ((3, 2, 2, 20), 5, SPATIAL, 20),    # one t-slice per slab, odd step count
])
def test_host_stream_matches_device_path(gpu, prec, dims, n, dirs, chunks):
    U = fieldgen.near_identity_su3(dims, 700)
    ref, p_ref = _reference(U, prec, 0.125, n, dirs)
    h_in = _host(U, prec)
    h_out = np.empty_like(h_in)
    p = lq.stout_smear_host(h_in, h_out, dims, prec, 0.125, n, dirs, n_chunks=chunks)
    assert np.array_equal(h_out, ref)
    assert p == tuple(p_ref)
    assert np.array_equal(h_in, _host(U, prec))   # input untouched


@pytest.mark.parametrize("prec", [lq.LQ_F32, lq.LQ_F64])
def test_host_stream_in_place_and_pinned(gpu, prec):
    import torch
    dims = (4, 4, 6, 8)
    U = fieldgen.haar_su3(dims, 701)
    ref, p_ref = _reference(U, prec, 0.1, 2, ALL)
    h = _host(U, prec)
    pinned = torch.from_numpy(h.view(np.float32 if prec == lq.LQ_F32 else np.float64).copy()).pin_memory()
    p = lq.stout_smear_host(pinned, pinned, dims, prec, 0.1, 2, ALL, n_chunks=3)   # host_out == host_in
    got = pinned.numpy().view(h.dtype).reshape(h.shape)
    assert np.array_equal(got, ref)
    assert p == tuple(p_ref)
    h2 = h.copy()
    lq.stout_smear_host(h2, h2, dims, prec, 0.1, 2, ALL, n_chunks=5)              # pageable, in place
    assert np.array_equal(h2, ref)


def test_host_stream_rejects_bad_arguments(gpu):
    dims = (4, 4, 4, 4)
    h = _host(fieldgen.unit_links(dims), lq.LQ_F64)
    out = np.empty_like(h)
    with pytest.raises(lq.LqError):
        lq.stout_smear_host(h, out, dims, 7, 0.1, 1)                          # precision
    with pytest.raises(lq.LqError):
        lq.stout_smear_host(h, out, dims, lq.LQ_F64, -0.1, 1)                 # rho
    with pytest.raises(lq.LqError):
        lq.stout_smear_host(h, out, dims, lq.LQ_F64, 0.1, 1, dirs=())         # empty direction set
    with pytest.raises(lq.LqError):
        lq.stout_smear_host(h, out, dims, lq.LQ_F64, 0.1, 1, n_chunks=-1)
    with pytest.raises(ValueError):
        lq.stout_smear_host(h.reshape(-1)[:10], out, dims, lq.LQ_F64, 0.1, 1)  # wrong size (binding check)


@pytest.mark.parametrize("n", [3, 6, 7])
def test_host_stream_trace_respects_dependencies(gpu, tmp_path, monkeypatch, n):
    """LQ_PIPELINE_TRACE timeline: every operation is recorded once, and on the
    device clock each step-1 launch starts after its slab's and both
    neighbours' transposes ended, each step after the previous step of the
    neighbouring slabs (or the previous whole-lattice launch: with more than
    four steps, the steps between the first two and the last two run whole,
    slab -1), and each download after
    the slab's last step."""
    dims, nc = (4, 4, 4, 12), 6
    path = tmp_path / "trace.txt"
    monkeypatch.setenv("LQ_PIPELINE_TRACE", str(path))
    U = fieldgen.near_identity_su3(dims, 702)
    h = _host(U, lq.LQ_F32)
    lq.stout_smear_host(h, np.empty_like(h), dims, lq.LQ_F32, 0.1, n, ALL, n_chunks=nc)
    ops = [ln.split() for ln in path.read_text().splitlines() if not ln.startswith("end")]
    t = {}
    for what, slab, step, a, b in ops:
        t[(what, int(slab), int(step))] = (float(a), float(b))
    assert sorted({w for w, _, _ in t}) == ["d2h", "h2d", "plaq", "step", "to_aos", "to_soa"]
    whole = set(range(3, n - 1)) if n > 4 else set()
    assert len(t) == 4 * nc + (n - len(whole)) * nc + len(whole) + 1
    eps = 1e-3   # ms: event resolution

    def end_of(k, slabs):
        return max(t[("step", -1, k)][1] if k in whole else t[("step", j, k)][1] for j in slabs)

    for k in whole:
        assert t[("step", -1, k)][0] >= end_of(k - 1, range(nc)) - eps
    for i in range(nc):
        nb = ((i - 1) % nc, i, (i + 1) % nc)
        assert t[("to_soa", i, 0)][0] >= t[("h2d", i, 0)][1] - eps
        assert t[("d2h", i, n)][0] >= t[("to_aos", i, n)][1] - eps
        for j in nb:
            assert t[("step", i, 1)][0] >= t[("to_soa", j, 0)][1] - eps
        for k in range(2, n + 1):
            if k not in whole:
                assert t[("step", i, k)][0] >= end_of(k - 1, nb) - eps
        assert t[("to_aos", i, n)][0] >= t[("step", i, n)][1] - eps


@pytest.mark.parametrize("prec", [lq.LQ_F32, lq.LQ_F64])
def test_host_stream_pinned_16_slabs(gpu, prec):
    """Page-locked buffers, 16 slabs over 6 steps: bit-identical to the
    device path."""
    import torch
    dims = (2, 3, 4, 32)
    U = fieldgen.near_identity_su3(dims, 703)
    ref, p_ref = _reference(U, prec, 0.125, 6, ALL)
    h = _host(U, prec)
    fl = np.float32 if prec == lq.LQ_F32 else np.float64
    hin = torch.from_numpy(h.view(fl).copy()).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    p = lq.stout_smear_host(hin, hout, dims, prec, 0.125, 6, ALL)
    assert np.array_equal(hout.numpy().view(h.dtype).reshape(h.shape), ref)
    assert p == tuple(p_ref)
