"""The t-slab domain decomposition on the GPU: each rank smears its slab with
lq_stout_step_range after a halo exchange, and the assembled result equals
lq_stout_smear of the whole lattice bit for bit (the same kernel and
arithmetic per link); the plaquette from the ranks' summed lq_plaquette_sums
equals lq_plaquette to 1e-14.  Two ranks run as two processes on the one
GPU with a host-staged gloo exchange, so no kernel ever waits on another
rank; a single rank fills its halos from its own edge slices."""
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import fieldgen
import paper_1105_2279_gb300 as lq
from paper_1105_2279_gb300 import domain
from tests import dd_workers
from tests.gpu_util import upload_links

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _whole(U, prec, n, dirs):
    f = upload_links(U, prec)
    lq.stout_smear(f, 0.1, n, dirs)
    return f.download(), lq.plaquette(f)


@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
def test_single_rank_slab_equals_whole_lattice(gpu, prec):
    dims = (8, 8, 8, 16)
    U = fieldgen.near_identity_su3(dims, 710)
    ref, p_ref = _whole(U, prec, 3, (0, 1, 2, 3))
    slab = domain.TSlab(dims, 0, 1)
    f = lq.Field.from_host(slab.local_geometry(), lq.LQ_LINKS, prec, slab.local_from_global(U))
    domain.stout_smear(f, slab, 0.1, 3, (0, 1, 2, 3))
    assert np.array_equal(slab.owned(f.download()), ref)
    p = domain.plaquette(f, slab)
    assert max(abs(a - b) for a, b in zip(p, p_ref)) < 1e-14


@pytest.mark.parametrize("prec_name,n,dirs", [("f64", 3, (0, 1, 2, 3)), ("f32", 4, (0, 1, 2, 3)),
                                              ("f32", 3, (0, 1, 2))])
def test_two_ranks_equal_whole_lattice(gpu, prec_name, n, dirs):
    dims = (8, 8, 8, 16)
    prec = lq.LQ_F64 if prec_name == "f64" else lq.LQ_F32
    U = fieldgen.near_identity_su3(dims, 711)
    ref, p_ref = _whole(U, prec, n, dirs)
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=dd_workers.gpu_rank, args=(r, 2, port, U, prec_name, 0.1, n, dirs, out))
             for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    got = np.concatenate([out[0][0], out[1][0]], axis=0)
    assert np.array_equal(got, ref)
    for r in range(2):
        assert max(abs(a - b) for a, b in zip(out[r][1], p_ref)) < 1e-14


def test_step_range_leaves_other_sites_untouched(gpu):
    """lq_stout_step_range writes only the requested sites and directions."""
    import torch
    dims = (4, 4, 4, 6)
    U = fieldgen.near_identity_su3(dims, 712)
    a = upload_links(U, lq.LQ_F64)
    full = upload_links(U, lq.LQ_F64)
    lq.stout_smear(full, 0.1, 1, (0, 2))
    out = lq.Field(a.geom, lq.LQ_LINKS, lq.LQ_F64)
    out.tensor.fill_(7.0)
    v3 = 64
    lq.stout_step_range(a, out, 0.1, 2 * v3, 4 * v3, (0, 2))
    o, f = out.tensor, full.tensor
    for mu in range(4):
        if mu in (0, 2):
            assert torch.equal(o[mu, :, 2 * v3:4 * v3], f[mu, :, 2 * v3:4 * v3])
        else:
            assert bool((o[mu, :, 2 * v3:4 * v3] == 7.0).all())
        assert bool((o[mu, :, :2 * v3] == 7.0).all()) and bool((o[mu, :, 4 * v3:] == 7.0).all())
    with pytest.raises(lq.LqError):
        lq.stout_step_range(a, out, 0.1, 3 * v3, 2 * v3, (0, 2))
    with pytest.raises(lq.LqError):
        lq.stout_step_range(a, a, 0.1, 0, v3, (0, 2))
