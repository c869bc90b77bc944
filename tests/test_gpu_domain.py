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


def _whole_force(U, prec, n, dirs, seed=None):
    f = upload_links(U, prec)
    F = lq.Field(f.geom, lq.LQ_LINKS, prec)
    G = lq.Field(f.geom, lq.LQ_LINKS, prec)
    s = upload_links(seed, prec) if seed is not None else None
    lq.stout_backward(f, 0.1, n, dirs, F, grad_seed=s, beta=6.0, grad_out=G)
    return F.download(), G.download()


@pytest.mark.parametrize("prec,n,dirs,with_seed", [(lq.LQ_F64, 2, (0, 1, 2, 3), False),
                                                   (lq.LQ_F32, 3, (0, 1, 2, 3), True),
                                                   (lq.LQ_F64, 0, (0, 1, 2, 3), False)])
def test_single_rank_force_equals_whole_lattice(gpu, prec, n, dirs, with_seed):
    """domain.stout_backward on one rank (halos from its own edge slices) runs
    the kernels of lq_stout_backward step by step over the owned sites:
    force and gradient equal the whole lattice's bit for bit."""
    dims = (6, 4, 6, 8)
    U = fieldgen.near_identity_su3(dims, 713)
    seed = fieldgen.haar_su3(dims, 714) * 0.5 if with_seed else None
    F_ref, G_ref = _whole_force(U, prec, n, dirs, seed)
    slab = domain.TSlab(dims, 0, 1)
    g = slab.local_geometry()
    f = lq.Field.from_host(g, lq.LQ_LINKS, prec, slab.local_from_global(U))
    s = lq.Field.from_host(g, lq.LQ_LINKS, prec, slab.local_from_global(seed)) if with_seed else None
    F, G = lq.Field(g, lq.LQ_LINKS, prec), lq.Field(g, lq.LQ_LINKS, prec)
    domain.stout_backward(f, slab, 0.1, n, dirs, force_out=F, grad_out=G, grad_seed=s)
    assert np.array_equal(slab.owned(F.download()), F_ref)
    assert np.array_equal(slab.owned(G.download()), G_ref)


@pytest.mark.parametrize("prec_name,n,dirs,with_seed", [("f64", 2, (0, 1, 2, 3), False),
                                                        ("f32", 3, (0, 1, 2, 3), True),
                                                        ("f32", 2, (0, 1, 2), False)])
def test_two_ranks_force_equals_whole_lattice(gpu, prec_name, n, dirs, with_seed):
    """The stout force of a lattice split into two t-slabs (two processes on
    the one GPU, K's and the links' halos exchanged over gloo between the
    steps) equals lq_stout_backward of the whole lattice bit for bit."""
    dims = (8, 8, 8, 16)
    prec = lq.LQ_F64 if prec_name == "f64" else lq.LQ_F32
    U = fieldgen.near_identity_su3(dims, 715)
    seed = fieldgen.haar_su3(dims, 716) * 0.5 if with_seed else None
    F_ref, G_ref = _whole_force(U, prec, n, dirs, seed)
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=dd_workers.gpu_backward_rank,
                         args=(r, 2, port, U, seed, prec_name, 0.1, n, dirs, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    assert np.array_equal(np.concatenate([out[0][0], out[1][0]], axis=0), F_ref)
    assert np.array_equal(np.concatenate([out[0][1], out[1][1]], axis=0), G_ref)


def test_backward_step_checks_its_arguments(gpu):
    dims = (4, 4, 4, 4)
    f = upload_links(fieldgen.unit_links(dims), lq.LQ_F64)
    g = lq.Field(f.geom, lq.LQ_LINKS, lq.LQ_F64)
    k = lq.Field(f.geom, lq.LQ_LINKS, lq.LQ_F64)
    with pytest.raises(lq.LqError, match="source needs"):          # gather without K of the next step
        lq.stout_backward_step(f, lq.LQ_BWD_SOURCE_GATHER, 0.1, 0, 256, u_next=f, g_in=g, g_out=g, k_out=k)
    with pytest.raises(lq.LqError, match="alias"):
        lq.stout_backward_step(f, lq.LQ_BWD_SOURCE_WILSON, 0.1, 0, 256, u_next=f, g_out=f, k_out=k)
    with pytest.raises(lq.LqError, match="s_begin"):
        lq.stout_backward_step(f, lq.LQ_BWD_SOURCE_WILSON, 0.1, 0, 257, u_next=f, g_out=g, k_out=k)
    with pytest.raises(lq.LqError, match="k_out"):                 # a link stage needs both outputs
        lq.stout_backward_step(f, lq.LQ_BWD_SOURCE_WILSON, 0.1, 0, 256, u_next=f, k_out=k)
