"""The t-slab domain decomposition (paper_1105_2279_gb300.domain) on the CPU:
gloo ranks exchange halos with TSlab and smear their slabs with the oracle's
stout step; the assembled slabs equal the oracle's smearing of the whole
lattice bit for bit (the per-site arithmetic is the same), and the summed
plaquette equals the whole lattice's to rounding.  One, two and four ranks,
all four directions and the spatial ones, slabs of one to four slices."""
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import fieldgen
from oracle import gauge, stout
from tests import dd_workers


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("world,dims,n,dirs", [
    (2, (3, 4, 2, 8), 2, (0, 1, 2, 3)),
    (2, (3, 2, 3, 4), 3, (0, 1, 2)),
    (4, (2, 3, 2, 4), 2, (0, 1, 2, 3)),     # one owned slice per rank
    (1, (3, 2, 2, 5), 2, (0, 1, 2, 3)),     # a single rank: halos from its own edges
])
def test_tslab_ranks_reproduce_the_whole_lattice(world, dims, n, dirs):
    U = fieldgen.near_identity_su3(dims, 700)
    ref = stout.stout_smear(U, 0.1, n, dirs)
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=dd_workers.oracle_rank, args=(r, world, port, U, 0.1, n, dirs, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    got = np.concatenate([out[r][0] for r in range(world)], axis=0)
    assert np.array_equal(got, ref)
    V = float(np.prod(dims))
    s, t = out[0][1], out[0][2]
    assert all(out[r][1:] == (s, t) for r in range(world))
    p_ref = gauge.plaquette(ref)
    assert abs((s + t) / (18 * V) - p_ref[0]) < 1e-14
    assert abs(s / (9 * V) - p_ref[1]) < 1e-14 and abs(t / (9 * V) - p_ref[2]) < 1e-14


def test_tslab_rejects_uneven_split():
    from paper_1105_2279_gb300.domain import TSlab
    with pytest.raises(ValueError):
        TSlab((4, 4, 4, 6), 0, 4)
    s = TSlab((4, 4, 4, 8), 1, 2)
    assert s.local_dims == (4, 4, 4, 6) and s.t0 == 4 and s.interior == (64, 320)


@pytest.mark.parametrize("world,dims,n,dirs,with_seed", [
    (2, (3, 2, 2, 6), 2, (0, 1, 2, 3), False),
    (2, (2, 3, 2, 4), 1, (0, 1, 2), True),
    (4, (2, 2, 2, 4), 2, (0, 1, 2, 3), False),    # one owned slice per rank
    (1, (2, 3, 2, 3), 0, (0, 1, 2, 3), False),    # n = 0: the Wilson force itself
])
def test_tslab_force_reproduces_the_oracle(world, dims, n, dirs, with_seed):
    """domain.stout_backward on gloo ranks, its library calls replaced by
    host steps in gather form built from the oracle's reverse-mode pieces:
    the ranks' halo exchanges of the links and of K between the backward
    steps, the sources and the last step assemble the oracle's whole-lattice
    force and gradient to rounding (the gather sums the staple terms in
    another order than the oracle's scatter)."""
    from oracle import backward, gauge
    U = fieldgen.near_identity_su3(dims, 720)
    seed = fieldgen.haar_su3(dims, 721) * 0.5 if with_seed else None
    if with_seed:
        G_ref = backward.stout_backward(U, 0.1, n, dirs, seed)
        F_ref = gauge.force_from_grad(G_ref, U)
    else:
        F_ref, G_ref = backward.smeared_wilson_force(U, 0.1, n, dirs, 6.0)
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=dd_workers.oracle_backward_rank, args=(r, world, port, U, seed, 0.1, n, dirs, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    F = np.concatenate([out[r][0] for r in range(world)], axis=0)
    G = np.concatenate([out[r][1] for r in range(world)], axis=0)
    assert np.max(np.abs(F - F_ref)) <= 1e-13 * np.max(np.abs(F_ref))
    assert np.max(np.abs(G - G_ref)) <= 1e-13 * np.max(np.abs(G_ref))


def test_tslab_force_rejects_bad_arguments():
    import types

    from paper_1105_2279_gb300 import domain
    slab = domain.TSlab((2, 2, 2, 4), 0, 1)
    f = types.SimpleNamespace(geom=slab.local_dims, prec=None, tensor=None)
    with pytest.raises(ValueError, match="force_out"):
        domain.stout_backward(f, slab, 0.1, 1)
    with pytest.raises(ValueError, match="n_steps"):
        domain.stout_backward(f, slab, 0.1, -1, force_out=f)
