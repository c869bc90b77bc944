"""Rank bodies of the domain-decomposition tests, run in spawned processes
(importable without torch's CUDA state or the built library)."""
import os


def tensor_from_aos(U):
    """Host AoS links (Lt, Lz, Ly, Lx, 4, 3, 3) -> CPU tensor [dir][comp][site](re, im), float64."""
    import numpy as np
    import torch
    V = int(np.prod(U.shape[:4]))
    a = U.reshape(V, 4, 9).transpose(1, 2, 0)
    return torch.from_numpy(np.ascontiguousarray(np.stack([a.real, a.imag], axis=-1)))


def aos_from_tensor(t, dims):
    lx, ly, lz, lt = dims
    a = t[..., 0].numpy() + 1j * t[..., 1].numpy()          # [dir][comp][site]
    return a.transpose(2, 0, 1).reshape(lt, lz, ly, lx, 4, 3, 3)


def oracle_rank(rank, world, port, U, rho, n, dirs, out):
    """One rank of a t-split lattice on the CPU: TSlab's halo exchange over
    gloo, the oracle's stout step on the local lattice (halos included) with
    the owned slices kept, then the plaquette sums of the owned sites."""
    import types

    import numpy as np
    import torch
    import torch.distributed as dist

    from oracle import gauge, stout
    from paper_1105_2279_gb300.domain import TSlab
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lt, lz, ly, lx = U.shape[:4]
    slab = TSlab((lx, ly, lz, lt), rank, world)
    f = types.SimpleNamespace(tensor=tensor_from_aos(slab.local_from_global(U)))
    lo, hi = slab.interior
    for _ in range(n):
        slab.exchange(f)
        new = stout.stout_step(aos_from_tensor(f.tensor, slab.local_dims), rho, dirs)
        f.tensor[:, :, lo:hi] = tensor_from_aos(new)[:, :, lo:hi]
    slab.exchange(f)
    loc = aos_from_tensor(f.tensor, slab.local_dims)
    sums = torch.zeros(2, dtype=torch.float64)
    for mu in range(3):
        for nu in range(mu + 1, 4):
            sums[0 if nu < 3 else 1] += float(np.sum(gauge.plaquette_field(loc, mu, nu)[1:slab.nt + 1]))
    dist.all_reduce(sums)
    out[rank] = (slab.owned(loc), float(sums[0]), float(sums[1]))
    dist.destroy_process_group()


def gpu_rank(rank, world, port, U, prec_name, rho, n, dirs, out):
    """One rank of a t-split lattice on cuda:0 (all ranks share the GPU; the
    halo exchange is host-staged over gloo, so no kernel waits on another
    rank): paper_1105_2279_gb300.domain's smearing and plaquette."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1105_2279_gb300 as lq
    from paper_1105_2279_gb300 import domain
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    prec = lq.LQ_F64 if prec_name == "f64" else lq.LQ_F32
    lt, lz, ly, lx = U.shape[:4]
    slab = domain.TSlab((lx, ly, lz, lt), rank, world)
    f = lq.Field.from_host(slab.local_geometry(), lq.LQ_LINKS, prec, slab.local_from_global(U))
    domain.stout_smear(f, slab, rho, n, dirs)
    plaq = domain.plaquette(f, slab)
    out[rank] = (np.ascontiguousarray(slab.owned(f.download())), plaq)
    dist.destroy_process_group()


def gpu_backward_rank(rank, world, port, U, seed, prec_name, rho, n, dirs, out):
    """One rank of the t-split stout force on cuda:0 (host-staged gloo halo
    exchanges between the steps): paper_1105_2279_gb300.domain.stout_backward."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1105_2279_gb300 as lq
    from paper_1105_2279_gb300 import domain
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    prec = lq.LQ_F64 if prec_name == "f64" else lq.LQ_F32
    lt, lz, ly, lx = U.shape[:4]
    slab = domain.TSlab((lx, ly, lz, lt), rank, world)
    g = slab.local_geometry()
    f = lq.Field.from_host(g, lq.LQ_LINKS, prec, slab.local_from_global(U))
    s = lq.Field.from_host(g, lq.LQ_LINKS, prec, slab.local_from_global(seed)) if seed is not None else None
    F, G = lq.Field(g, lq.LQ_LINKS, prec), lq.Field(g, lq.LQ_LINKS, prec)
    domain.stout_backward(f, slab, rho, n, dirs, force_out=F, grad_out=G, grad_seed=s, beta=6.0)
    out[rank] = (np.ascontiguousarray(slab.owned(F.download())), np.ascontiguousarray(slab.owned(G.download())))
    dist.destroy_process_group()


class _HostField:
    """A stand-in for paper_1105_2279_gb300.Field on the CPU: a float64 tensor
    [dir][comp][site](re, im) of the local lattice `geom` (its dims)."""

    def __init__(self, geom, kind=None, prec=None, tensor=None):
        import numpy as np
        import torch
        self.geom, self.prec = geom, prec
        V = int(np.prod(geom))
        self.tensor = tensor if tensor is not None else torch.zeros((4, 9, V, 2), dtype=torch.float64)


def _host_step_range(inp, out, rho, s0, s1, dirs, stream=None, **opts):
    """lq_stout_step_range with the oracle's step: the links of `dirs` on the sites [s0, s1)."""
    from oracle import stout
    new = tensor_from_aos(stout.stout_step(aos_from_tensor(inp.tensor, inp.geom), rho, dirs))
    for mu in dirs:
        out.tensor[mu, :, s0:s1] = new[mu, :, s0:s1]


def _host_backward_step(u_cur, source, rho, s0, s1, dirs, u_next=None, k_next=None, g_in=None, g_out=None,
                        k_out=None, force_out=None, beta=6.0, stream=None):
    """lq_stout_backward_step in gather form, built from the oracle's reverse-mode
    pieces (the staple vjp, the exponential's Frechet derivative): G' from the
    source, then the link stage (G_U(local), K) or the last step (G', force)."""
    from oracle import backward, gauge, stout
    from oracle.expm import expm_frechet, expm_series
    from oracle.su3 import adj, ta
    dims = u_cur.geom

    def aos(f):
        return aos_from_tensor(f.tensor, dims)
    if source == 0:       # Wilson action of u_next
        Gp = gauge.wilson_action_grad(aos(u_next), beta)
    else:
        Gp = aos(g_in).copy()
        if source == 2:   # plus the staple-insertion terms of K of the step after
            acc = 0.0 * Gp
            Un, K = aos(u_next), aos(k_next)
            for mu in dirs:
                backward.staple_vjp(Un, mu, dirs, K[..., mu, :, :], acc)
            for a in dirs:
                Gp[..., a, :, :] += acc[..., a, :, :]

    def put(f, A, which):
        t = tensor_from_aos(A)
        for a in which:
            f.tensor[a, :, s0:s1] = t[a, :, s0:s1]
    if k_out is not None:
        Uc = aos(u_cur)
        Gout, Kout = Gp.copy(), 0.0 * Gp
        for a in dirs:
            Ua = Uc[..., a, :, :]
            C = rho * stout.staple_sum(Uc, a, dirs)
            X = ta(C @ adj(Ua))
            G_Om = ta(expm_frechet(adj(X), Gp[..., a, :, :] @ adj(Ua)))
            Gout[..., a, :, :] = adj(expm_series(X)) @ Gp[..., a, :, :] + adj(G_Om) @ C
            Kout[..., a, :, :] = rho * (G_Om @ Ua)
        put(g_out, Gout, range(4))
        put(k_out, Kout, dirs)
    else:
        if g_out is not None:
            put(g_out, Gp, range(4))
        if force_out is not None:
            put(force_out, gauge.force_from_grad(Gp, aos(u_cur)), range(4))


def oracle_backward_rank(rank, world, port, U, seed, rho, n, dirs, out):
    """One rank of the t-split stout force on the CPU: domain.stout_backward's
    own step sequence and halo exchanges (gloo), with the library calls
    replaced by the oracle-based host steps above."""
    import numpy as np
    import torch.distributed as dist

    from paper_1105_2279_gb300 import domain
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    domain.Field = _HostField
    domain.stout_step_range = _host_step_range
    domain.stout_backward_step = _host_backward_step
    lt, lz, ly, lx = U.shape[:4]
    slab = domain.TSlab((lx, ly, lz, lt), rank, world)
    g = slab.local_dims
    f = _HostField(g, tensor=tensor_from_aos(slab.local_from_global(U)))
    s = _HostField(g, tensor=tensor_from_aos(slab.local_from_global(seed))) if seed is not None else None
    F, G = _HostField(g), _HostField(g)
    domain.stout_backward(f, slab, rho, n, dirs, force_out=F, grad_out=G, grad_seed=s, beta=6.0)
    out[rank] = (np.ascontiguousarray(slab.owned(aos_from_tensor(F.tensor, g))),
                 np.ascontiguousarray(slab.owned(aos_from_tensor(G.tensor, g))))
    dist.destroy_process_group()
