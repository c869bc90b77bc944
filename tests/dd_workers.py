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
