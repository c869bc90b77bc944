"""Stout smearing of one lattice split over ranks (Winter, "Accelerating
QDP++ using GPUs", Sec. 8, names parallelisation over several GPUs as the
next step; here along t, one slab of t-slices per rank).

Rank r of P owns the global t-slices [r T, (r+1) T), T = Lt / P, and holds
them in a LINKS field of the local lattice (Lx, Ly, Lz, T + 2): local slice
0 is a copy of global slice r T - 1 (the lower halo), slices 1..T the owned
ones, slice T + 1 a copy of global slice (r+1) T (the upper halo), all
periodic in t.  A stout step reads neighbours at most one slice away (the
staples of U_mu(x) use x +- nu, x + mu and x + mu - nu), so after a halo
exchange lq_stout_step_range smears the owned slices exactly as the
single-lattice step does, bit for bit; a split along t alone needs no edge
exchange, since a halo slice carries all four link directions.  The
plaquette of the owned sites reads the upper halo; the ranks add their two
FP64 sums with one all-reduce.

The exchange is the only communication: per step, each rank sends its first
owned slice to rank r - 1 (its upper halo) and its last owned slice to rank
r + 1 (its lower halo), all four directions, 2 x 36 x Lx Ly Lz complex
numbers.  It goes through torch.distributed point-to-point calls: device
tensors with an NCCL group, host copies with a gloo group.  A single rank
(P = 1) copies its own edge slices into its halos.
"""
import numpy as np

from . import (Field, Geometry, LQ_BWD_SOURCE_GATHER, LQ_BWD_SOURCE_GIVEN, LQ_BWD_SOURCE_WILSON, LQ_LINKS,
               plaquette_sums, stout_backward_step, stout_step_range)


class TSlab:
    """The t-slab of `rank` out of `world` ranks of a (Lx, Ly, Lz, Lt) lattice."""

    def __init__(self, dims, rank, world):
        lx, ly, lz, lt = (int(d) for d in dims)
        if world < 1 or not 0 <= rank < world or lt % world != 0:
            raise ValueError(f"Lt = {lt} must split evenly over {world} ranks (rank {rank})")
        self.dims, self.rank, self.world = (lx, ly, lz, lt), rank, world
        self.nt = lt // world
        self.t0 = rank * self.nt
        self.v3 = lx * ly * lz
        self.local_dims = (lx, ly, lz, self.nt + 2)
        self.interior = (self.v3, self.v3 * (self.nt + 1))   # local site range of the owned slices

    def local_geometry(self):
        return Geometry(self.local_dims)

    def local_from_global(self, U):
        """The local array (halos included) of a global host link array (Lt, Lz, Ly, Lx, 4, 3, 3)."""
        lt = self.dims[3]
        return U[[(self.t0 - 1 + k) % lt for k in range(self.nt + 2)]]

    def owned(self, U_local):
        """The owned slices of a local host array (halos dropped)."""
        return U_local[1:self.nt + 1]

    def _slice(self, t, k):
        return t[:, :, k * self.v3:(k + 1) * self.v3]

    def exchange(self, field, group=None):
        """Fills both halo slices of `field` (its .tensor, [dir][comp][site](re, im)) from the neighbours."""
        t = field.tensor
        lo_halo, first = self._slice(t, 0), self._slice(t, 1)
        last, hi_halo = self._slice(t, self.nt), self._slice(t, self.nt + 1)
        if self.world == 1:
            lo_halo.copy_(last)
            hi_halo.copy_(first)
            return
        import torch.distributed as dist
        on_device = dist.get_backend(group) == "nccl"

        def staged(x):
            return x.contiguous() if on_device else x.contiguous().cpu()
        down, up = (self.rank - 1) % self.world, (self.rank + 1) % self.world
        send_down, send_up = staged(first), staged(last)
        recv_from_down, recv_from_up = torch_empty_like(send_down), torch_empty_like(send_up)
        # tag 0: a rank's first owned slice (the upper halo of the rank below);
        # tag 1: its last owned slice (the lower halo of the rank above).  The
        # receives are posted in the order the peer sends (first, then last),
        # so that they also pair up where messages match in order (NCCL; two
        # ranks, where the rank below is the rank above).
        ops = [dist.P2POp(dist.isend, send_down, _global(group, down), group, 0),
               dist.P2POp(dist.isend, send_up, _global(group, up), group, 1),
               dist.P2POp(dist.irecv, recv_from_up, _global(group, up), group, 0),
               dist.P2POp(dist.irecv, recv_from_down, _global(group, down), group, 1)]
        for r in dist.batch_isend_irecv(ops):
            r.wait()
        lo_halo.copy_(recv_from_down)
        hi_halo.copy_(recv_from_up)


def torch_empty_like(x):
    import torch
    return torch.empty_like(x)


def _global(group, r):
    """Global rank of group rank r (the default group: r itself)."""
    if group is None:
        return r
    import torch.distributed as dist
    return dist.get_global_rank(group, r)


def stout_smear(field, slab, rho, n_steps, dirs=(0, 1, 2, 3), group=None, stream=None, **opts):
    """n_steps stout steps of the lattice held slab-wise by the ranks of
    `group`; `field` is this rank's local LINKS field (halos included), smeared
    in place on its owned slices.  Collective: every rank of the group calls it."""
    if n_steps <= 0:
        return
    work = Field(field.geom, LQ_LINKS, field.prec)
    work.tensor.copy_(field.tensor)   # directions outside dirs pass through both buffers
    cur, nxt = field, work
    for _ in range(n_steps):
        slab.exchange(cur, group)
        stout_step_range(cur, nxt, rho, slab.interior[0], slab.interior[1], dirs, stream=stream, **opts)
        cur, nxt = nxt, cur
    if n_steps % 2 == 1:
        field.tensor.copy_(work.tensor)


def stout_backward(field, slab, rho, n_steps, dirs=(0, 1, 2, 3), force_out=None, grad_out=None, grad_seed=None,
                   beta=6.0, group=None, stream=None):
    """Gradient of S(stout^n(U)) w.r.t. the thin links of the lattice held
    slab-wise by the ranks of `group`, as lq_stout_backward computes it for
    the whole lattice (MP Sec. IV): S is the Wilson action of the smeared
    field at `beta`, or given by its gradient `grad_seed` at U^(n) (this
    rank's local field; owned slices read).  `field` holds this rank's thin
    links (halos included) and is not modified; force_out and grad_out
    (local LINKS fields) receive the force TA(G U^dag) and the gradient G on
    the owned slices.  Collective: every rank of the group calls it.

    The forward steps are kept (one local field per step, each with its
    halos exchanged).  Each backward step reads K of the step after it one
    slice beyond the owned ones, so K's halos are exchanged between the
    steps, just as the links' are between forward steps; G passes between
    steps at the link itself and needs no exchange."""
    if force_out is None and grad_out is None:
        raise ValueError("give force_out and/or grad_out")
    if n_steps < 0:
        raise ValueError("n_steps must be >= 0")
    s0, s1 = slab.interior
    U = [Field(field.geom, LQ_LINKS, field.prec)]
    U[0].tensor.copy_(field.tensor)
    slab.exchange(U[0], group)
    for _ in range(n_steps):
        nxt = Field(field.geom, LQ_LINKS, field.prec)
        nxt.tensor.copy_(U[-1].tensor)   # directions outside dirs pass through
        stout_step_range(U[-1], nxt, rho, s0, s1, dirs, stream=stream)
        slab.exchange(nxt, group)
        U.append(nxt)
    G = [Field(field.geom, LQ_LINKS, field.prec) for _ in range(2)]
    K = [Field(field.geom, LQ_LINKS, field.prec) for _ in range(2)]
    for f in K:
        f.tensor.zero_()
    source = LQ_BWD_SOURCE_GIVEN if grad_seed is not None else LQ_BWD_SOURCE_WILSON
    g_in, k_next = grad_seed, None
    for j in range(n_steps - 1, -1, -1):
        g_out, k_out = G[j % 2], K[j % 2]
        stout_backward_step(U[j], source, rho, s0, s1, dirs, u_next=U[j + 1], k_next=k_next, g_in=g_in,
                            g_out=g_out, k_out=k_out, beta=beta, stream=stream)
        slab.exchange(k_out, group)
        source, g_in, k_next = LQ_BWD_SOURCE_GATHER, g_out, k_out
    # the gather of step 0's K on the thin links (n = 0: the seed at them)
    stout_backward_step(U[0], source, rho, s0, s1, dirs, u_next=U[0], k_next=k_next, g_in=g_in, g_out=grad_out,
                        force_out=force_out, beta=beta, stream=stream)


def plaquette(field, slab, group=None, stream=None):
    """(average, spatial, temporal) plaquette of the whole lattice; collective."""
    slab.exchange(field, group)
    s, t = plaquette_sums(field, slab.interior[0], slab.interior[1], stream=stream)
    if slab.world > 1:
        import torch
        import torch.distributed as dist
        dev = field.tensor.device if dist.get_backend(group) == "nccl" else "cpu"
        v = torch.tensor([s, t], dtype=torch.float64, device=dev)
        dist.all_reduce(v, group=group)
        s, t = float(v[0]), float(v[1])
    V = float(np.prod(slab.dims))
    return ((s + t) / (18.0 * V), s / (9.0 * V), t / (9.0 * V))
