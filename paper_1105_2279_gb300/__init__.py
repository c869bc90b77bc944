"""Python binding of liblqcd, the GB300 (sm_103a) library for lattice field
expressions and stout link smearing.

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels, reached through the C ABI of include/lqcd.h via
ctypes.  PyTorch supplies device memory (fields are torch tensors in the
structure-of-arrays layout [ndir, ncomp, V, 2]) and the current CUDA stream.
The functions carry the C names without the ``lq_`` prefix; the raw C
entry points are available as ``paper_1105_2279_gb300.capi()``.
"""
import ctypes
from ctypes import byref, c_double, c_int, c_longlong, c_size_t, c_void_p

import numpy as np

from . import _lib as L
from ._lib import (LQ_COLOR_MATRIX, LQ_COLOR_VECTOR, LQ_COMPLEX, LQ_F32, LQ_F64, LQ_FERMION,  # noqa: F401
                   LQ_LINKS, LQ_REAL, LqBackwardOpts, LqOp, LqStoutOpts)

KIND_SHAPE = {LQ_LINKS: (4, 9), LQ_COLOR_MATRIX: (1, 9), LQ_COLOR_VECTOR: (1, 3), LQ_COMPLEX: (1, 1),
              LQ_REAL: (1, 1), LQ_FERMION: (1, 12)}
# per-site trailing shape of the host (AoS) arrays
SITE_SHAPE = {LQ_LINKS: (4, 3, 3), LQ_COLOR_MATRIX: (3, 3), LQ_COLOR_VECTOR: (3,), LQ_COMPLEX: (), LQ_REAL: (),
              LQ_FERMION: (4, 3)}


class LqError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


def capi():
    return L.load()


def _check(st, what):
    if st != L.LQ_OK:
        msg = L.load().lq_last_error().decode(errors="replace")
        raise LqError(st, f"{what}: {L.STATUS_NAMES.get(st, st)}: {msg}")


def _stream(stream):
    if stream is not None:
        if hasattr(stream, "cuda_stream"):      # torch.cuda.Stream
            return c_void_p(stream.cuda_stream)
        return c_void_p(int(stream))
    import torch
    return c_void_p(torch.cuda.current_stream().cuda_stream)


def dirs_mask(dirs):
    if isinstance(dirs, int):
        return dirs
    m = 0
    for mu in dirs:
        m |= 1 << int(mu)
    return m


class Geometry:
    """Periodic 4D lattice (Lx, Ly, Lz, Lt); site index x fastest."""

    def __init__(self, dims):
        self.dims = tuple(int(d) for d in dims)
        arr = (c_int * 4)(*self.dims)
        h = c_void_p()
        _check(L.load().lq_geom_create(arr, byref(h)), "lq_geom_create")
        self.handle = h
        self.volume = int(np.prod(self.dims))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and L._lib is not None:
            L._lib.lq_geom_destroy(h)
            self.handle = None


class Field:
    """A lattice field in device memory: a torch tensor wrapped as an lq_field."""

    def __init__(self, geom, kind, prec, tensor=None, device="cuda"):
        import torch
        self.geom, self.kind, self.prec = geom, kind, prec
        nd, nc = KIND_SHAPE[kind]
        dt = torch.float64 if prec == LQ_F64 else torch.float32
        shape = (nd, nc, geom.volume) if kind == LQ_REAL else (nd, nc, geom.volume, 2)
        if tensor is None:
            tensor = torch.empty(shape, dtype=dt, device=device)
        if tuple(tensor.shape) != shape or tensor.dtype != dt or not tensor.is_contiguous():
            raise ValueError(f"tensor must be contiguous {dt} of shape {shape}")
        self.tensor = tensor
        h = c_void_p()
        _check(L.load().lq_field_wrap(geom.handle, kind, prec, c_void_p(tensor.data_ptr()),
                                      tensor.numel() * tensor.element_size(), byref(h)), "lq_field_wrap")
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and L._lib is not None:
            L._lib.lq_field_free(h)
            self.handle = None

    @property
    def nbytes(self):
        return self.tensor.numel() * self.tensor.element_size()

    def host_dtype(self):
        if self.kind == LQ_REAL:
            return np.float64 if self.prec == LQ_F64 else np.float32
        return np.complex128 if self.prec == LQ_F64 else np.complex64

    def host_shape(self):
        lx, ly, lz, lt = self.geom.dims
        return (lt, lz, ly, lx) + SITE_SHAPE[self.kind]

    def upload(self, host, stream=None):
        """host: array in the AoS interchange layout (any shape with the right size); converted to
        the field precision on the host, then copied and transposed on the device."""
        a = np.ascontiguousarray(np.asarray(host).astype(self.host_dtype(), copy=False))
        if a.nbytes != self.nbytes:
            raise ValueError(f"host array has {a.nbytes} bytes, field needs {self.nbytes}")
        _check(L.load().lq_field_upload(self.handle, c_void_p(a.ctypes.data), _stream(stream)), "lq_field_upload")

    def upload_ptr(self, host_ptr, stream=None):
        _check(L.load().lq_field_upload(self.handle, c_void_p(host_ptr), _stream(stream)), "lq_field_upload")

    def download(self, stream=None):
        a = np.empty(self.host_shape(), dtype=self.host_dtype())
        _check(L.load().lq_field_download(self.handle, c_void_p(a.ctypes.data), _stream(stream)),
               "lq_field_download")
        return a

    def download_ptr(self, host_ptr, stream=None):
        _check(L.load().lq_field_download(self.handle, c_void_p(host_ptr), _stream(stream)), "lq_field_download")

    def save(self, path, stream=None):
        """lq_field_save: header + AoS payload."""
        _check(L.load().lq_field_save(self.handle, str(path).encode(), _stream(stream)), "lq_field_save")

    def load(self, path, stream=None):
        """lq_field_load: refuses files of another geometry, kind or precision."""
        _check(L.load().lq_field_load(self.handle, str(path).encode(), _stream(stream)), "lq_field_load")

    @classmethod
    def from_host(cls, geom, kind, prec, host, device="cuda", stream=None):
        f = cls(geom, kind, prec, device=device)
        f.upload(host, stream)
        return f


def shift(out, inp, mu, sign, stream=None):
    """out(x) = inp(x + sign*mu) (sign +1 FORWARD, -1 BACKWARD)."""
    _check(L.load().lq_shift(out.handle, inp.handle, int(mu), int(sign), _stream(stream)), "lq_shift")


def compile_program(prog):
    """Tuple program (oracle.expr notation) -> ctypes array of LqOp."""
    ops = []
    for op in prog:
        k = op[0]
        o = LqOp()
        if k == "load":
            o.code, o.dst, o.a, o.mu, o.sign = L.LQ_OP_LOAD, op[1], op[2], op[3], op[4]
        elif k == "loadl":
            o.code, o.dst, o.a, o.dir, o.mu, o.sign = L.LQ_OP_LOAD, op[1], op[2], op[3], op[4], op[5]
        elif k in ("adj", "trace", "retr"):
            o.code = {"adj": L.LQ_OP_ADJ, "trace": L.LQ_OP_TRACE, "retr": L.LQ_OP_RETR}[k]
            o.dst, o.a = op[1], op[2]
        elif k in ("mul", "add", "sub"):
            o.code = {"mul": L.LQ_OP_MUL, "add": L.LQ_OP_ADD, "sub": L.LQ_OP_SUB}[k]
            o.dst, o.a, o.b = op[1], op[2], op[3]
        elif k == "scale":
            o.code, o.dst, o.a, o.re, o.im = L.LQ_OP_SCALE, op[1], op[2], float(op[3]), float(op[4])
        elif k == "store":
            o.code, o.a = L.LQ_OP_STORE, op[1]
        else:
            raise ValueError(f"op {k!r} has no C-ABI form (shifts apply to loads)")
        ops.append(o)
    arr = (LqOp * len(ops))(*ops)
    return arr, len(ops)


def expr_eval(prog, operands, out=None, reduce=False, stream=None):
    """Evaluates a per-site program; returns sum_x tr(result) if reduce."""
    arr, n = compile_program(prog)
    hs = (c_void_p * len(operands))(*[f.handle for f in operands])
    red = (c_double * 2)()
    _check(L.load().lq_expr_eval(out.handle if out is not None else None, arr, n, hs, len(operands),
                                 red if reduce else None, _stream(stream)), "lq_expr_eval")
    return complex(red[0], red[1]) if reduce else None


def expr_eval_jit(prog, operands, out=None, reduce=False, stream=None):
    """expr_eval through an NVRTC-compiled kernel (lq_expr_eval_jit)."""
    arr, n = compile_program(prog)
    hs = (c_void_p * len(operands))(*[f.handle for f in operands])
    red = (c_double * 2)()
    _check(L.load().lq_expr_eval_jit(out.handle if out is not None else None, arr, n, hs, len(operands),
                                     red if reduce else None, _stream(stream)), "lq_expr_eval_jit")
    return complex(red[0], red[1]) if reduce else None


def expr_jit_prepare(prog, operands, out=None, reduce=False):
    """Compiles (or finds cached) the JIT kernel of a program without launching it."""
    arr, n = compile_program(prog)
    hs = (c_void_p * len(operands))(*[f.handle for f in operands])
    _check(L.load().lq_expr_jit_prepare(out.handle if out is not None else None, arr, n, hs, len(operands),
                                        int(bool(reduce))), "lq_expr_jit_prepare")


def jit_cache_dir(path=None):
    _check(L.load().lq_jit_cache_dir(path.encode() if path else None), "lq_jit_cache_dir")


def jit_stats():
    """(NVRTC compilations, memory hits, disk hits, module loads)."""
    out = (ctypes.c_longlong * 4)()
    _check(L.load().lq_jit_stats(out), "lq_jit_stats")
    return tuple(out)


def reduce_sum(f, stream=None):
    r = (c_double * 2)()
    _check(L.load().lq_reduce_sum(f.handle, r, _stream(stream)), "lq_reduce_sum")
    return complex(r[0], r[1])


def reduce_trace(f, stream=None):
    r = (c_double * 2)()
    _check(L.load().lq_reduce_trace(f.handle, r, _stream(stream)), "lq_reduce_trace")
    return complex(r[0], r[1])


def plaquette(links, stream=None):
    """(average, spatial, temporal) plaquette."""
    r = (c_double * 3)()
    _check(L.load().lq_plaquette(links.handle, r, _stream(stream)), "lq_plaquette")
    return (r[0], r[1], r[2])


def plaquette_sums(links, s_begin, s_end, stream=None):
    """Unnormalised (spatial, temporal) Re tr P sums over the sites [s_begin, s_end)."""
    r = (c_double * 2)()
    _check(L.load().lq_plaquette_sums(links.handle, int(s_begin), int(s_end), r, _stream(stream)),
           "lq_plaquette_sums")
    return (r[0], r[1])


def wilson_action(links, beta, stream=None):
    r = c_double()
    _check(L.load().lq_wilson_action(links.handle, float(beta), byref(r), _stream(stream)), "lq_wilson_action")
    return r.value


def stout_opts(reproject=None, use_graph=False, variant=0, block=0, sites_per_thread=0, work=None):
    o = LqStoutOpts()
    o.struct_size = ctypes.sizeof(LqStoutOpts)
    o.reproject = -1 if reproject is None else int(bool(reproject))
    o.use_graph = int(bool(use_graph))
    o.variant, o.block, o.sites_per_thread = int(variant), int(block), int(sites_per_thread)
    if work is not None:
        o.work = c_void_p(work.data_ptr())
        o.work_bytes = work.numel() * work.element_size()
    return o


def stout_smear(links, rho, n_steps, dirs=(0, 1, 2, 3), stream=None, **opts):
    """In-place stout smearing of a LINKS field (see lq_stout_smear)."""
    o = stout_opts(**opts)
    _check(L.load().lq_stout_smear(links.handle, float(rho), int(n_steps), dirs_mask(dirs), byref(o),
                                   _stream(stream)), "lq_stout_smear")


def stout_step_range(inp, out, rho, s_begin, s_end, dirs=(0, 1, 2, 3), stream=None, **opts):
    """One stout step from `inp` into `out` over the sites [s_begin, s_end) (lq_stout_step_range)."""
    o = stout_opts(**opts)
    _check(L.load().lq_stout_step_range(inp.handle, out.handle, float(rho), dirs_mask(dirs), int(s_begin),
                                        int(s_end), byref(o), _stream(stream)), "lq_stout_step_range")


LQ_BWD_SOURCE_WILSON, LQ_BWD_SOURCE_GIVEN, LQ_BWD_SOURCE_GATHER = 0, 1, 2


def stout_backward_step(u_cur, source, rho, s_begin, s_end, dirs=(0, 1, 2, 3), u_next=None, k_next=None,
                        g_in=None, g_out=None, k_out=None, force_out=None, beta=6.0, stream=None):
    """One step of the stout force recursion on the sites [s_begin, s_end) (lq_stout_backward_step)."""
    def h(f):
        return f.handle if f is not None else None
    _check(L.load().lq_stout_backward_step(h(u_next), h(k_next), h(g_in), u_cur.handle, h(g_out), h(k_out),
                                           h(force_out), int(source), float(rho), float(beta), dirs_mask(dirs),
                                           int(s_begin), int(s_end), _stream(stream)), "lq_stout_backward_step")


def stout_smear_noalloc(links, rho, n_steps, dirs=(0, 1, 2, 3), stream=None):
    """lq_stout_smear_noalloc: same result as stout_smear, no device allocation (fields up to 32 MiB)."""
    _check(L.load().lq_stout_smear_noalloc(links.handle, float(rho), int(n_steps), dirs_mask(dirs), _stream(stream)),
           "lq_stout_smear_noalloc")


def _host_ptr(a):
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):       # torch tensor (e.g. page-locked)
        return int(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host array must be C-contiguous")
        return int(a.ctypes.data)
    raise TypeError(f"cannot take a host pointer from {type(a).__name__}")


def stout_smear_host(host_in, host_out, geom, prec, rho, n_steps, dirs=(0, 1, 2, 3), n_chunks=0, stream=None,
                     **opts):
    """lq_stout_smear_host: AoS links in host memory -> smeared AoS links in host memory, the
    transfers overlapped with the smearing; returns lq_plaquette of the result.  host_in/out:
    numpy arrays, torch tensors (page-locked for asynchronous copies) or raw pointers."""
    g = geom if isinstance(geom, Geometry) else Geometry(geom)
    for a in (host_in, host_out):
        nb = getattr(a, "nbytes", None)
        if nb is None and hasattr(a, "element_size"):
            nb = a.element_size() * a.numel()
        need = g.volume * 36 * (8 if prec == LQ_F32 else 16)
        if nb is not None and nb != need:
            raise ValueError(f"host buffer has {nb} bytes, the links need {need}")
    o = stout_opts(**opts)
    out = (c_double * 3)()
    _check(L.load().lq_stout_smear_host(c_void_p(_host_ptr(host_in)), c_void_p(_host_ptr(host_out)), g.handle,
                                        int(prec), float(rho), int(n_steps), dirs_mask(dirs), int(n_chunks), out,
                                        byref(o), _stream(stream)), "lq_stout_smear_host")
    return out[0], out[1], out[2]


def stout_ch_stats(links, rho, n_steps, dirs=(0, 1, 2, 3), stream=None):
    """(link updates, updates on the series branch, sum of series orders K) of
    n_steps stout steps of `links` (lq_stout_ch_stats; links unchanged)."""
    c = (c_longlong * 3)()
    _check(L.load().lq_stout_ch_stats(links.handle, float(rho), int(n_steps), dirs_mask(dirs), c,
                                      _stream(stream)), "lq_stout_ch_stats")
    return int(c[0]), int(c[1]), int(c[2])


def peak_probe(prec, stream=None):
    """Measured FMA throughput of the FP32 or FP64 pipe in TFLOP/s (lq_peak_probe)."""
    t = c_double()
    _check(L.load().lq_peak_probe(int(prec), byref(t), _stream(stream)), "lq_peak_probe")
    return t.value


def expiq(out, q, stream=None):
    """out = exp(iQ) per site (Cayley-Hamilton, FP64 coefficients) of a COLOR_MATRIX field."""
    _check(L.load().lq_expiq(out.handle, q.handle, _stream(stream)), "lq_expiq")


def ape_smear(links, alpha, n_steps, dirs=(0, 1, 2, 3), stream=None):
    """In-place APE smearing of a LINKS field (lq_ape_smear)."""
    _check(L.load().lq_ape_smear(links.handle, float(alpha), int(n_steps), dirs_mask(dirs), _stream(stream)),
           "lq_ape_smear")


def hyp_smear(links, a1=0.75, a2=0.6, a3=0.3, n_steps=1, stream=None):
    """In-place HYP smearing of a LINKS field, all four directions (lq_hyp_smear)."""
    _check(L.load().lq_hyp_smear(links.handle, float(a1), float(a2), float(a3), int(n_steps), _stream(stream)),
           "lq_hyp_smear")


class LqJacobiOpts(ctypes.Structure):
    _fields_ = [("struct_size", c_int), ("compress_links", c_int), ("block", c_int), ("sites_per_thread", c_int)]


def jacobi_smear(links, chi, kappa, n_iter, norm=1.0, dirs=(0, 1, 2, 3), stream=None, compress_links=False,
                 block=0, sites_per_thread=0):
    """In-place Jacobi smearing of a COLOR_VECTOR or FERMION field (Listing 1); compress_links
    reads rows 0-1 of each link and rebuilds row 2; block / sites_per_thread set the thread
    geometry N_threads / N_site (0: tuned or default) (lq_jacobi_smear_ex)."""
    o = LqJacobiOpts(ctypes.sizeof(LqJacobiOpts), int(bool(compress_links)), int(block), int(sites_per_thread))
    _check(L.load().lq_jacobi_smear_ex(links.handle, chi.handle, float(kappa), int(n_iter), float(norm),
                                       dirs_mask(dirs), byref(o), _stream(stream)), "lq_jacobi_smear")


def stout_smear_batch(fields, rho, n_steps, dirs=(0, 1, 2), stream=None, **opts):
    o = stout_opts(**opts)
    hs = (c_void_p * len(fields))(*[f.handle for f in fields])
    _check(L.load().lq_stout_smear_batch(hs, len(fields), float(rho), int(n_steps), dirs_mask(dirs), byref(o),
                                         _stream(stream)), "lq_stout_smear_batch")


def stout_backward(thin, rho, n_steps, dirs, force_out, grad_seed=None, beta=6.0, grad_out=None,
                   checkpoint_every=1, stream=None):
    o = LqBackwardOpts()
    o.struct_size = ctypes.sizeof(LqBackwardOpts)
    o.checkpoint_every = int(checkpoint_every)
    _check(L.load().lq_stout_backward(thin.handle, float(rho), int(n_steps), dirs_mask(dirs),
                                      grad_seed.handle if grad_seed is not None else None, float(beta),
                                      force_out.handle if force_out is not None else None,
                                      grad_out.handle if grad_out is not None else None,
                                      byref(o), _stream(stream)), "lq_stout_backward")


def ape_backward(thin, alpha, n_steps, dirs, force_out, grad_seed=None, beta=6.0, grad_out=None,
                 checkpoint_every=1, stream=None):
    o = LqBackwardOpts()
    o.struct_size = ctypes.sizeof(LqBackwardOpts)
    o.checkpoint_every = int(checkpoint_every)
    _check(L.load().lq_ape_backward(thin.handle, float(alpha), int(n_steps), dirs_mask(dirs),
                                    grad_seed.handle if grad_seed is not None else None, float(beta),
                                    force_out.handle if force_out is not None else None,
                                    grad_out.handle if grad_out is not None else None,
                                    byref(o), _stream(stream)), "lq_ape_backward")


def hyp_backward(thin, a1, a2, a3, n_steps, force_out, grad_seed=None, beta=6.0, grad_out=None,
                 checkpoint_every=1, stream=None):
    o = LqBackwardOpts()
    o.struct_size = ctypes.sizeof(LqBackwardOpts)
    o.checkpoint_every = int(checkpoint_every)
    _check(L.load().lq_hyp_backward(thin.handle, float(a1), float(a2), float(a3), int(n_steps),
                                    grad_seed.handle if grad_seed is not None else None, float(beta),
                                    force_out.handle if force_out is not None else None,
                                    grad_out.handle if grad_out is not None else None,
                                    byref(o), _stream(stream)), "lq_hyp_backward")


def tune(cache_path=None):
    _check(L.load().lq_tune(cache_path.encode() if cache_path else None), "lq_tune")


def tune_lookup(prec, dims, dirs):
    b, n, v = c_int(), c_int(), c_int()
    st = L.load().lq_tune_lookup(int(prec), (c_int * 4)(*dims), dirs_mask(dirs), byref(b), byref(n), byref(v))
    return (b.value, n.value, v.value) if st == L.LQ_OK else None


def free_all():
    _check(L.load().lq_free_all(), "lq_free_all")


def field_bytes(geom, kind, prec):
    n = c_size_t()
    _check(L.load().lq_field_bytes(geom.handle, kind, prec, byref(n)), "lq_field_bytes")
    return n.value


def geom_info(geom):
    d = (c_int * 4)()
    v = c_longlong()
    _check(L.load().lq_geom_info(geom.handle, d, byref(v)), "lq_geom_info")
    return tuple(d), v.value


def _prec_of(t):
    import torch
    if t.dtype == torch.float64:
        return LQ_F64
    if t.dtype == torch.float32:
        return LQ_F32
    raise TypeError("links tensors are float32 or float64, shaped [4, 9, V, 2]")


def _autograd():
    import torch

    class StoutSmear(torch.autograd.Function):
        """U -> stout^n(U) on a links tensor [4, 9, V, 2] (structure of arrays).

        The gradient w.r.t. the tensor's real components is the field
        G = dL/dRe U + i dL/dIm U in the same layout, which is exactly the seed
        lq_stout_backward expects; its result is returned in the same form."""

        @staticmethod
        def forward(ctx, links, dims, rho, n_steps, dirs):
            geom = Geometry(dims)
            prec = _prec_of(links)
            out = torch.empty_like(links)
            out.copy_(links)
            stout_smear(Field(geom, LQ_LINKS, prec, tensor=out), rho, n_steps, dirs)
            ctx.save_for_backward(links)
            ctx.args = (dims, rho, n_steps, dirs, prec)
            return out

        @staticmethod
        def backward(ctx, grad):
            (links,) = ctx.saved_tensors
            dims, rho, n_steps, dirs, prec = ctx.args
            geom = Geometry(dims)
            thin = Field(geom, LQ_LINKS, prec, tensor=links.contiguous())
            seed = Field(geom, LQ_LINKS, prec, tensor=grad.contiguous())
            gout = Field(geom, LQ_LINKS, prec)
            stout_backward(thin, rho, n_steps, dirs, None, grad_seed=seed, grad_out=gout)
            return gout.tensor, None, None, None, None

    class ApeSmear(torch.autograd.Function):
        """U -> ape^n(U) on a links tensor [4, 9, V, 2]; gradients as in StoutSmear."""

        @staticmethod
        def forward(ctx, links, dims, alpha, n_steps, dirs):
            geom = Geometry(dims)
            prec = _prec_of(links)
            out = torch.empty_like(links)
            out.copy_(links)
            ape_smear(Field(geom, LQ_LINKS, prec, tensor=out), alpha, n_steps, dirs)
            ctx.save_for_backward(links)
            ctx.args = (dims, alpha, n_steps, dirs, prec)
            return out

        @staticmethod
        def backward(ctx, grad):
            (links,) = ctx.saved_tensors
            dims, alpha, n_steps, dirs, prec = ctx.args
            geom = Geometry(dims)
            thin = Field(geom, LQ_LINKS, prec, tensor=links.contiguous())
            seed = Field(geom, LQ_LINKS, prec, tensor=grad.contiguous())
            gout = Field(geom, LQ_LINKS, prec)
            ape_backward(thin, alpha, n_steps, dirs, None, grad_seed=seed, grad_out=gout)
            return gout.tensor, None, None, None, None

    class HypSmear(torch.autograd.Function):
        """U -> hyp^n(U) on a links tensor [4, 9, V, 2]; gradients as in StoutSmear."""

        @staticmethod
        def forward(ctx, links, dims, weights, n_steps):
            geom = Geometry(dims)
            prec = _prec_of(links)
            out = torch.empty_like(links)
            out.copy_(links)
            hyp_smear(Field(geom, LQ_LINKS, prec, tensor=out), *weights, n_steps)
            ctx.save_for_backward(links)
            ctx.args = (dims, weights, n_steps, prec)
            return out

        @staticmethod
        def backward(ctx, grad):
            (links,) = ctx.saved_tensors
            dims, weights, n_steps, prec = ctx.args
            geom = Geometry(dims)
            thin = Field(geom, LQ_LINKS, prec, tensor=links.contiguous())
            seed = Field(geom, LQ_LINKS, prec, tensor=grad.contiguous())
            gout = Field(geom, LQ_LINKS, prec)
            hyp_backward(thin, *weights, n_steps, None, grad_seed=seed, grad_out=gout)
            return gout.tensor, None, None, None

    class WilsonAction(torch.autograd.Function):
        """S = beta sum_x sum_{mu<nu} (1 - Re tr P_{mu nu}(x)/3) of a links tensor (FP64 scalar)."""

        @staticmethod
        def forward(ctx, links, dims, beta):
            geom = Geometry(dims)
            prec = _prec_of(links)
            s = wilson_action(Field(geom, LQ_LINKS, prec, tensor=links.contiguous()), beta)
            ctx.save_for_backward(links)
            ctx.args = (dims, beta, prec)
            return torch.tensor(s, dtype=torch.float64, device=links.device)

        @staticmethod
        def backward(ctx, grad):
            (links,) = ctx.saved_tensors
            dims, beta, prec = ctx.args
            geom = Geometry(dims)
            thin = Field(geom, LQ_LINKS, prec, tensor=links.contiguous())
            gout = Field(geom, LQ_LINKS, prec)
            # the Wilson gradient is linear in beta: scale the upstream factor into it
            stout_backward(thin, 0.0, 0, 15, None, beta=beta * float(grad), grad_out=gout)
            return gout.tensor, None, None

    return StoutSmear, WilsonAction, ApeSmear, HypSmear


def stout_smear_autograd(links, dims, rho, n_steps, dirs=(0, 1, 2, 3)):
    return _autograd()[0].apply(links, tuple(dims), float(rho), int(n_steps), dirs_mask(dirs))


def ape_smear_autograd(links, dims, alpha, n_steps, dirs=(0, 1, 2, 3)):
    return _autograd()[2].apply(links, tuple(dims), float(alpha), int(n_steps), dirs_mask(dirs))


def hyp_smear_autograd(links, dims, a1=0.75, a2=0.6, a3=0.3, n_steps=1):
    return _autograd()[3].apply(links, tuple(dims), (float(a1), float(a2), float(a3)), int(n_steps))


def wilson_action_autograd(links, dims, beta):
    return _autograd()[1].apply(links, tuple(dims), float(beta))
