"""GPU stout smearing through the C ABI vs the FP64 oracle.

FP64 path: max |U_gpu - U_oracle| <= 1e-12 per link element (elements of SU(3)
matrices are at most 1 in magnitude, so this is also the relative error with
respect to the link).

FP32 path (FP32 matrix algebra, FP64 Cayley-Hamilton coefficients and
re-projection), stated bound on the max per-element error against the exact
(FP64) result, for up to 6 steps:
  3e-7 on near-identity fields (exp(i 0.3 H)) up to 12^3 x 24,
  4e-7 over the whole 48^3 x 96 lattice (4.2e8 elements: a larger maximum),
  6e-7 on Haar-random fields (rho <= 0.4; links past the series domain).
Measured on GB300 (3 seeds per case): 1.1e-7 .. 1.9e-7, 2.58e-7 and
3.4e-7 .. 4.2e-7.  The error does not grow with the number of steps (48^3 x 96:
2.43e-7 after 1 step, 2.58e-7 after 6): the input's own FP32 rounding
(<= 4.2e-8) and each step's rounding are not amplified, since smearing is
contractive and the FP64 re-projection holds every link on SU(3).
Unitarity of FP32 results <= 1e-6.
"""
import numpy as np
import pytest

import fieldgen
import paper_1105_2279_gb300 as lq
from oracle import gauge, lattice, stout
from oracle.su3 import unitarity_violation
from tests.gpu_util import links_err, upload_links

pytestmark = pytest.mark.gpu
ALL, SPATIAL = (0, 1, 2, 3), (0, 1, 2)
F64_TOL = 1e-12
F32_TOL = {"near": 3e-7, "haar": 6e-7}
F32_TOL_48C96 = 4e-7


def _run(U, prec, rho, n, dirs, **opts):
    f = upload_links(U, prec)
    lq.stout_smear(f, rho, n, dirs, **opts)
    return f.download()


@pytest.mark.parametrize("dims,gen,rho,n,dirs", [
    ((4, 4, 4, 4), "haar", 0.1, 1, ALL),          # the 4^4 plain-method workload
    ((2, 2, 2, 2), "haar", 0.1, 2, ALL),          # x+mu == x-mu
    ((3, 4, 5, 6), "near", 0.125, 3, ALL),        # odd extents, V not a multiple of any block
    ((3, 4, 5, 6), "near", 0.1, 3, SPATIAL),
    ((5, 3, 2, 7), "haar", 0.25, 2, (1, 3)),
    ((6, 6, 6, 12), "near", 0.1, 4, ALL),
    ((8, 8, 8, 16), "near", 0.1, 2, SPATIAL),
    ((4, 4, 4, 4), "haar", 0.4, 2, ALL),          # ~40 % of links past the series domain c1 <= 3/4
])
def test_f64_matches_oracle(gpu, dims, gen, rho, n, dirs):
    U = fieldgen.haar_su3(dims, 100) if gen == "haar" else fieldgen.near_identity_su3(dims, 100)
    ref = stout.stout_smear(U, rho, n, dirs)
    got = _run(U, lq.LQ_F64, rho, n, dirs)
    a, r = links_err(got, ref)
    assert a <= F64_TOL and r <= F64_TOL, (a, r)
    for mu in range(4):
        if mu not in dirs:
            assert np.array_equal(got[..., mu, :, :], U[..., mu, :, :])


@pytest.mark.parametrize("dims,gen,rho,n,dirs", [
    ((4, 4, 4, 4), "haar", 0.1, 1, ALL),
    ((3, 4, 5, 6), "near", 0.125, 3, ALL),
    ((6, 5, 4, 8), "near", 0.1, 6, SPATIAL),
    ((2, 2, 2, 2), "haar", 0.1, 2, ALL),
    ((4, 4, 4, 4), "haar", 0.4, 2, ALL),
])
def test_f32_mixed_matches_oracle(gpu, dims, gen, rho, n, dirs):
    U = fieldgen.haar_su3(dims, 101) if gen == "haar" else fieldgen.near_identity_su3(dims, 101)
    ref = stout.stout_smear(U, rho, n, dirs)
    got = _run(U, lq.LQ_F32, rho, n, dirs)
    a, _ = links_err(got, ref)
    assert a <= F32_TOL[gen], a
    du, dd = unitarity_violation(got.astype(np.complex128))
    assert du < 1e-6 and dd < 1e-6, (du, dd)


def test_unit_field_and_rho_zero(gpu):
    dims = (4, 3, 2, 5)
    U1 = fieldgen.unit_links(dims)
    for prec in (lq.LQ_F64, lq.LQ_F32):
        got = _run(U1, prec, 0.2, 3, ALL)
        assert np.array_equal(got.astype(np.complex128), U1)
    U = fieldgen.haar_su3(dims, 102)
    got = _run(U, lq.LQ_F64, 0.0, 2, ALL)
    assert np.array_equal(got, U)


def test_unitarity_f64(gpu):
    U = fieldgen.haar_su3((4, 4, 4, 4), 103)
    got = _run(U, lq.LQ_F64, 0.125, 5, ALL)
    du, dd = unitarity_violation(got)
    assert du < 1e-13 and dd < 1e-13


def test_gauge_covariance_gpu(gpu):
    dims = (4, 3, 4, 3)
    U = fieldgen.haar_su3(dims, 104)
    g = fieldgen.gauge_field_g(dims, 105)
    a = _run(gauge.gauge_transform(U, g), lq.LQ_F64, 0.1, 2, ALL)
    b = gauge.gauge_transform(_run(U, lq.LQ_F64, 0.1, 2, ALL), g)
    assert np.max(np.abs(a - b)) < 1e-12


@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
def test_launch_shapes_graph_and_workspace_agree_bitwise(gpu, prec):
    import torch
    dims = (5, 6, 3, 7)
    U = fieldgen.near_identity_su3(dims, 106)
    base = _run(U, prec, 0.1, 3, ALL)
    for block, ns in [(32, 1), (64, 2), (256, 4), (128, 3)]:
        got = _run(U, prec, 0.1, 3, ALL, block=block, sites_per_thread=ns)
        assert np.array_equal(got, base), (block, ns)
    for _ in range(2):   # graph recorded on the first call, replayed on the second
        assert np.array_equal(_run(U, prec, 0.1, 3, ALL, use_graph=True), base)
    f = upload_links(U, prec)
    work = torch.empty_like(f.tensor)
    lq.stout_smear(f, 0.1, 3, ALL, work=work)
    assert np.array_equal(f.download(), base)


@pytest.mark.parametrize("dims,dirs", [((8, 8, 8, 16), ALL), ((5, 6, 7, 9), ALL), ((3, 4, 5, 6), SPATIAL),
                                       ((2, 2, 2, 2), ALL), ((1, 4, 3, 5), (1, 2, 3)), ((12, 4, 8, 3), (0, 3))])
def test_shared_memory_variant_bitwise_equal(gpu, dims, dirs):
    """The shared-memory staged kernel (FP32) performs the same arithmetic in the
    same order as the global-load kernel: results are bit-identical, for ragged
    tiles, lattices smaller than a tile and any number of t-slices per block."""
    U = fieldgen.near_identity_su3(dims, 108)
    base = _run(U, lq.LQ_F32, 0.1, 3, dirs, block=128, sites_per_thread=1)
    for tchunk in (1, 3, 8, 100):
        got = _run(U, lq.LQ_F32, 0.1, 3, dirs, variant=2, sites_per_thread=tchunk)
        assert np.array_equal(got, base), tchunk
    got = _run(U, lq.LQ_F32, 0.1, 2, dirs, variant=2, reproject=False)
    assert np.array_equal(got, _run(U, lq.LQ_F32, 0.1, 2, dirs, block=64, reproject=False))


def test_shared_memory_variant_is_fp32_only(gpu):
    f = upload_links(fieldgen.unit_links((2, 2, 2, 2)), lq.LQ_F64)
    with pytest.raises(lq.LqError) as e:
        lq.stout_smear(f, 0.1, 1, ALL, variant=2)
    assert e.value.status == -7


def test_autotuner_keeps_results(gpu, tmp_path):
    dims = (6, 4, 4, 8)
    U = fieldgen.near_identity_su3(dims, 107)
    base = _run(U, lq.LQ_F64, 0.1, 2, ALL, block=128, sites_per_thread=1)
    path = str(tmp_path / "tune.txt")
    lq.tune(path)
    got = _run(U, lq.LQ_F64, 0.1, 2, ALL)
    assert np.array_equal(got, base)
    assert lq.tune_lookup(lq.LQ_F64, dims, ALL) is not None
    assert "stout" in open(path).read()


def test_16c32_ten_spatial_steps_f64(gpu):
    """16^3 x 32, links exp(i 0.3 H), 10 steps rho = 0.1 over the spatial
    directions, FP64: every link element against the oracle."""
    dims = (16, 16, 16, 32)
    U = fieldgen.near_identity_su3(dims, 1)
    ref = stout.stout_smear(U, 0.1, 10, SPATIAL)
    got = _run(U, lq.LQ_F64, 0.1, 10, SPATIAL)
    a, r = links_err(got, ref)
    assert a <= F64_TOL and r <= F64_TOL, (a, r)
    p_ref = gauge.plaquette(ref)
    f = upload_links(got, lq.LQ_F64)
    assert np.allclose(lq.plaquette(f), p_ref, rtol=0, atol=1e-13)


def test_48c96_six_steps(gpu):
    """48^3 x 96, exp(i 0.3 H) links, 6 steps rho = 0.125 in 4 dims, in the launch
    configuration the benchmark uses.  FP64: 32 sampled sites against the
    oracle run on periodic boxes of side 13 around them (6 steps reach at most
    6 sites in every direction, so the box centre is exact).  FP32: every
    element of the lattice against the FP64 result (compared on the device),
    and the sampled sites against the oracle."""
    import torch
    from tests.oracle_pool import stout_box_centers
    dims = (48, 48, 48, 96)
    n, rho = 6, 0.125
    Ut = fieldgen.near_identity_su3_torch(dims, 2, device="cuda")
    g = lq.Geometry(dims)
    U = Ut.cpu().numpy()
    del Ut
    torch.cuda.empty_cache()
    f64 = lq.Field(g, lq.LQ_LINKS, lq.LQ_F64)
    f64.upload(U)
    lq.stout_smear(f64, rho, n, ALL)
    f32 = lq.Field(g, lq.LQ_LINKS, lq.LQ_F32)
    f32.upload(U)
    lq.stout_smear(f32, rho, n, ALL)
    worst_all = 0.0
    for mu in range(4):   # |U32 - U64| per complex element, one direction at a time
        d = (f32.tensor[mu].double() - f64.tensor[mu]).pow(2).sum(-1).sqrt()
        worst_all = max(worst_all, float(d.max()))
        del d
    assert worst_all <= F32_TOL_48C96, worst_all
    rng = np.random.default_rng(5)
    sites = [[int(rng.integers(L)) for L in dims] for _ in range(32)]
    refs = stout_box_centers([lattice.sub_box(U, c, n) for c in sites], rho, n, ALL)
    got64, got32 = f64.download(), f32.download()
    w64 = max(float(np.max(np.abs(got64[c[3], c[2], c[1], c[0]] - r))) for c, r in zip(sites, refs))
    w32 = max(float(np.max(np.abs(got32[c[3], c[2], c[1], c[0]].astype(np.complex128) - r)))
              for c, r in zip(sites, refs))
    assert w64 <= F64_TOL, w64
    assert w32 <= F32_TOL_48C96, w32


@pytest.mark.parametrize("dims", [(1, 1, 1, 1), (1, 2, 1, 3), (2, 1, 1, 1), (1, 1, 5, 1)])
def test_degenerate_extents(gpu, dims):
    """Extents of 1 (x + mu = x - mu = x) and 2 in every combination."""
    U = fieldgen.haar_su3(dims, 109)
    ref = stout.stout_smear(U, 0.1, 2, ALL)
    got = _run(U, lq.LQ_F64, 0.1, 2, ALL)
    assert np.max(np.abs(got - ref)) <= F64_TOL
    f = upload_links(U, lq.LQ_F64)
    assert np.allclose(lq.plaquette(f), gauge.plaquette(U), rtol=0, atol=1e-14)


def _pure_gauge_links(dims, prec, seed):
    """U_mu(x) = g(x) g(x+mu)^dag with g(x) = diag(e^{i phi}, e^{-i phi}, 1), built on the
    device in the [dir][comp][site][re,im] layout; returns (tensor, field)."""
    import torch
    lx, ly, lz, lt = dims
    dt = torch.float64 if prec == lq.LQ_F64 else torch.float32
    gen = torch.Generator(device="cuda").manual_seed(seed)
    phi = (torch.rand((lt, lz, ly, lx), generator=gen, device="cuda", dtype=torch.float64) * 6.283185307179586)
    V = lx * ly * lz * lt
    t = torch.zeros((4, 9, V, 2), dtype=dt, device="cuda")
    for mu, axis in enumerate((3, 2, 1, 0)):
        d = (phi - torch.roll(phi, -1, dims=axis)).reshape(-1)
        c, s = torch.cos(d).to(dt), torch.sin(d).to(dt)
        t[mu, 0, :, 0], t[mu, 0, :, 1] = c, s
        t[mu, 4, :, 0], t[mu, 4, :, 1] = c, -s
        t[mu, 8, :, 0] = 1
        del d, c, s
    del phi
    g = lq.Geometry(dims)
    return t, lq.Field(g, lq.LQ_LINKS, prec, tensor=t)


@pytest.mark.parametrize("prec,dims", [(lq.LQ_F32, (128, 128, 128, 128)), (lq.LQ_F64, (128, 128, 128, 64))])
def test_largest_volumes_pure_gauge_fixed_point(gpu, prec, dims):
    """2^28 sites (FP32, 77 GB of links) and 2^27 sites (FP64, 77 GB): with the
    library's double buffer these are the largest powers of two that fit in HBM,
    and element offsets exceed 2^32.  A pure-gauge field is a fixed point of stout
    smearing (every staple equals U_mu(x), so Q = 0), has plaquette 1, and any wrong
    neighbour index would break both."""
    import torch
    t, f = _pure_gauge_links(dims, prec, 7)
    ref_planes = [t[mu, c].clone() for mu, c in ((0, 0), (3, 4))]
    lq.stout_smear(f, 0.1, 2, ALL)
    tol = 2e-6 if prec == lq.LQ_F32 else 1e-13
    for (mu, c), ref in zip(((0, 0), (3, 4)), ref_planes):
        assert torch.max(torch.abs(t[mu, c] - ref)).item() <= tol
    del ref_planes
    for mu in range(4):   # off-diagonal components stay exactly zero
        assert torch.count_nonzero(t[mu, 1]).item() == 0 and torch.count_nonzero(t[mu, 6]).item() == 0
    p = lq.plaquette(f)
    assert abs(p[0] - 1.0) <= (1e-6 if prec == lq.LQ_F32 else 1e-13)
    del f, t
    torch.cuda.empty_cache()
    lq.free_all()


@pytest.mark.parametrize("prec", [lq.LQ_F32, lq.LQ_F64])
@pytest.mark.parametrize("scale", [1.0, 1.02])
def test_reprojection(gpu, prec, scale):
    """FP64 re-projection after each step: links come out in SU(3) (rows
    orthonormal, det 1) whether the rows enter unitary to rounding (the
    polynomial normalisation) or 2 % off (the Newton path), and on unitary
    input it moves the FP32 links by no more than their rounding."""
    dims = (4, 3, 4, 5)
    U = fieldgen.near_identity_su3(dims, 710) * scale
    got = _run(U, prec, 0.1, 2, ALL, reproject=True).astype(np.complex128)
    du, dd = unitarity_violation(got)
    tol = 5e-7 if prec == lq.LQ_F32 else 1e-14
    assert du < tol and dd < tol, (du, dd)
    if scale == 1.0:
        plain = _run(U, prec, 0.1, 2, ALL, reproject=False).astype(np.complex128)
        assert np.max(np.abs(got - plain)) < (1e-6 if prec == lq.LQ_F32 else 1e-14)


def _gram_schmidt_f64(u):
    """FP64 Gram-Schmidt of rows 0 and 1, row 2 = conj(r0 x r1), of complex64 links."""
    m = u.astype(np.complex128)
    r0 = m[..., 0, :] / np.sqrt(np.sum(np.abs(m[..., 0, :]) ** 2, axis=-1))[..., None]
    r1 = m[..., 1, :] - np.sum(np.conj(r0) * m[..., 1, :], axis=-1)[..., None] * r0
    r1 = r1 / np.sqrt(np.sum(np.abs(r1) ** 2, axis=-1))[..., None]
    return np.stack([r0, r1, np.conj(np.cross(r0, r1))], axis=-2)


@pytest.mark.parametrize("gen,rho", [("near", 0.1), ("haar", 0.25)])
def test_fp32_reprojection_is_the_fp64_gram_schmidt(gpu, gen, rho):
    """One FP32 step with and without the re-projection: the re-projected links
    are the FP64 Gram-Schmidt of the others rounded to FP32, except elements
    whose exact value lies within ~1e-12 of an FP32 rounding boundary (the
    kernel applies the small corrections in FP32), which may differ by one
    unit in the last place."""
    dims = (8, 8, 8, 8)
    U = fieldgen.haar_su3(dims, 712) if gen == "haar" else fieldgen.near_identity_su3(dims, 712)
    plain = _run(U, lq.LQ_F32, rho, 1, ALL, reproject=False)
    got = _run(U, lq.LQ_F32, rho, 1, ALL, reproject=True)
    ref = _gram_schmidt_f64(plain).astype(np.complex64)
    differ = np.count_nonzero(got != ref)
    assert differ <= 1e-4 * got.size, differ
    ulp = np.spacing(np.maximum(np.abs(ref.real), np.abs(ref.imag)).astype(np.float32))
    assert np.all(np.abs(got.real - ref.real) <= ulp) and np.all(np.abs(got.imag - ref.imag) <= ulp)


@pytest.mark.parametrize("dims,gen,rho,n,dirs", [
    ((4, 4, 4, 4), "haar", 0.1, 1, ALL),
    ((3, 4, 5, 6), "near", 0.125, 3, ALL),
    ((3, 4, 5, 6), "near", 0.1, 2, SPATIAL),
    ((5, 3, 2, 7), "haar", 0.25, 2, (1, 3)),
    ((2, 2, 2, 2), "haar", 0.1, 2, ALL),
    ((4, 4, 4, 4), "haar", 0.4, 2, ALL),
])
def test_two_link_product_variant(gpu, dims, gen, rho, n, dirs):
    """Variant 3 (two-link products W_{mu nu}(y) = U_mu(y) U_nu(y+mu) formed
    once per step, staples from them) against the oracle and against the
    one-kernel step: the same staples with the products associated
    differently, so equal to rounding."""
    U = fieldgen.haar_su3(dims, 120) if gen == "haar" else fieldgen.near_identity_su3(dims, 120)
    ref = stout.stout_smear(U, rho, n, dirs)
    got = _run(U, lq.LQ_F64, rho, n, dirs, variant=3)
    a, r = links_err(got, ref)
    assert a <= F64_TOL and r <= F64_TOL, (a, r)
    assert np.max(np.abs(got - _run(U, lq.LQ_F64, rho, n, dirs, variant=1))) <= 1e-14
    got32 = _run(U, lq.LQ_F32, rho, n, dirs, variant=3)
    assert np.max(np.abs(got32.astype(np.complex128) - ref)) <= F32_TOL[gen]
    for mu in range(4):
        if mu not in dirs:
            assert np.array_equal(got[..., mu, :, :], U[..., mu, :, :])


def test_two_link_product_variant_in_graph(gpu):
    dims = (4, 3, 4, 5)
    U = fieldgen.near_identity_su3(dims, 121)
    a = _run(U, lq.LQ_F64, 0.1, 3, ALL, variant=3, use_graph=True)
    b = _run(U, lq.LQ_F64, 0.1, 3, ALL, variant=3)
    assert np.array_equal(a, b)
