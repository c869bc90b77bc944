"""GPU APE force (lq_ape_backward) vs the oracle's reverse-mode gradient
(oracle/ape_force.py: Daleckii-Krein in numpy's eigenbasis, where the CUDA
path solves a Lyapunov equation in closed form) and vs central finite
differences of the GPU forward.

FP64: max |F_gpu - F_oracle| <= 1e-11 * max |F_oracle|, as for the stout
force (the projection's gradient adds ~20 products per link at rounding
1e-16 each, times the condition number of V, below 10 on these fields).
FP32 (FP32 staples and mixing, FP64 projection and its gradient):
<= 3e-5 * n * max |F|.
"""
import numpy as np
import pytest

import fieldgen
import paper_1105_2279_gb300 as lq
from oracle import ape, ape_force, gauge, lattice
from oracle.su3 import adj
from tests.gpu_util import upload_links

pytestmark = pytest.mark.gpu
ALL, SPATIAL = (0, 1, 2, 3), (0, 1, 2)


def gpu_force(U, prec, alpha, n, dirs, beta=6.0, seed=None, every=1):
    f = upload_links(U, prec)
    F = lq.Field(f.geom, lq.LQ_LINKS, prec)
    G = lq.Field(f.geom, lq.LQ_LINKS, prec)
    s = upload_links(seed, prec) if seed is not None else None
    lq.ape_backward(f, alpha, n, dirs, F, grad_seed=s, beta=beta, grad_out=G, checkpoint_every=every)
    return F.download(), G.download()


@pytest.mark.parametrize("dims,gen,alpha,n,dirs,every", [
    ((3, 4, 3, 4), "near", 0.6, 0, ALL, 1),
    ((3, 4, 3, 4), "near", 0.6, 1, ALL, 1),
    ((4, 3, 4, 3), "haar", 0.5, 2, ALL, 1),
    ((4, 3, 4, 3), "near", 0.7, 3, ALL, 2),
    ((3, 4, 5, 3), "near", 0.6, 3, SPATIAL, 1),
    ((4, 4, 3, 3), "haar", 0.45, 2, (0, 3), 3),
    ((2, 2, 2, 2), "near", 0.6, 2, ALL, 1),
    ((3, 2, 4, 3), "near", 0.6, 2, (2,), 1),
])
def test_force_f64_matches_oracle(gpu, dims, gen, alpha, n, dirs, every):
    U = fieldgen.haar_su3(dims, 400) if gen == "haar" else fieldgen.near_identity_su3(dims, 400)
    F_ref, G_ref = ape_force.smeared_wilson_force(U, alpha, n, dirs, 6.0)
    F, G = gpu_force(U, lq.LQ_F64, alpha, n, dirs, every=every)
    assert np.max(np.abs(F - F_ref)) <= 1e-11 * np.max(np.abs(F_ref))
    assert np.max(np.abs(G - G_ref)) <= 1e-11 * np.max(np.abs(G_ref))


def test_force_with_given_seed(gpu):
    dims = (3, 4, 3, 4)
    U = fieldgen.near_identity_su3(dims, 401)
    seed = fieldgen.haar_su3(dims, 402) * 0.7      # any complex field works as dS/dU^(n)
    G_ref = ape_force.ape_backward(U, 0.6, 2, ALL, seed)
    _, G = gpu_force(U, lq.LQ_F64, 0.6, 2, ALL, seed=seed)
    assert np.max(np.abs(G - G_ref)) <= 1e-11 * np.max(np.abs(G_ref))


def test_checkpoint_policies_agree_bitwise(gpu):
    """Recomputed steps run the same kernels on the same inputs."""
    dims = (4, 3, 4, 3)
    U = fieldgen.near_identity_su3(dims, 403)
    F1, G1 = gpu_force(U, lq.LQ_F64, 0.6, 4, ALL, every=1)
    F3, G3 = gpu_force(U, lq.LQ_F64, 0.6, 4, ALL, every=3)
    assert np.array_equal(F1, F3) and np.array_equal(G1, G3)


@pytest.mark.parametrize("n,dirs", [(1, ALL), (2, SPATIAL)])
def test_force_f32(gpu, n, dirs):
    dims = (4, 3, 4, 3)
    U = fieldgen.near_identity_su3(dims, 404)
    F_ref, _ = ape_force.smeared_wilson_force(U, 0.6, n, dirs, 6.0)
    F, _ = gpu_force(U, lq.LQ_F32, 0.6, n, dirs)
    assert np.max(np.abs(F.astype(np.complex128) - F_ref)) <= 3e-5 * n * np.max(np.abs(F_ref))


@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
def test_links_left_in_place_give_the_wilson_force(gpu, prec):
    """alpha = 0 keeps every link (P(U) = U on SU(3)): the force is the thin
    field's Wilson force, here from lq_stout_backward with n = 0."""
    dims = (3, 4, 3, 4)
    U = fieldgen.haar_su3(dims, 405)
    F, _ = gpu_force(U, prec, 0.0, 2, ALL)
    f = upload_links(U, prec)
    F0 = lq.Field(f.geom, lq.LQ_LINKS, prec)
    lq.stout_backward(f, 0.1, 0, ALL, F0)
    tol = 1e-13 if prec == lq.LQ_F64 else 2e-5
    assert np.max(np.abs(F - F0.download())) <= tol * np.max(np.abs(F))


@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
def test_force_vanishes_on_unit_field(gpu, prec):
    U = fieldgen.unit_links((3, 4, 2, 3))
    F, _ = gpu_force(U, prec, 0.6, 2, ALL)
    assert np.max(np.abs(F)) <= (1e-14 if prec == lq.LQ_F64 else 1e-6)


def test_autograd_chain_matches_oracle(gpu):
    dims = (3, 4, 3, 4)
    U = fieldgen.near_identity_su3(dims, 406)
    f = upload_links(U, lq.LQ_F64)
    t = f.tensor.clone().requires_grad_(True)
    S = lq.wilson_action_autograd(lq.ape_smear_autograd(t, dims, 0.6, 2, ALL), dims, 6.0)
    S.backward()
    assert abs(S.item() - gauge.wilson_action(ape.ape_smear(U, 0.6, 2, ALL), 6.0)) < 1e-10
    g = t.grad.cpu().numpy()
    G = (g[..., 0] + 1j * g[..., 1]).transpose(2, 0, 1).reshape(lattice.field_shape(dims) + (4, 3, 3))
    _, G_ref = ape_force.smeared_wilson_force(U, 0.6, 2, ALL, 6.0)
    assert np.max(np.abs(G - G_ref)) <= 1e-11 * np.max(np.abs(G_ref))


def test_rejects_bad_arguments(gpu):
    f = upload_links(fieldgen.unit_links((2, 2, 2, 2)), lq.LQ_F64)
    F = lq.Field(f.geom, lq.LQ_LINKS, lq.LQ_F64)
    with pytest.raises(lq.LqError):
        lq.ape_backward(f, float("nan"), 1, ALL, F)
    with pytest.raises(lq.LqError):
        lq.ape_backward(f, 0.6, -1, ALL, F)
    with pytest.raises(lq.LqError):
        lq.ape_backward(f, 0.6, 1, ALL, None)
    with pytest.raises(lq.LqError):
        lq.ape_backward(f, 0.6, 1, ALL, f)
    F32 = lq.Field(f.geom, lq.LQ_LINKS, lq.LQ_F32)
    with pytest.raises(lq.LqError):
        lq.ape_backward(f, 0.6, 1, ALL, F32)


def _plane_diff_programs():
    """Per plane: Re tr P(operand 0) - Re tr P(operand 1), summed per site before reduction."""
    progs = []
    for mu in range(4):
        for nu in range(mu + 1, 4):
            p = []
            for k, r0 in ((0, 0), (1, 4)):
                p += [("loadl", r0, k, mu, 0, 0), ("loadl", r0 + 1, k, nu, mu, +1), ("mul", r0, r0, r0 + 1),
                      ("loadl", r0 + 1, k, nu, 0, 0), ("loadl", r0 + 2, k, mu, nu, +1),
                      ("mul", r0 + 1, r0 + 1, r0 + 2), ("adj", r0 + 1, r0 + 1), ("mul", r0, r0, r0 + 1),
                      ("retr", r0, r0)]
            p += [("sub", 0, 0, 4), ("store", 0)]
            progs.append(p)
    return progs


def test_24c48_three_steps_fd_and_oracle(gpu):
    """24^3 x 48, exp(i 0.3 H) links, 3 APE steps alpha = 0.6 in 4 dims, Wilson
    action beta = 6 of the smeared field: the FP64 GPU force against central
    finite differences of the GPU forward along random unit su(3) directions
    at 16 random links (step 1e-4: truncation ~1e-9 -> 2e-8; the action
    difference is formed per site and plane before summation), and against
    the oracle gradient at one link (periodic box of side 15: the force at a
    link depends on links at most 2n+1 = 7 sites away)."""
    from scipy.linalg import expm
    dims = (24, 24, 24, 48)
    n, alpha, beta = 3, 0.6, 6.0
    U = fieldgen.near_identity_su3(dims, 4)
    F, _ = gpu_force(U, lq.LQ_F64, alpha, n, ALL, beta=beta, every=2)
    g = lq.Geometry(dims)
    fp, fm = lq.Field(g, lq.LQ_LINKS, lq.LQ_F64), lq.Field(g, lq.LQ_LINKS, lq.LQ_F64)
    progs = _plane_diff_programs()
    rng = np.random.default_rng(45)
    worst, e = 0.0, 1e-4
    for _ in range(16):
        mu = int(rng.integers(4))
        x = tuple(int(rng.integers(L)) for L in lattice.field_shape(dims))
        X = fieldgen.su3_direction(rng)
        an = float(np.real(np.trace(adj(F[x + (mu,)]) @ X)))
        up, dn = U.copy(), U.copy()
        up[x + (mu,)] = expm(e * X) @ U[x + (mu,)]
        dn[x + (mu,)] = expm(-e * X) @ U[x + (mu,)]
        fp.upload(up)
        fm.upload(dn)
        lq.ape_smear(fp, alpha, n, ALL)
        lq.ape_smear(fm, alpha, n, ALL)
        d_retr = sum(lq.expr_eval(p, [fp, fm], reduce=True).real for p in progs) / 3.0
        fd = -(beta / 3.0) * d_retr / (2 * e)
        worst = max(worst, abs(fd - an) / max(1.0, abs(an)))
    assert worst < 2e-8, worst
    r = 2 * n + 1
    mu = int(rng.integers(4))
    c = [int(rng.integers(L)) for L in dims]
    box = lattice.sub_box(U, c, r)
    Fb, _ = ape_force.smeared_wilson_force(box, alpha, n, ALL, beta)
    ref = Fb[r, r, r, r, mu]
    got = F[c[3], c[2], c[1], c[0], mu]
    assert np.max(np.abs(got - ref)) <= 1e-11 * max(1.0, np.max(np.abs(ref)))


def test_24c48_f32_force_vs_f64(gpu):
    dims = (24, 24, 24, 48)
    U = fieldgen.near_identity_su3(dims, 4)
    F64, _ = gpu_force(U, lq.LQ_F64, 0.6, 3, ALL)
    F32, _ = gpu_force(U, lq.LQ_F32, 0.6, 3, ALL)
    assert np.max(np.abs(F32.astype(np.complex128) - F64)) <= 1e-4 * np.max(np.abs(F64))
