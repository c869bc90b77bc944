"""GPU HYP force (lq_hyp_backward) vs the oracle's reverse-mode gradient
(oracle/hyp_force.py) and vs central finite differences of the GPU forward.

FP64: max |F_gpu - F_oracle| <= 1e-11 * max |F_oracle| (three projections
and their gradients per link and step, each at FP64 rounding times the
condition number of its V).  FP32 (FP32 staples, mixing and staple
gradients; FP64 projections and their gradients): <= 1e-4 * n * max |F|.
"""
import numpy as np
import pytest

import fieldgen
import paper_1105_2279_gb300 as lq
from oracle import gauge, hyp, hyp_force, lattice
from oracle.su3 import adj
from tests.gpu_util import upload_links

pytestmark = pytest.mark.gpu
W = (0.75, 0.6, 0.3)


def gpu_force(U, prec, weights, n, beta=6.0, seed=None, every=1):
    f = upload_links(U, prec)
    F = lq.Field(f.geom, lq.LQ_LINKS, prec)
    G = lq.Field(f.geom, lq.LQ_LINKS, prec)
    s = upload_links(seed, prec) if seed is not None else None
    lq.hyp_backward(f, *weights, n, F, grad_seed=s, beta=beta, grad_out=G, checkpoint_every=every)
    return F.download(), G.download()


@pytest.mark.parametrize("dims,gen,weights,n,every", [
    ((3, 4, 3, 4), "near", W, 0, 1),
    ((3, 4, 3, 4), "near", W, 1, 1),
    ((4, 3, 4, 3), "haar", W, 1, 1),
    ((3, 3, 4, 3), "near", (0.6, 0.5, 0.4), 2, 1),
    ((3, 4, 3, 3), "near", W, 3, 2),
    ((2, 2, 2, 2), "near", W, 1, 1),
])
def test_force_f64_matches_oracle(gpu, dims, gen, weights, n, every):
    U = fieldgen.haar_su3(dims, 500) if gen == "haar" else fieldgen.near_identity_su3(dims, 500)
    F_ref, G_ref = hyp_force.smeared_wilson_force(U, *weights, n, 6.0)
    F, G = gpu_force(U, lq.LQ_F64, weights, n, every=every)
    assert np.max(np.abs(F - F_ref)) <= 1e-11 * np.max(np.abs(F_ref))
    assert np.max(np.abs(G - G_ref)) <= 1e-11 * np.max(np.abs(G_ref))


def test_force_with_given_seed(gpu):
    dims = (3, 4, 3, 4)
    U = fieldgen.near_identity_su3(dims, 501)
    seed = fieldgen.haar_su3(dims, 502) * 0.7
    G_ref = hyp_force.hyp_backward(U, *W, 2, seed)
    _, G = gpu_force(U, lq.LQ_F64, W, 2, seed=seed)
    assert np.max(np.abs(G - G_ref)) <= 1e-11 * np.max(np.abs(G_ref))


def test_checkpoint_policies_agree_bitwise(gpu):
    dims = (3, 4, 3, 4)
    U = fieldgen.near_identity_su3(dims, 503)
    F1, G1 = gpu_force(U, lq.LQ_F64, W, 3, every=1)
    F2, G2 = gpu_force(U, lq.LQ_F64, W, 3, every=2)
    assert np.array_equal(F1, F2) and np.array_equal(G1, G2)


@pytest.mark.parametrize("n", [1, 2])
def test_force_f32(gpu, n):
    dims = (4, 3, 4, 3)
    U = fieldgen.near_identity_su3(dims, 504)
    F_ref, _ = hyp_force.smeared_wilson_force(U, *W, n, 6.0)
    F, _ = gpu_force(U, lq.LQ_F32, W, n)
    assert np.max(np.abs(F.astype(np.complex128) - F_ref)) <= 1e-4 * n * np.max(np.abs(F_ref))


def test_outer_level_alone_is_the_ape_force(gpu):
    """a2 = a3 = 0: the inner levels return the thin links, and the force is
    lq_ape_backward's with alpha = a1 (same projection gradient, different
    staple gathers)."""
    dims = (3, 4, 3, 4)
    U = fieldgen.near_identity_su3(dims, 505)
    F, _ = gpu_force(U, lq.LQ_F64, (0.7, 0.0, 0.0), 2)
    f = upload_links(U, lq.LQ_F64)
    Fa = lq.Field(f.geom, lq.LQ_LINKS, lq.LQ_F64)
    lq.ape_backward(f, 0.7, 2, (0, 1, 2, 3), Fa)
    assert np.max(np.abs(F - Fa.download())) <= 1e-12 * np.max(np.abs(F))


@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
def test_zero_weights_and_unit_field(gpu, prec):
    dims = (3, 4, 3, 4)
    U = fieldgen.haar_su3(dims, 506)
    F, _ = gpu_force(U, prec, (0.0, 0.0, 0.0), 2)
    f = upload_links(U, prec)
    F0 = lq.Field(f.geom, lq.LQ_LINKS, prec)
    lq.stout_backward(f, 0.1, 0, (0, 1, 2, 3), F0)
    tol = 1e-13 if prec == lq.LQ_F64 else 2e-5
    assert np.max(np.abs(F - F0.download())) <= tol * np.max(np.abs(F))
    Fu, _ = gpu_force(fieldgen.unit_links(dims), prec, W, 2)
    assert np.max(np.abs(Fu)) <= (1e-14 if prec == lq.LQ_F64 else 1e-6)


def test_autograd_chain_matches_oracle(gpu):
    dims = (3, 4, 3, 4)
    U = fieldgen.near_identity_su3(dims, 507)
    f = upload_links(U, lq.LQ_F64)
    t = f.tensor.clone().requires_grad_(True)
    S = lq.wilson_action_autograd(lq.hyp_smear_autograd(t, dims, *W, 2), dims, 6.0)
    S.backward()
    assert abs(S.item() - gauge.wilson_action(hyp.hyp_smear(U, *W, 2), 6.0)) < 1e-10
    g = t.grad.cpu().numpy()
    G = (g[..., 0] + 1j * g[..., 1]).transpose(2, 0, 1).reshape(lattice.field_shape(dims) + (4, 3, 3))
    _, G_ref = hyp_force.smeared_wilson_force(U, *W, 2, 6.0)
    assert np.max(np.abs(G - G_ref)) <= 1e-11 * np.max(np.abs(G_ref))


def test_rejects_bad_arguments(gpu):
    f = upload_links(fieldgen.unit_links((2, 2, 2, 2)), lq.LQ_F64)
    F = lq.Field(f.geom, lq.LQ_LINKS, lq.LQ_F64)
    with pytest.raises(lq.LqError):
        lq.hyp_backward(f, float("nan"), 0.6, 0.3, 1, F)
    with pytest.raises(lq.LqError):
        lq.hyp_backward(f, *W, -1, F)
    with pytest.raises(lq.LqError):
        lq.hyp_backward(f, *W, 1, f)


def _plane_diff_programs():
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


def test_16c32_two_steps_fd(gpu):
    """16^3 x 32, exp(i 0.3 H) links, 2 HYP steps (0.75, 0.6, 0.3), Wilson
    action beta = 6 of the smeared field: the FP64 GPU force against central
    finite differences of the GPU forward along random unit su(3) directions
    at 8 random links (step 1e-4: truncation ~1e-9 -> 2e-8)."""
    from scipy.linalg import expm
    dims = (16, 16, 16, 32)
    n, beta, e = 2, 6.0, 1e-4
    U = fieldgen.near_identity_su3(dims, 1)
    F, _ = gpu_force(U, lq.LQ_F64, W, n, beta=beta)
    g = lq.Geometry(dims)
    fp, fm = lq.Field(g, lq.LQ_LINKS, lq.LQ_F64), lq.Field(g, lq.LQ_LINKS, lq.LQ_F64)
    progs = _plane_diff_programs()
    rng = np.random.default_rng(46)
    worst = 0.0
    for _ in range(8):
        mu = int(rng.integers(4))
        x = tuple(int(rng.integers(L)) for L in lattice.field_shape(dims))
        X = fieldgen.su3_direction(rng)
        an = float(np.real(np.trace(adj(F[x + (mu,)]) @ X)))
        up, dn = U.copy(), U.copy()
        up[x + (mu,)] = expm(e * X) @ U[x + (mu,)]
        dn[x + (mu,)] = expm(-e * X) @ U[x + (mu,)]
        fp.upload(up)
        fm.upload(dn)
        lq.hyp_smear(fp, *W, n)
        lq.hyp_smear(fm, *W, n)
        d_retr = sum(lq.expr_eval(p, [fp, fm], reduce=True).real for p in progs) / 3.0
        fd = -(beta / 3.0) * d_retr / (2 * e)
        worst = max(worst, abs(fd - an) / max(1.0, abs(an)))
    assert worst < 2e-8, worst
