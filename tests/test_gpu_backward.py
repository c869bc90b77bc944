"""GPU stout force (lq_stout_backward) vs the oracle's reverse-mode gradient
and vs central finite differences of the GPU forward.

FP64: max |F_gpu - F_oracle| <= 1e-12 * max |F_oracle|, the FP64 target
(measured on GB300 over the cases below: <= 3.5e-14 for F, <= 3e-15 for G).  FP32 (FP32 matrix
algebra, FP64 coefficients): <= 2e-5 * max |F| per step.
"""
import numpy as np
import pytest

import fieldgen
import paper_1105_2279_gb300 as lq
from oracle import backward, gauge, lattice, stout
from oracle.su3 import adj
from tests.gpu_util import upload_links

pytestmark = pytest.mark.gpu
ALL, SPATIAL = (0, 1, 2, 3), (0, 1, 2)


def gpu_force(U, prec, rho, n, dirs, beta=6.0, seed=None, every=1):
    f = upload_links(U, prec)
    F = lq.Field(f.geom, lq.LQ_LINKS, prec)
    G = lq.Field(f.geom, lq.LQ_LINKS, prec)
    s = upload_links(seed, prec) if seed is not None else None
    lq.stout_backward(f, rho, n, dirs, F, grad_seed=s, beta=beta, grad_out=G, checkpoint_every=every)
    return F.download(), G.download()


@pytest.mark.parametrize("dims,gen,rho,n,dirs,every", [
    ((3, 4, 3, 4), "near", 0.1, 0, ALL, 1),
    ((3, 4, 3, 4), "near", 0.1, 1, ALL, 1),
    ((4, 3, 4, 3), "haar", 0.1, 2, ALL, 1),
    ((4, 3, 4, 3), "near", 0.125, 3, ALL, 2),
    ((3, 4, 5, 3), "near", 0.1, 3, SPATIAL, 1),
    ((4, 4, 3, 3), "haar", 0.2, 2, (0, 3), 3),
    ((2, 2, 2, 2), "near", 0.1, 2, ALL, 1),
])
def test_force_f64_matches_oracle(gpu, dims, gen, rho, n, dirs, every):
    U = fieldgen.haar_su3(dims, 300) if gen == "haar" else fieldgen.near_identity_su3(dims, 300)
    F_ref, G_ref = backward.smeared_wilson_force(U, rho, n, dirs, 6.0)
    F, G = gpu_force(U, lq.LQ_F64, rho, n, dirs, every=every)
    scale = np.max(np.abs(F_ref))
    assert np.max(np.abs(F - F_ref)) <= 1e-12 * scale
    assert np.max(np.abs(G - G_ref)) <= 1e-12 * np.max(np.abs(G_ref))


def test_force_with_given_seed(gpu):
    dims = (3, 4, 3, 4)
    U = fieldgen.near_identity_su3(dims, 301)
    seed = fieldgen.haar_su3(dims, 302) * 0.7      # any complex field works as dS/dU^(n)
    G_ref = backward.stout_backward(U, 0.1, 2, ALL, seed)
    _, G = gpu_force(U, lq.LQ_F64, 0.1, 2, ALL, seed=seed)
    assert np.max(np.abs(G - G_ref)) <= 1e-12 * np.max(np.abs(G_ref))


@pytest.mark.parametrize("eps", [0.02, 0.002])
def test_force_smooth_fields(gpu, eps):
    """Fields near the identity give |Q| ~ 6 rho eps, where the closed-form
    derivative coefficients of MP Sec. IV lose accuracy like 1e-16/|Q|^4
    (2e-9 relative at |Q| = 0.01); the gradient must stay at FP64 rounding."""
    dims = (3, 4, 3, 4)
    U = fieldgen.near_identity_su3(dims, 304, eps=eps)
    seed = fieldgen.haar_su3(dims, 305) * 0.7
    G_ref = backward.stout_backward(U, 0.1, 2, ALL, seed)
    _, G = gpu_force(U, lq.LQ_F64, 0.1, 2, ALL, seed=seed)
    assert np.max(np.abs(G - G_ref)) <= 1e-12 * np.max(np.abs(G_ref))


@pytest.mark.parametrize("n,dirs", [(1, ALL), (2, SPATIAL)])
def test_force_f32(gpu, n, dirs):
    dims = (4, 3, 4, 3)
    U = fieldgen.near_identity_su3(dims, 303)
    F_ref, _ = backward.smeared_wilson_force(U, 0.1, n, dirs, 6.0)
    F, _ = gpu_force(U, lq.LQ_F32, 0.1, n, dirs)
    assert np.max(np.abs(F.astype(np.complex128) - F_ref)) <= 2e-5 * max(1, n) * np.max(np.abs(F_ref))


def test_autograd_chain_matches_oracle(gpu):
    import torch
    dims = (3, 4, 3, 4)
    U = fieldgen.near_identity_su3(dims, 304)
    f = upload_links(U, lq.LQ_F64)
    t = f.tensor.clone().requires_grad_(True)
    S = lq.wilson_action_autograd(lq.stout_smear_autograd(t, dims, 0.1, 2, ALL), dims, 6.0)
    S.backward()
    assert abs(S.item() - gauge.wilson_action(stout.stout_smear(U, 0.1, 2, ALL), 6.0)) < 1e-10
    # tensor gradient [dir][comp][site][re/im] -> complex AoS
    g = t.grad.cpu().numpy()
    G = (g[..., 0] + 1j * g[..., 1]).transpose(2, 0, 1).reshape(lattice.field_shape(dims) + (4, 3, 3))
    _, G_ref = backward.smeared_wilson_force(U, 0.1, 2, ALL, 6.0)
    assert np.max(np.abs(G - G_ref)) <= 1e-12 * np.max(np.abs(G_ref))


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
    """24^3 x 48, exp(i 0.3 H) links, 3 steps rho = 0.1 in 4 dims, Wilson action
    beta = 6 of the smeared field: the FP64 GPU force against central finite
    differences along random unit su(3) directions at 32 random links (the
    action difference is formed per site and plane before summation), with
    step 1e-6 (rounding-limited: ~7e-9 absolute per-site noise summed over the
    ~4e4 changed plaquettes and divided by 2e-6 -> 5e-7) and step 1e-4
    (truncation ~1e-9 -> 2e-8), and against the oracle gradient at one link
    (periodic box of side 15: the force at a link depends on links at most
    2n+1 = 7 sites away)."""
    from scipy.linalg import expm
    dims = (24, 24, 24, 48)
    n, rho, beta = 3, 0.1, 6.0
    U = fieldgen.near_identity_su3(dims, 4)
    F, _ = gpu_force(U, lq.LQ_F64, rho, n, ALL, beta=beta, every=2)
    g = lq.Geometry(dims)
    fp, fm = lq.Field(g, lq.LQ_LINKS, lq.LQ_F64), lq.Field(g, lq.LQ_LINKS, lq.LQ_F64)
    progs = _plane_diff_programs()
    rng = np.random.default_rng(44)
    worst = {1e-6: 0.0, 1e-4: 0.0}
    for _ in range(32):
        mu = int(rng.integers(4))
        x = tuple(int(rng.integers(L)) for L in lattice.field_shape(dims))
        X = fieldgen.su3_direction(rng)
        an = float(np.real(np.trace(adj(F[x + (mu,)]) @ X)))
        for e in worst:
            up, dn = U.copy(), U.copy()
            up[x + (mu,)] = expm(e * X) @ U[x + (mu,)]
            dn[x + (mu,)] = expm(-e * X) @ U[x + (mu,)]
            fp.upload(up)
            fm.upload(dn)
            lq.stout_smear(fp, rho, n, ALL)
            lq.stout_smear(fm, rho, n, ALL)
            # each program stores (Re tr P+ - Re tr P-) * 1, whose trace is 3x the difference
            d_retr = sum(lq.expr_eval(p, [fp, fm], reduce=True).real for p in progs) / 3.0
            fd = -(beta / 3.0) * d_retr / (2 * e)
            worst[e] = max(worst[e], abs(fd - an) / max(1.0, abs(an)))
    assert worst[1e-6] < 5e-7 and worst[1e-4] < 2e-8, worst
    r = 2 * n + 1
    for _ in range(1):
        mu = int(rng.integers(4))
        c = [int(rng.integers(L)) for L in dims]
        box = lattice.sub_box(U, c, r)
        Fb, _ = backward.smeared_wilson_force(box, rho, n, ALL, beta)
        ref = Fb[r, r, r, r, mu]
        got = F[c[3], c[2], c[1], c[0], mu]
        assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_24c48_f32_force_vs_f64(gpu):
    dims = (24, 24, 24, 48)
    U = fieldgen.near_identity_su3(dims, 4)
    F64, _ = gpu_force(U, lq.LQ_F64, 0.1, 3, ALL)
    F32, _ = gpu_force(U, lq.LQ_F32, 0.1, 3, ALL)
    assert np.max(np.abs(F32.astype(np.complex128) - F64)) <= 6e-5 * np.max(np.abs(F64))


@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
def test_force_vanishes_on_unit_field(gpu, prec):
    """The unit field is a fixed point and a minimum of the Wilson action: the
    force through the smearing is zero (the Q -> 0 branch of the coefficients)."""
    U = fieldgen.unit_links((3, 4, 2, 3))
    F, G = gpu_force(U, prec, 0.1, 2, ALL)
    assert np.max(np.abs(F)) <= (1e-14 if prec == lq.LQ_F64 else 1e-6)


@pytest.mark.parametrize("prec", [lq.LQ_F64, lq.LQ_F32])
@pytest.mark.parametrize("with_seed", [False, True])
def test_checkpoint_policies_and_outputs_agree(gpu, prec, with_seed):
    """Every checkpoint policy recomputes the same U^(j) with the same kernels,
    so the force is bit-identical across them; the force alone and the
    gradient alone equal the outputs of a call that asks for both."""
    dims = (4, 3, 4, 3)
    U = fieldgen.near_identity_su3(dims, 303)
    seed = fieldgen.haar_su3(dims, 304) * 0.5 if with_seed else None
    F1, G1 = gpu_force(U, prec, 0.1, 4, ALL, seed=seed, every=1)
    for every in (2, 3, 5):
        F, G = gpu_force(U, prec, 0.1, 4, ALL, seed=seed, every=every)
        assert np.array_equal(F, F1) and np.array_equal(G, G1), every
    f = upload_links(U, prec)
    s = upload_links(seed, prec) if seed is not None else None
    F_only = lq.Field(f.geom, lq.LQ_LINKS, prec)
    lq.stout_backward(f, 0.1, 4, ALL, F_only, grad_seed=s, beta=6.0)
    G_only = lq.Field(f.geom, lq.LQ_LINKS, prec)
    lq.stout_backward(f, 0.1, 4, ALL, None, grad_seed=s, beta=6.0, grad_out=G_only)
    assert np.array_equal(F_only.download(), F1)
    assert np.array_equal(G_only.download(), G1)
