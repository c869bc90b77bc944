"""Secondary benchmark workloads of bench.py (each prints one JSON line):

* batch64    -- 64 independent lattices L^3 x 2L, L uniform in {8,12,16,20,24}
                (seed 3), 6 spatial stout steps rho = 0.1, FP32 links with FP64
                coefficients and re-projection: one persistent launch per step
                replayed as a CUDA graph, vs the same persistent sequence
                without a graph, vs one lq_stout_smear call per configuration.
* backward24 -- 24^3 x 48, 3 stout steps rho = 0.1 in 4 dims, gradient of the
                Wilson action (beta = 6) of the smeared field w.r.t. the thin
                links, FP64 and FP32, every step checkpointed vs recomputed.
* jacobi32   -- Jacobi smearing of Listing 1 (Sec. 6), the paper's own
                application: 32^3 x 64 (the largest lattice of the paper's
                Table 1), 20 iterations kappa = 0.21 over 4 directions, colour
                vector and 4-spin fermion, FP32; and 24^3 x 48 in FP64.
* micro16    -- 16^3 x 32, 10 spatial steps rho = 0.1 in FP64, and the fused
                expression micro-suite on the same field: sum_mu tr(U_mu(x)
                U_mu(x+mu)), U_mu(x) U_nu(x+mu)^dag, plaquette; the two
                programs interpreted and NVRTC-compiled.
* ape48      -- 48^3 x 96, 6 APE steps alpha = 0.5 in 4 dims, FP32 (FP64
                projection) and FP64.
* hyp32      -- 32^3 x 64, 2 HYP steps (0.75, 0.6, 0.3), FP32 (FP64
                projections) and FP64.
* apeforce24 -- 24^3 x 48, 3 APE steps alpha = 0.6 in 4 dims, gradient of the
                Wilson action (beta = 6) of the smeared field w.r.t. the thin
                links, FP64 and FP32 (FP64 projection and its gradient), every
                step checkpointed vs recomputed.
* hypforce24 -- 24^3 x 48, 2 HYP steps (0.75, 0.6, 0.3), gradient of the
                Wilson action (beta = 6) of the smeared field w.r.t. the thin
                links, FP64 and FP32 (FP64 projections and their gradients).
Inputs are resident on the device before timing; times are CUDA events.
"""
import json

import numpy as np


def _events(torch, fn, steps, warmup, reset=None):
    """Mean CUDA-event time of fn over `steps` calls after `warmup` calls; with
    `reset`, the inputs are restored before every call, outside its interval
    (smearing in place smooths a field, and a smoother field takes less FP64
    work in the coefficient series)."""
    for _ in range(warmup):
        if reset:
            reset()
        fn()
    torch.cuda.synchronize()
    if reset is None:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps
    total = 0.0
    for _ in range(steps):
        reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    return total / steps


def _dims(args, default):
    """--dims Lx,Ly,Lz,Lt overrides a workload's lattice (smaller profiling cases)."""
    return tuple(int(x) for x in args.dims.split(",")) if args.dims else default


def _precs(args, lq):
    """The (name, precision) legs to run: both by default, or the one --prec names."""
    legs = (("f64", lq.LQ_F64), ("f32", lq.LQ_F32))
    want = getattr(args, "prec", "both")
    return [leg for leg in legs if want in ("both", leg[0])]


def _field(lq, fieldgen, dims, seed, prec, device="cuda"):
    import torch
    U = fieldgen.near_identity_su3_torch(dims, seed, device=device).cpu().numpy()
    torch.cuda.empty_cache()
    return lq.Field.from_host(lq.Geometry(dims), lq.LQ_LINKS, prec, U), U


def _fp64_peak_tflops():
    import bench
    return 2.0 * bench.FP64_FMA_PER_CLK * 2070.0 * 1e6 / 1e12


def batch64(args, torch, lq, fieldgen):
    import bench
    from oracle import stout
    Ls = fieldgen.batch_sizes(3, 64)
    fields = []
    for i, L in enumerate(Ls):
        f, _ = _field(lq, fieldgen, (L, L, L, 2 * L), 3 + i, lq.LQ_F32)
        fields.append(f)
    orig = [f.tensor.clone() for f in fields]
    sites = sum(2 * L ** 4 for L in Ls)
    links = 6 * sites * 3
    dirs = (0, 1, 2)
    def restore():
        for f, o in zip(fields, orig):
            f.tensor.copy_(o)
    t_graph = _events(torch, lambda: lq.stout_smear_batch(fields, 0.1, 6, dirs, use_graph=True), args.steps,
                      args.warmup, reset=restore)
    t_plain = _events(torch, lambda: lq.stout_smear_batch(fields, 0.1, 6, dirs), args.steps, args.warmup,
                      reset=restore)

    def separate():
        for f in fields:
            lq.stout_smear(f, 0.1, 6, dirs)
    t_sep = _events(torch, separate, args.steps, args.warmup, reset=restore)
    # FP64 work of the coefficient stage on these inputs (series orders per link)
    tot = [0, 0, 0]
    for f, o in zip(fields, orig):
        f.tensor.copy_(o)
        st = lq.stout_ch_stats(f, 0.1, 6, dirs)
        tot = [a + b for a, b in zip(tot, st)]
    f64_flops = bench.ch_flops_per_link(tot) + bench.REPROJECT_FLOPS_PER_LINK
    peak = _fp64_peak_tflops()
    achieved = f64_flops * links / (t_graph * 1e-3) / 1e12
    # accuracy: one graph-replayed batch call against separate calls (bit for bit) and,
    # for the smallest lattice, against the FP64 oracle on the FP32-rounded input
    lq.stout_smear_batch(fields, 0.1, 6, dirs, use_graph=True)
    equal = True
    for f, o in zip(fields, orig):
        sep = lq.Field(f.geom, lq.LQ_LINKS, lq.LQ_F32)
        sep.tensor.copy_(o)
        lq.stout_smear(sep, 0.1, 6, dirs)
        equal = equal and bool(torch.equal(sep.tensor, f.tensor))
    i0 = int(np.argmin(Ls))
    src = lq.Field(fields[i0].geom, lq.LQ_LINKS, lq.LQ_F32)
    src.tensor.copy_(orig[i0])
    ref = stout.stout_smear(src.download().astype(np.complex128), 0.1, 6, dirs)
    err = float(np.max(np.abs(fields[i0].download().astype(np.complex128) - ref)))
    return {"metric": "stout link-updates/s (batch of 64 uneven lattices)", "value": links / (t_graph * 1e-3),
            "unit": "link-updates/s", "ms_per_step": t_graph, "dtype": "f32",
            "config": {"workload": "64 x L^3x2L, L in {8,12,16,20,24} seed 3, 6 spatial steps rho=0.1",
                       "L": Ls, "sites": sites},
            "persistent_no_graph": {"value": links / (t_plain * 1e-3), "ms_per_step": t_plain},
            "separate_calls": {"value": links / (t_sep * 1e-3), "ms_per_step": t_sep,
                               "launches_per_step": 64 * 6},
            "speedup_vs_separate": t_sep / t_graph,
            "roofline": {"bound": "alu", "pipe": "fp64", "unit": "TFLOP/s", "achieved": achieved, "peak": peak,
                         "frac": achieved / peak, "fp64_flops_per_link": f64_flops,
                         "peak_source": f"derived: {bench.FP64_FMA_PER_CLK} FP64 FMA/clk x 2 x 2070 MHz",
                         "ch_stats": tot},
            "accuracy": {"equal_to_separate_calls": equal,
                         "fp32_vs_oracle_max_abs": err,
                         "oracle_config": f"L={Ls[i0]} (config {i0}), FP64 oracle on the FP32-rounded input"}}


def _plane_diff_programs():
    """Per plane: Re tr P(operand 0) - Re tr P(operand 1) per site (the action
    difference of two fields formed before the sum over sites)."""
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


def backward_fd(lq, fieldgen, thin, F, rho, n, beta, n_links, eps=1e-4, seed=44):
    """Central finite differences of the smeared Wilson action along random
    unit su(3) directions at n_links random links (FP64 links on the device),
    against the force F (host array); returns the max relative difference."""
    from scipy.linalg import expm
    import torch
    g = thin.geom
    dims = g.dims
    fp, fm = lq.Field(g, lq.LQ_LINKS, lq.LQ_F64), lq.Field(g, lq.LQ_LINKS, lq.LQ_F64)
    progs = _plane_diff_programs()
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(n_links):
        mu = int(rng.integers(4))
        c = [int(rng.integers(L)) for L in dims]
        s = c[0] + dims[0] * (c[1] + dims[1] * (c[2] + dims[2] * c[3]))
        X = fieldgen.su3_direction(rng)
        t = thin.tensor[mu, :, s, :].cpu().numpy()
        u = (t[:, 0] + 1j * t[:, 1]).reshape(3, 3)
        an = float(np.real(np.trace(F[c[3], c[2], c[1], c[0], mu].conj().T @ X)))
        for fld, sign in ((fp, 1.0), (fm, -1.0)):
            fld.tensor.copy_(thin.tensor)
            w = (expm(sign * eps * X) @ u).reshape(9)
            fld.tensor[mu, :, s, 0] = torch.from_numpy(w.real.copy()).to(fld.tensor.device)
            fld.tensor[mu, :, s, 1] = torch.from_numpy(w.imag.copy()).to(fld.tensor.device)
            lq.stout_smear(fld, rho, n, (0, 1, 2, 3))
        d_retr = sum(lq.expr_eval(p, [fp, fm], reduce=True).real for p in progs) / 3.0
        fd = -(beta / 3.0) * d_retr / (2 * eps)
        worst = max(worst, abs(fd - an) / max(1.0, abs(an)))
    return worst


# Algorithmic flops per link of the backward (4 smeared directions), counted
# from its kernels: the local step (staple sum 2484, C and Omega 216, Q 20,
# Q^2 40, G_E 198, traces 148, M = a1 Q + a2 Q^2 + f1 H + f2 (QH + HQ) 684,
# G_Omega 30, exp(iQ) 70, E^dag G' 198, G_Omega^dag C 216, K 216), the
# factored six-term gather (3 directions x 2 groups x (2 products + 3
# accumulating products) = 6264), and in FP64 the coefficients with their
# derivatives: 35 + 48 + 24 per differentiated Horner step (2K + 4 steps for
# the links' series order K plus one, K read from lq.stout_ch_stats of the
# links themselves).
BWD_LOCAL_FLOPS = 2484 + 216 + 20 + 40 + 198 + 148 + 684 + 30 + 70 + 198 + 216 + 216
BWD_GATHER_FLOPS = 6264
WILSON_GRAD_FLOPS = 2484 + 18
FORCE_FLOPS = 198 + 30


def backward24(args, torch, lq, fieldgen):
    import bench
    dims = _dims(args, (24, 24, 24, 48))
    V = int(np.prod(dims))
    n, rho = 3, 0.1
    out = {"metric": "stout force link-updates/s (3 steps, Wilson action)", "unit": "link-updates/s",
           "config": {"workload": f"{'x'.join(map(str, dims))}, exp(i*0.3*H) links seed 4, 3 stout steps rho=0.1 in 4 dims, beta=6"}}
    forces = {}
    for name, prec in _precs(args, lq):
        f, _ = _field(lq, fieldgen, dims, 4, prec)
        F = lq.Field(f.geom, lq.LQ_LINKS, prec)
        stats = lq.stout_ch_stats(f, rho, n, (0, 1, 2, 3))
        g64 = lq.Field(f.geom, lq.LQ_LINKS, lq.LQ_F64)
        g64.upload(f.download().astype(np.complex128))
        stats64 = lq.stout_ch_stats(g64, rho, n, (0, 1, 2, 3))
        del g64
        mean_k = stats64[2] / max(1, stats64[1])
        # the derivative series runs at the links' own table order plus one:
        # 2K + 4 differentiated steps
        own_k = stats[2] / max(1, stats[1])
        ch_deriv = 35 + 48 + 24 * (2 * own_k + 4)
        fwd_f64 = bench.ch_flops_per_link(stats) + (bench.REPROJECT_FLOPS_PER_LINK if prec == lq.LQ_F32
                                                     else bench.MATRIX_FLOPS_PER_LINK)
        algebra = n * (BWD_LOCAL_FLOPS + BWD_GATHER_FLOPS) + WILSON_GRAD_FLOPS + FORCE_FLOPS
        algebra += 0 if prec == lq.LQ_F64 else n * bench.MATRIX_FLOPS_PER_LINK   # FP32 forward recompute
        flops64 = n * (ch_deriv + fwd_f64) + (algebra if prec == lq.LQ_F64 else 0)
        flops32 = 0 if prec == lq.LQ_F64 else algebra
        res = {}
        for every in (1, 3):
            t = _events(torch, lambda: lq.stout_backward(f, rho, n, (0, 1, 2, 3), F, beta=6.0, checkpoint_every=every),
                        args.steps, args.warmup)
            res[f"checkpoint_every_{every}"] = {"ms": t, "value": n * V * 4 / (t * 1e-3)}
        t1 = res["checkpoint_every_1"]["ms"] * 1e-3
        mhz = 2070.0
        p64 = 2.0 * bench.FP64_FMA_PER_CLK * mhz * 1e6
        p32 = 2.0 * bench.FP32_FMA_PER_CLK * mhz * 1e6
        res["roofline"] = {"bound": "alu", "pipe": "fp64", "unit": "TFLOP/s",
                           "fp64_flops_per_link": flops64, "fp32_flops_per_link": flops32,
                           "achieved": flops64 * 4 * V / t1 / 1e12, "peak": p64 / 1e12,
                           "frac": flops64 * 4 * V / t1 / p64,
                           "t_bound_ms": {"fp64": 1e3 * flops64 * 4 * V / p64, "fp32": 1e3 * flops32 * 4 * V / p32},
                           "peak_source": f"derived: {bench.FP64_FMA_PER_CLK} FP64 FMA/clk x 2 x {mhz:.0f} MHz",
                           "mean_series_order_fp64_table": mean_k, "mean_series_order_own_table": own_k,
                           "note": "checkpoint_every=1; flops of the forward recompute included"}
        g = lq.Field(f.geom, lq.LQ_LINKS, prec)

        res["forward_ms"] = _events(torch, lambda: lq.stout_smear(g, 0.1, 3, (0, 1, 2, 3)), args.steps,
                                    args.warmup, reset=lambda: g.tensor.copy_(f.tensor))
        res["forward_ms_note"] = "3 steps from the thin links (restored before every call, untimed)"
        lq.stout_backward(f, rho, n, (0, 1, 2, 3), F, beta=6.0)
        forces[name] = F.download()
        if name == "f64" and getattr(args, "fd_links", 4) > 0:
            res["fd_max_rel"] = backward_fd(lq, fieldgen, f, forces[name], rho, n, 6.0, args.fd_links)
            res["fd_config"] = f"central differences, step 1e-4, at {args.fd_links} random links (seed 44)"
        out[name] = res
    if "f32" in forces and "f64" in forces:
        scale = float(np.max(np.abs(forces["f64"])))
        out["accuracy"] = {"fp32_vs_fp64_force_max_rel": float(np.max(np.abs(
            forces["f32"].astype(np.complex128) - forces["f64"]))) / scale}
    first = "f64" if "f64" in out else "f32"
    out["value"] = out[first]["checkpoint_every_1"]["value"]
    out["dtype"] = first
    return out


# flops per site, spin and iteration: 8 colour matrix-vector products (66 each),
# 7 vector sums (6 each), the axpy (12); bytes: 4 links + chi + s0 read, chi written
JACOBI_FLOPS_PER_SPIN = 8 * 66 + 7 * 6 + 12


def jacobi32(args, torch, lq, fieldgen):
    import json as _json
    import os
    peaks = {}
    try:
        peaks = _json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    out = {"metric": "Jacobi smearing GFLOP/s (Listing 1)", "unit": "GFLOP/s",
           "config": {"workload": "Jacobi smearing, 20 iterations kappa=0.21, 4 dirs, exp(i*0.3*H) links",
                      "paper_table1_context": "GTX 480: 21.31 GFLOPS SP at 32^3x64, 7.91 DP at 24^3x48 (whole routine)"}}
    n_iter = 20
    for name, dims, prec in (("f32_32c64", (32, 32, 32, 64), lq.LQ_F32), ("f64_24c48", (24, 24, 24, 48), lq.LQ_F64)):
        V = int(np.prod(dims))
        fU, _ = _field(lq, fieldgen, dims, 5, prec)
        res = {}
        for kind, nspin in (("vector", 1), ("fermion", 4)):
            k = lq.LQ_COLOR_VECTOR if nspin == 1 else lq.LQ_FERMION
            chi = lq.Field(fU.geom, k, prec)
            chi.tensor.normal_()
            eb = 8 if prec == lq.LQ_F32 else 16
            flops = JACOBI_FLOPS_PER_SPIN * nspin * V * n_iter
            for packed in (False, True):
                t = _events(torch, lambda: lq.jacobi_smear(fU, chi, 0.21, n_iter, 1.0, compress_links=packed),
                            args.steps, args.warmup)
                # per iteration: each link (rows 0-1 only when packed) and chi, s0 read once, chi written;
                # packing reads rows 0-1 and writes them once per call
                bytes_site = 4 * (6 if packed else 9) * eb + 3 * 3 * nspin * eb
                total = bytes_site * V * n_iter + (2 * 4 * 6 * eb * V if packed else 0)
                res[kind + ("_compressed" if packed else "")] = {
                    "ms": t, "gflops": flops / (t * 1e-3) / 1e9, "gb_s": total / (t * 1e-3) / 1e9,
                    "hbm_frac": total / (t * 1e-3) / 1e9 / hbm}
        out[name] = res
    # thread geometry of Sec. 4.4 (the paper's Figs. 1-2 axes N_threads, N_site), FP32
    # colour vector on 32^3 x 64: every shape of the tuner's search space
    dims = (32, 32, 32, 64)
    V = int(np.prod(dims))
    fU, _ = _field(lq, fieldgen, dims, 5, lq.LQ_F32)
    chi = lq.Field(fU.geom, lq.LQ_COLOR_VECTOR, lq.LQ_F32)
    chi.tensor.normal_()
    flops = JACOBI_FLOPS_PER_SPIN * V * n_iter
    sweep = {}
    for block in (32, 64, 128, 256):
        for nsite in (1, 2, 4, 8):
            t = _events(torch, lambda: lq.jacobi_smear(fU, chi, 0.21, n_iter, 1.0, block=block,
                                                       sites_per_thread=nsite), args.steps, args.warmup)
            sweep[f"{block}x{nsite}"] = {"ms": t, "gflops": flops / (t * 1e-3) / 1e9}
    best = max(sweep, key=lambda k: sweep[k]["gflops"])
    out["thread_geometry_f32_32c64_vector"] = {"shapes": sweep, "best": best,
                                               "default_128x1_gflops": sweep["128x1"]["gflops"]}
    del fU, chi
    torch.cuda.empty_cache()
    # the lattices of the paper's Table 1, tuned launch shape, colour vector
    lq.tune(None)
    table = {}
    paper = {"8^3x16": (1.64, 1.49), "12^3x24": (6.53, 4.41), "16^3x32": (11.86, 6.26), "20^3x40": (16.56, 7.51),
             "24^3x48": (19.09, 7.91), "32^3x64": (21.31, None)}
    for L in (8, 12, 16, 20, 24, 32):
        dims = (L, L, L, 2 * L)
        V = int(np.prod(dims))
        row = {}
        for name, prec in (("f32", lq.LQ_F32), ("f64", lq.LQ_F64)):
            if L == 32 and prec == lq.LQ_F64:
                continue
            fU, _ = _field(lq, fieldgen, dims, 5, prec)
            chi = lq.Field(fU.geom, lq.LQ_COLOR_VECTOR, prec)
            chi.tensor.normal_()
            t = _events(torch, lambda: lq.jacobi_smear(fU, chi, 0.21, n_iter, 1.0), args.steps, args.warmup)
            row[name + "_gflops"] = JACOBI_FLOPS_PER_SPIN * V * n_iter / (t * 1e-3) / 1e9
        key = f"{L}^3x{2 * L}"
        row["paper_gtx480_sp_gflops"], row["paper_gtx480_dp_gflops"] = paper[key]
        table[key] = row
    out["table1_lattices"] = {"rows": table, "note": "colour vector, 20 iterations, tuned N_threads x N_site; the "
                                                      "paper's numbers are its whole routine on a GTX 480 (context)"}
    out["value"] = out["f32_32c64"]["vector"]["gflops"]
    out["dtype"] = "f32"
    return out


# FP64 flops per link of the APE projection, counted from csrc/ape.cu: A = V^dag V 108,
# eigenvalues and divided differences ~105, A^2 (Hermitian, compact) 40, X 30,
# W = V X 198, det V 60, cube root of the determinant phase ~40, W * phase 54 (the
# Newton refinements of 7 inverse square roots and 2 reciprocals are not counted);
# mixing 36 and the staple sum 2484 in the field precision.
APE_PROJECTION_FLOPS = 108 + 105 + 40 + 30 + 198 + 60 + 40 + 54
APE_MIX_FLOPS = 2484 + 36


def ape48(args, torch, lq, fieldgen):
    import bench
    dims, n, alpha = (48, 48, 48, 96), 6, 0.5
    V = int(np.prod(dims))
    links = n * V * 4
    out = {"metric": "APE link-updates/s", "unit": "link-updates/s",
           "config": {"workload": "48^3x96, exp(i*0.3*H) links seed 2, 6 APE steps alpha=0.5 in 4 dims"}}
    mhz = 2070.0
    p64 = 2.0 * bench.FP64_FMA_PER_CLK * mhz * 1e6
    for name, prec in (("f32", lq.LQ_F32), ("f64", lq.LQ_F64)):
        f, _ = _field(lq, fieldgen, dims, 2, prec)
        orig = f.tensor.clone()
        t = _events(torch, lambda: lq.ape_smear(f, alpha, n, (0, 1, 2, 3)), args.steps, args.warmup,
                    reset=lambda: f.tensor.copy_(orig))
        del orig
        f64_flops = APE_PROJECTION_FLOPS + (APE_MIX_FLOPS if prec == lq.LQ_F64 else 0)
        out[name] = {"ms": t, "value": links / (t * 1e-3),
                     "roofline": {"bound": "alu", "pipe": "fp64", "fp64_flops_per_link": f64_flops,
                                  "achieved": f64_flops * links / (t * 1e-3) / 1e12, "peak": p64 / 1e12,
                                  "frac": f64_flops * links / (t * 1e-3) / p64, "unit": "TFLOP/s",
                                  "note": "Newton refinements of square roots and reciprocals not counted"}}
        del f
        torch.cuda.empty_cache()
    out["value"] = out["f32"]["value"]
    out["dtype"] = "f32"
    return out


# HYP per site and step: level 3 12 links x (4 products + mixing 36), level 2
# 12 x (8 + 36), level 1 4 x (12 + 36) in the field precision (38.4 k flops),
# and 28 FP64 projections.
HYP_MIX_FLOPS_PER_SITE = 12 * (4 * 198 + 36) + 12 * (8 * 198 + 36) + 4 * (12 * 198 + 36)
HYP_PROJECTIONS_PER_SITE = 28


def hyp32(args, torch, lq, fieldgen):
    import bench
    dims, n = (32, 32, 32, 64), 2
    V = int(np.prod(dims))
    links = n * V * 4
    out = {"metric": "HYP link-updates/s", "unit": "link-updates/s",
           "config": {"workload": "32^3x64, exp(i*0.3*H) links seed 2, 2 HYP steps (0.75, 0.6, 0.3)"}}
    mhz = 2070.0
    p64 = 2.0 * bench.FP64_FMA_PER_CLK * mhz * 1e6
    for name, prec in (("f32", lq.LQ_F32), ("f64", lq.LQ_F64)):
        f, _ = _field(lq, fieldgen, dims, 2, prec)
        orig = f.tensor.clone()
        t = _events(torch, lambda: lq.hyp_smear(f, 0.75, 0.6, 0.3, n), args.steps, args.warmup,
                    reset=lambda: f.tensor.copy_(orig))
        del orig
        f64_site = HYP_PROJECTIONS_PER_SITE * APE_PROJECTION_FLOPS + (HYP_MIX_FLOPS_PER_SITE if prec == lq.LQ_F64
                                                                      else 0)
        ach = f64_site * V * n / (t * 1e-3)
        out[name] = {"ms": t, "value": links / (t * 1e-3),
                     "roofline": {"bound": "alu", "pipe": "fp64", "fp64_flops_per_link": f64_site / 4,
                                  "achieved": ach / 1e12, "peak": p64 / 1e12, "frac": ach / p64,
                                  "unit": "TFLOP/s",
                                  "note": "Newton refinements of square roots and reciprocals not counted"}}
        del f
        torch.cuda.empty_cache()
    out["value"] = out["f32"]["value"]
    out["dtype"] = "f32"
    return out


# Gradient of the projection per link (FP64): Im tr(G'^dag P) 90, G_W 90,
# Z = Herm(V^dag W) 210, invariants 8, two Hermitian inverses 180, p1 A + p3 12,
# Herm(V^dag G_W) 210, C = H N / 2 216, A C + C A 396, Z C, C Z, (Z C) Z 612,
# Y combination and Hermitian part 84, (G_W - 2 W Y) X 432, the two scaled
# outputs 36; plus the projection itself again (APE_PROJECTION_FLOPS).
APE_VJP_FLOPS = 90 + 90 + 210 + 8 + 180 + 12 + 210 + 216 + 396 + 612 + 84 + 432 + 36


def apeforce24(args, torch, lq, fieldgen):
    import bench
    dims = _dims(args, (24, 24, 24, 48))
    V = int(np.prod(dims))
    n, alpha = 3, 0.6
    out = {"metric": "APE force link-updates/s (3 steps, Wilson action)", "unit": "link-updates/s",
           "config": {"workload": f"{'x'.join(map(str, dims))}, exp(i*0.3*H) links seed 4, 3 APE steps alpha=0.6 in 4 dims, beta=6"}}
    mhz = 2070.0
    p64 = 2.0 * bench.FP64_FMA_PER_CLK * mhz * 1e6
    p32 = 2.0 * bench.FP32_FMA_PER_CLK * mhz * 1e6
    for name, prec in (("f64", lq.LQ_F64), ("f32", lq.LQ_F32)):
        f, _ = _field(lq, fieldgen, dims, 4, prec)
        F = lq.Field(f.geom, lq.LQ_LINKS, prec)
        # per link and step: forward recompute (mix + projection), backward link
        # kernel (mix + projection + its gradient), staple gather
        proj64 = 2 * APE_PROJECTION_FLOPS + APE_VJP_FLOPS
        algebra = n * (2 * APE_MIX_FLOPS + BWD_GATHER_FLOPS) + WILSON_GRAD_FLOPS + FORCE_FLOPS
        flops64 = n * proj64 + (algebra if prec == lq.LQ_F64 else 0)
        flops32 = 0 if prec == lq.LQ_F64 else algebra
        res = {}
        for every in (1, 3):
            t = _events(torch, lambda: lq.ape_backward(f, alpha, n, (0, 1, 2, 3), F, beta=6.0,
                                                       checkpoint_every=every), args.steps, args.warmup)
            res[f"checkpoint_every_{every}"] = {"ms": t, "value": n * V * 4 / (t * 1e-3)}
        t1 = res["checkpoint_every_1"]["ms"] * 1e-3
        res["roofline"] = {"bound": "alu", "pipe": "fp64", "unit": "TFLOP/s",
                           "fp64_flops_per_link": flops64, "fp32_flops_per_link": flops32,
                           "achieved": flops64 * 4 * V / t1 / 1e12, "peak": p64 / 1e12,
                           "frac": flops64 * 4 * V / t1 / p64,
                           "t_bound_ms": {"fp64": 1e3 * flops64 * 4 * V / p64, "fp32": 1e3 * flops32 * 4 * V / p32},
                           "peak_source": f"derived: {bench.FP64_FMA_PER_CLK} FP64 FMA/clk x 2 x {mhz:.0f} MHz",
                           "note": "checkpoint_every=1; flops of the forward recompute included; Newton "
                                   "refinements of square roots and reciprocals not counted"}
        g = lq.Field(f.geom, lq.LQ_LINKS, prec)
        res["forward_ms"] = _events(torch, lambda: lq.ape_smear(g, alpha, n, (0, 1, 2, 3)), args.steps, args.warmup,
                                    reset=lambda: g.tensor.copy_(f.tensor))
        out[name] = res
        del f, F, g
        torch.cuda.empty_cache()
    out["value"] = out["f64"]["checkpoint_every_1"]["value"]
    out["dtype"] = "f64"
    return out


# HYP force per site and step.  Field precision: the forward step of the
# checkpoint pass (HYP_MIX_FLOPS_PER_SITE), levels 3 and 2 recomputed in the
# gradient step (12 x (4 x 198 + 36) + 12 x (8 x 198 + 36)), the sums of
# levels 1, 2, 3 again in their gradient kernels (4 x (12 x 198 + 36) +
# 12 x (8 x 198 + 36) + 12 x (4 x 198 + 36)), the gathers (12 x 12 + 12 x 24 +
# 4 x 36 products).  FP64: 28 + 24 + 28 projections and 28 projection gradients.
HYPF_MIX_FLOPS_PER_SITE = (HYP_MIX_FLOPS_PER_SITE + 12 * (4 * 198 + 36) + 12 * (8 * 198 + 36)
                           + 4 * (12 * 198 + 36) + 12 * (8 * 198 + 36) + 12 * (4 * 198 + 36)
                           + (12 * 12 + 12 * 24 + 4 * 36) * 198)
HYPF_F64_FLOPS_PER_SITE = 80 * APE_PROJECTION_FLOPS + 28 * APE_VJP_FLOPS


def hypforce24(args, torch, lq, fieldgen):
    import bench
    dims, n, w = _dims(args, (24, 24, 24, 48)), 2, (0.75, 0.6, 0.3)
    V = int(np.prod(dims))
    out = {"metric": "HYP force link-updates/s (2 steps, Wilson action)", "unit": "link-updates/s",
           "config": {"workload": f"{'x'.join(map(str, dims))}, exp(i*0.3*H) links seed 4, 2 HYP steps (0.75, 0.6, 0.3), beta=6"}}
    mhz = 2070.0
    p64 = 2.0 * bench.FP64_FMA_PER_CLK * mhz * 1e6
    for name, prec in (("f64", lq.LQ_F64), ("f32", lq.LQ_F32)):
        f, _ = _field(lq, fieldgen, dims, 4, prec)
        F = lq.Field(f.geom, lq.LQ_LINKS, prec)
        t = _events(torch, lambda: lq.hyp_backward(f, *w, n, F, beta=6.0), args.steps, args.warmup)
        f64_site = n * (HYPF_F64_FLOPS_PER_SITE + (HYPF_MIX_FLOPS_PER_SITE if prec == lq.LQ_F64 else 0))
        ach = f64_site * V / (t * 1e-3)
        g = lq.Field(f.geom, lq.LQ_LINKS, prec)
        tf = _events(torch, lambda: lq.hyp_smear(g, *w, n), args.steps, args.warmup,
                     reset=lambda: g.tensor.copy_(f.tensor))
        out[name] = {"ms": t, "value": n * V * 4 / (t * 1e-3), "forward_ms": tf,
                     "roofline": {"bound": "alu", "pipe": "fp64", "fp64_flops_per_link": f64_site / (4 * n),
                                  "achieved": ach / 1e12, "peak": p64 / 1e12, "frac": ach / p64, "unit": "TFLOP/s",
                                  "note": "every step checkpointed; Newton refinements of square roots and "
                                          "reciprocals not counted"}}
        del f, F, g
        torch.cuda.empty_cache()
    out["value"] = out["f64"]["value"]
    out["dtype"] = "f64"
    return out


def micro16(args, torch, lq, fieldgen):
    dims = (16, 16, 16, 32)
    V = int(np.prod(dims))
    f, U = _field(lq, fieldgen, dims, 1, lq.LQ_F64)
    g = lq.Field(f.geom, lq.LQ_LINKS, lq.LQ_F64)
    t_smear = _events(torch, lambda: lq.stout_smear(g, 0.1, 10, (0, 1, 2)), args.steps, args.warmup,
                      reset=lambda: g.tensor.copy_(f.tensor))
    p_tr = []
    for mu in range(4):
        p_tr += [("loadl", 0, 0, mu, 0, 0), ("loadl", 1, 0, mu, mu, +1), ("mul", 2, 0, 1)]
        p_tr += [("add", 3, 3, 2)] if mu else [("add", 3, 2, 2), ("sub", 3, 3, 2)]
    p_tr += [("store", 3)]
    p_adj = [("loadl", 0, 0, 0, 0, 0), ("loadl", 1, 0, 1, 0, +1), ("adj", 2, 1), ("mul", 3, 0, 2), ("store", 3)]
    out = lq.Field(f.geom, lq.LQ_COLOR_MATRIX, lq.LQ_F64)
    t_tr = _events(torch, lambda: lq.expr_eval(p_tr, [f], reduce=True), args.steps, args.warmup)
    t_adj = _events(torch, lambda: lq.expr_eval(p_adj, [f], out=out), args.steps, args.warmup)
    t_plaq = _events(torch, lambda: lq.plaquette(f), args.steps, args.warmup)
    lq.expr_eval_jit(p_tr, [f], reduce=True)          # compile once (not timed)
    lq.expr_eval_jit(p_adj, [f], out=out)
    t_tr_jit = _events(torch, lambda: lq.expr_eval_jit(p_tr, [f], reduce=True), args.steps, args.warmup)
    t_adj_jit = _events(torch, lambda: lq.expr_eval_jit(p_adj, [f], out=out), args.steps, args.warmup)
    links = 10 * V * 3
    # accuracy against the oracle: spatial smearing never leaves a time slice
    # (staples over x, y, z only), so the oracle on single slices (periodic
    # 16^3 x 1 lattices) is exact for them; the micro-suite sums on the whole field
    from oracle import expr as oexpr, gauge, stout
    g.tensor.copy_(f.tensor)
    lq.stout_smear(g, 0.1, 10, (0, 1, 2))
    got = g.download()
    e_smear = 0.0
    for t in (0, 17):
        ref = stout.stout_smear(U[t:t + 1], 0.1, 10, (0, 1, 2))
        e_smear = max(e_smear, float(np.max(np.abs(got[t:t + 1] - ref))))
    tr_gpu = lq.expr_eval(p_tr, [f], reduce=True)
    tr_ref = oexpr.trace_sum(oexpr.eval_program(p_tr, [U]))
    plaq_ref = gauge.plaquette(U)[0]
    accuracy = {"smear_vs_oracle_max_abs": e_smear, "smear_oracle_sample": "time slices t=0 and t=17 (exact)",
                "trace_sum_rel": abs(tr_gpu - tr_ref) / abs(tr_ref),
                "plaquette_abs": abs(lq.plaquette(f)[0] - plaq_ref)}
    return {"metric": "stout link-updates/s (16^3x32, 10 spatial steps, FP64)", "value": links / (t_smear * 1e-3),
            "accuracy": accuracy,
            "unit": "link-updates/s", "ms_per_step": t_smear, "dtype": "f64",
            "config": {"workload": "16^3x32, exp(i*0.3*H) links seed 1, 10 stout steps rho=0.1 spatial"},
            "micro_suite_ms": {"trace_sum_mu_tr_UU_shift": t_tr, "shifted_adjoint_product": t_adj,
                               "plaquette": t_plaq, "trace_sum_jit": t_tr_jit, "shifted_adjoint_product_jit": t_adj_jit},
            "micro_suite_gb_s": {"trace_sum": V * 4 * 2 * 144 / (t_tr * 1e-3) / 1e9 / 2,
                                 "shifted_adjoint_product": V * (2 * 144 + 144) / (t_adj * 1e-3) / 1e9}}


def run(args):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import fieldgen
    import paper_1105_2279_gb300 as lq
    torch.cuda.set_device(0)
    fn = {"batch64": batch64, "backward24": backward24, "micro16": micro16, "jacobi32": jacobi32,
          "ape48": ape48, "hyp32": hyp32, "apeforce24": apeforce24,
          "hypforce24": hypforce24}[args.workload]
    res = fn(args, torch, lq, fieldgen)
    res.update({"n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                "data": "synthetic", "workload_mode": args.workload})
    print(json.dumps(res), flush=True)
