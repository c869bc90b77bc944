"""Stout-smearing benchmark: link-updates/s on one GB300, FP32 (FP64
Cayley-Hamilton coefficients and re-projection) beside FP64.

Workload: 48^3 x 96 periodic lattice (10,616,832 sites), links exp(i 0.3 H)
with H random traceless Hermitian (seeded), 6 stout steps rho = 0.125 in all
4 directions followed by the FP64-accumulated plaquette.  One bench step =
that whole sequence on device-resident links; every step smears the same thin
links, restored by a device copy before the step and outside its CUDA-event
interval (the Cayley-Hamilton coefficients' series order, and with it the
FP64 work per link, falls as a field gets smoother: smearing the previous
output again would time an easier workload).  The 3 GB (FP32) / 6 GB (FP64)
link fields are far larger than the 129 MB L2, so no L2 flush is needed
between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun with N > 1 every rank smears
its own independent lattice (weak scaling, no data-path collective).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (48, 48, 48, 96)
N_SMEAR = 6
RHO = 0.125
DIRS = (0, 1, 2, 3)
SEED = 2
WORKLOAD = "48^3x96 periodic, exp(i*0.3*H) links seed 2, 6 stout steps rho=0.125 in 4 dirs + plaquette"
METRIC = "stout link-updates/s"

# Algorithmic counts per link update (4 smeared directions):
# minimum traffic = read every link once + write every updated link once;
# flops of the staple / Omega / Q / exp / U' matrix algebra, and of the FP64
# Cayley-Hamilton coefficients (+ FP64 re-projection in the FP32 path).
BYTES_PER_LINK = {"f32": 144.0, "f64": 288.0}
MATRIX_FLOPS_PER_LINK = 3019.0
# FP64 part of the FP32 links' re-projection: the two row norms (12 + 12), the
# row overlap (22) and the row-2 cross product with its FP32 correction
# folded into the accumulator (48); the corrections themselves are FP32
# (REPROJECT_FP32_FLOPS_PER_LINK: scale factors 14, rows 0 and 1 48, the two
# FP32 cross products and the correction of row 2 96).
REPROJECT_FLOPS_PER_LINK = 94.0
REPROJECT_FP32_FLOPS_PER_LINK = 158.0
# Cayley-Hamilton coefficients: c0 = det Q and c1 = tr(Q^2)/2 of Q made
# traceless by d2 = -(d0 + d1) (1 + 9 for the |Q_jk|^2 + 6 + 19 = 35 flops), then
# either the closed form (179 more) or the reduced Taylor series of degree
# 2K+1 by Horner's rule (14 per pair of terms: 14 (K-1) + 7).  K depends on
# c1, so the average is counted on the workload itself (lq.stout_ch_stats).
CH_PREAMBLE_FLOPS = 35.0
CH_CLOSED_FORM_FLOPS = 214.0


def ch_flops_per_link(stats):
    """Average FP64 flops of the coefficient stage from (updates, series updates, sum of K)."""
    n, n_series, sum_k = stats
    if n == 0:
        return CH_CLOSED_FORM_FLOPS
    series = n_series * (CH_PREAMBLE_FLOPS + 7.0 - 14.0) + 14.0 * sum_k
    return ((n - n_series) * CH_CLOSED_FORM_FLOPS + series) / n
# GB300 unit counts: 152 SMs x 2 FP64 FMA lanes (304 per cycle) and x 128 FP32 FMA lanes.
FP64_FMA_PER_CLK = 304
FP32_FMA_PER_CLK = 152 * 128
# Small-case (32^3x64) ncu DRAM bytes per launch of each step kernel divided by its
# 8,388,608 link updates, times the 42,467,328 link updates of one 48^3x96 launch
# (traffic grows in proportion to the links); see profiles/.
TRAFFIC_BYTES_PER_LINK_F32 = (634004224 + 582413824) / 8388608.0
TRAFFIC_BYTES_PER_LINK_F64 = (2151617000 + 1189766000) / 8388608.0


# The two-link product variant (3) forms each U_mu(y) U_nu(y+mu) once: 9 staple
# products per link instead of 12, for W written once and read once per link
# on top of the links (12 colour matrices per site over 4 links).
W_SAVED_FLOPS_PER_LINK = 3 * 198.0
W_BYTES_PER_LINK = {"f32": 2 * 3 * 72.0, "f64": 2 * 3 * 144.0}


def roofline(kernel_ms, links, prec, hbm_gbs, sm_mhz, ch_flops, variant=1):
    """Roofline of one step (its one or two kernel launches): time bound of each
    resource from the algorithmic counts, the binding one reported as achieved / peak."""
    matrix = MATRIX_FLOPS_PER_LINK - (W_SAVED_FLOPS_PER_LINK if variant == 3 else 0.0)
    f64_flops = ch_flops + (REPROJECT_FLOPS_PER_LINK if prec == "f32" else matrix)
    f32_flops = matrix + REPROJECT_FP32_FLOPS_PER_LINK if prec == "f32" else 0.0
    nbytes = BYTES_PER_LINK[prec] + (W_BYTES_PER_LINK[prec] if variant == 3 else 0.0)
    p64 = 2.0 * FP64_FMA_PER_CLK * sm_mhz * 1e6
    p32 = 2.0 * FP32_FMA_PER_CLK * sm_mhz * 1e6
    t = {"hbm": nbytes * links / (hbm_gbs * 1e9), "fp64": f64_flops * links / p64,
         "fp32": f32_flops * links / p32}
    sec = kernel_ms * 1e-3
    ach64 = f64_flops * links / sec / 1e12
    # ncu DRAM counts were taken on the one-kernel step
    traffic = None if variant != 1 else (
        (TRAFFIC_BYTES_PER_LINK_F32 if prec == "f32" else TRAFFIC_BYTES_PER_LINK_F64) * links)
    return {"bound": "alu", "pipe": "fp64", "achieved": ach64, "peak": p64 / 1e12, "unit": "TFLOP/s",
            "frac": ach64 / (p64 / 1e12), "traffic": traffic,
            "peak_source": f"derived: {FP64_FMA_PER_CLK} FP64 FMA/clk x 2 flops x {sm_mhz:.0f} MHz median SM clock",
            "fp64_flops_per_link": f64_flops, "ch_flops_per_link": ch_flops, "fp32_flops_per_link": f32_flops,
            "bytes_per_link": nbytes, "kernel_ms": kernel_ms,
            "t_bound_ms": {k: 1e3 * v for k, v in t.items()},
            "hbm_frac": nbytes * links / sec / 1e9 / hbm_gbs}


def peaks():
    p = {}
    try:
        p = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    return p


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value, dist, device="cuda"):
    """The largest `value` over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank, world, seconds):
    """Whole-job throughput: every rank processes units_per_rank in `seconds` (max over ranks)."""
    return world * units_per_rank / seconds


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def time_oracle_sample(n_steps=1, dims=(16, 16, 16, 32)):
    """Times the FP64 oracle on a bounded sample of the workload (same rho, dirs, generator)."""
    import fieldgen
    from oracle import stout
    U = fieldgen.near_identity_su3(dims, SEED)
    t0 = time.perf_counter()
    stout.stout_smear(U, RHO, n_steps, DIRS)
    dt = time.perf_counter() - t0
    links = n_steps * int(np.prod(dims)) * len(DIRS)
    return links / dt, dt, links


def _pool_noop(i):
    return i


def _oracle_slab_step(task):
    """One FP64 oracle stout step of the t-slices [t0, t1) of a lattice held in
    shared memory: the slab plus one halo slice on each side is smeared as a
    lattice of its own (a step reads neighbours one slice away, so its
    interior slices are exact) and the interior is written to the output."""
    from multiprocessing import shared_memory
    from oracle import stout
    name_in, name_out, shape, t0, t1 = task
    a, b = shared_memory.SharedMemory(name=name_in), shared_memory.SharedMemory(name=name_out)
    try:
        U = np.ndarray(shape, dtype=np.complex128, buffer=a.buf)
        out = np.ndarray(shape, dtype=np.complex128, buffer=b.buf)
        slab = U[[t % shape[0] for t in range(t0 - 1, t1 + 1)]]
        out[t0:t1] = stout.stout_step(slab, RHO, DIRS)[1:-1]
        del U, out
    finally:
        a.close()
        b.close()
    return t1 - t0


def time_oracle_all_cores(U):
    """The FP64 oracle's stout step on all host cores: t-slabs (one per core,
    each with a one-slice halo) in a spawned process pool over shared memory.
    Returns (link-updates/s, seconds, link updates, processes)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    procs = os.cpu_count() or 1
    Lt = U.shape[0]
    per = -(-Lt // procs)
    tasks_t = [(t0, min(Lt, t0 + per)) for t0 in range(0, Lt, per)]
    a = shared_memory.SharedMemory(create=True, size=U.nbytes)
    b = shared_memory.SharedMemory(create=True, size=U.nbytes)
    try:
        np.ndarray(U.shape, dtype=np.complex128, buffer=a.buf)[...] = U
        tasks = [(a.name, b.name, U.shape, t0, t1) for t0, t1 in tasks_t]
        with mp.get_context("spawn").Pool(processes=procs) as pool:
            pool.map(_pool_noop, range(procs))      # start-up, not timed
            t0 = time.perf_counter()
            pool.map(_oracle_slab_step, tasks, chunksize=1)
            dt = time.perf_counter() - t0
    finally:
        a.close()
        a.unlink()
        b.close()
        b.unlink()
    links = int(np.prod(U.shape[:4])) * len(DIRS)
    return links / dt, dt, links, procs


def run_reference(args, rank):
    """The oracle as the reference arm: each step a bounded sample (one stout step on 12^3 x 24)."""
    if rank != 0:
        return
    import fieldgen
    from oracle import gauge, stout
    dims = (12, 12, 12, 24)
    U = fieldgen.near_identity_su3(dims, SEED)
    for _ in range(args.warmup):
        stout.stout_step(U, RHO, DIRS)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        V1 = stout.stout_step(U, RHO, DIRS)
        gauge.plaquette(V1)
        times.append(time.perf_counter() - t0)
    links = int(np.prod(dims)) * len(DIRS)
    val = links / float(np.mean(times))
    sample = f"1 stout step + plaquette on 12^3x24 (same generator, rho, dirs) per bench step, numpy FP64"
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "link-updates/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "12^3x24"},
           "cpu_baseline": {"value": val, "unit": "link-updates/s", "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": val, "unit": "link-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def _compact_roof(r, probe):
    keep = {k: r[k] for k in ("bound", "pipe", "unit", "achieved", "peak", "frac", "fp64_flops_per_link")
            if k in r}
    if probe and "achieved" in r:
        keep["frac_of_measured_fp64"] = r["achieved"] / probe["fp64_tflops"]
    return keep


def run_secondary(sargs, torch, lq, fieldgen, bw, probe):
    """The 64-lattice batch, the 24^3x48 gradient and the 16^3x32 micro-suite,
    each as a compact object of the headline line (value, time, roofline,
    accuracy against the oracle or finite differences)."""
    out = {}
    t0 = time.perf_counter()
    b = bw.batch64(sargs, torch, lq, fieldgen)
    out["batch64"] = {"value": b["value"], "unit": b["unit"], "ms_per_step": b["ms_per_step"], "dtype": "f32",
                      "config": b["config"]["workload"], "separate_calls": b["separate_calls"],
                      "persistent_no_graph": b["persistent_no_graph"],
                      "speedup_vs_separate": b["speedup_vs_separate"],
                      "roofline": _compact_roof(b["roofline"], probe), "accuracy": b["accuracy"]}
    torch.cuda.empty_cache()
    g = bw.backward24(sargs, torch, lq, fieldgen)
    bk = {"metric": g["metric"], "unit": g["unit"], "config": g["config"]["workload"]}
    for prec in ("f64", "f32"):
        r = g[prec]
        bk[prec] = {"value": r["checkpoint_every_1"]["value"], "ms": r["checkpoint_every_1"]["ms"],
                    "recompute_every_3_ms": r["checkpoint_every_3"]["ms"],
                    "roofline": _compact_roof(r["roofline"], probe), "forward_ms": r["forward_ms"]}
        if "fd_max_rel" in r:
            bk[prec]["fd_max_rel"] = r["fd_max_rel"]
            bk[prec]["fd_config"] = r["fd_config"]
    bk["accuracy"] = g.get("accuracy")
    out["backward24"] = bk
    torch.cuda.empty_cache()
    m = bw.micro16(sargs, torch, lq, fieldgen)
    out["micro16"] = {"value": m["value"], "unit": m["unit"], "ms_per_step": m["ms_per_step"], "dtype": "f64",
                      "config": m["config"]["workload"], "micro_suite_ms": m["micro_suite_ms"],
                      "accuracy": m["accuracy"]}
    torch.cuda.empty_cache()
    out["secondary_wall_s"] = time.perf_counter() - t0
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the batch, gradient and micro-suite objects of the headline line")
    ap.add_argument("--fd-links", type=int, default=4, help="finite-difference links of the gradient check")
    ap.add_argument("--f64-steps", type=int, default=3)
    ap.add_argument("--dims", default=None, help="Lx,Ly,Lz,Lt override (smaller profiling cases)")
    ap.add_argument("--prec", default="both", choices=["both", "f32", "f64"],
                    help="secondary workloads with an FP32 and an FP64 leg: run only one of them")
    ap.add_argument("--variant", type=int, default=0,
                    help="step kernel: 0 auto-tuned (default), 1 global loads, 2 shared-memory staged (FP32)")
    ap.add_argument("--workload", default="stout48",
                    choices=["stout48", "batch64", "backward24", "micro16", "jacobi32", "ape48", "hyp32", "apeforce24", "hypforce24"],
                    help="stout48 (default, the headline line); the others print their own JSON line")
    args = ap.parse_args()
    if args.workload != "stout48" and args.impl == "ours":
        import bench_workloads
        bench_workloads.run(args)
        return
    global DIMS, WORKLOAD
    if args.dims:
        DIMS = tuple(int(x) for x in args.dims.split(","))
        WORKLOAD = WORKLOAD.replace("48^3x96", "x".join(map(str, DIMS)))
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import __graft_entry__
    __graft_entry__.build()
    import fieldgen
    import paper_1105_2279_gb300 as lq
    from oracle import lattice, stout

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    V = int(np.prod(DIMS))
    links_per_step = N_SMEAR * V * len(DIRS)
    g = lq.Geometry(DIMS)

    # inputs: generated on the device (seed + rank), staged once through the host AoS layout
    Ut = fieldgen.near_identity_su3_torch(DIMS, SEED + rank, device="cuda")
    U_host = Ut.cpu().numpy()
    del Ut
    torch.cuda.empty_cache()
    f32 = lq.Field(g, lq.LQ_LINKS, lq.LQ_F32)
    f64 = lq.Field(g, lq.LQ_LINKS, lq.LQ_F64)

    stream = torch.cuda.current_stream()
    if args.variant == 0:
        lq.tune(None)   # launch shapes tuned on the first (warm-up) call, kept in memory
    smear_opts = {"variant": args.variant} if args.variant else {}

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def timed(field, steps, warmup, opts=None):
        """Mean time of one bench step (6 smearing steps + plaquette).  Every step smears
        the same input: the links are restored from a device copy before each step,
        outside its timed interval (the coefficient series' order, and with it a
        step's FP64 work, falls as the field gets smoother, so smearing the previous
        output again would time an easier workload)."""
        field.upload(U_host)
        orig = field.tensor.clone()
        if opts is None:
            opts = smear_opts if field.prec == lq.LQ_F32 or args.variant != 2 else {}
        for _ in range(warmup):
            field.tensor.copy_(orig)
            lq.stout_smear(field, RHO, N_SMEAR, DIRS, **opts)
            lq.plaquette(field)
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1, e2 in ev:
            field.tensor.copy_(orig)
            e0.record(stream)
            lq.stout_smear(field, RHO, N_SMEAR, DIRS, **opts)   # N_SMEAR launches of the fused step kernel
            e1.record(stream)
            lq.plaquette(field)                          # 2 launches, synchronises
            e2.record(stream)
        barrier()
        step_ms = max_over_ranks(float(np.sum([a.elapsed_time(c) for a, _, c in ev])) / steps, dist)
        smear_ms = [a.elapsed_time(b) for a, b, _ in ev]
        del orig
        return step_ms, float(np.mean(smear_ms)) / N_SMEAR

    pk = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)

    with ClockSampler(local) as clk:
        step32, kern32 = timed(f32, args.steps, args.warmup)
        step64, kern64 = timed(f64, args.f64_steps, 1)
        # FP64 with the two-link product staples (variant 3, requested explicitly)
        step64w, kern64w = timed(f64, args.f64_steps, 1, {"variant": 3})
    clocks = clk.summary()

    # accuracy at the stated precision: fresh inputs, one 6-step smearing each
    f32.upload(U_host)
    f64.upload(U_host)
    lq.stout_smear(f32, RHO, N_SMEAR, DIRS, **smear_opts)
    lq.stout_smear(f64, RHO, N_SMEAR, DIRS)
    p32, p64 = lq.plaquette(f32), lq.plaquette(f64)
    # coefficient-stage work of this workload (series orders per link), for the flop count
    f32.upload(U_host)
    f64.upload(U_host)
    ch32 = lq.stout_ch_stats(f32, RHO, N_SMEAR, DIRS)
    ch64 = lq.stout_ch_stats(f64, RHO, N_SMEAR, DIRS)
    lq.stout_smear(f32, RHO, N_SMEAR, DIRS, **smear_opts)
    lq.stout_smear(f64, RHO, N_SMEAR, DIRS)
    d32 = f32.download()
    d64 = f64.download()
    err_32_64 = float(np.max(np.abs(d32.astype(np.complex128) - d64)))
    f64.upload(U_host)
    lq.stout_smear(f64, RHO, N_SMEAR, DIRS, variant=3)
    d64w = f64.download()
    err_w_64 = float(np.max(np.abs(d64w - d64)))
    rng = np.random.default_rng(7)
    e32o, e64o, e64wo = 0.0, 0.0, 0.0
    if rank == 0:
        for _ in range(3):
            c = [int(rng.integers(L)) for L in DIMS]
            ref = stout.stout_smear(lattice.sub_box(U_host, c, N_SMEAR), RHO, N_SMEAR, DIRS)[
                N_SMEAR, N_SMEAR, N_SMEAR, N_SMEAR]
            e32o = max(e32o, float(np.max(np.abs(d32[c[3], c[2], c[1], c[0]] - ref))))
            e64o = max(e64o, float(np.max(np.abs(d64[c[3], c[2], c[1], c[0]] - ref))))
            e64wo = max(e64wo, float(np.max(np.abs(d64w[c[3], c[2], c[1], c[0]] - ref))))
    del d32, d64, d64w

    # end to end through the C ABI with host buffers (page-locked): links in host memory ->
    # smeared links + plaquette in host memory, one lq_stout_smear_host call per step (the
    # copies and transposes of each t-slab overlap the smearing of the others)
    pin_in = torch.from_numpy(U_host.astype(np.complex64).view(np.float32)).pin_memory()
    pin_out = torch.empty_like(pin_in).pin_memory()
    e2e_steps = max(1, min(args.steps, 5))

    def e2e_step():
        return lq.stout_smear_host(pin_in, pin_out, g, lq.LQ_F32, RHO, N_SMEAR, DIRS, stream=stream)

    def e2e_sequential_step():
        f32.upload_ptr(pin_in.data_ptr())
        lq.stout_smear(f32, RHO, N_SMEAR, DIRS, **smear_opts)
        lq.plaquette(f32)
        f32.download_ptr(pin_out.data_ptr())

    def time_e2e(fn, calls):
        for _ in range(3):   # warm-up: the GPU idled during the CPU-side accuracy sampling
            fn()
        barrier()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(e2e_steps + 1)]
        evs[0].record(stream)
        for i in range(e2e_steps):
            fn()
            evs[i + 1].record(stream)
        barrier()
        calls.extend(evs[i].elapsed_time(evs[i + 1]) for i in range(e2e_steps))
        # the median call: each call ends by waiting on the host thread, so a
        # stall of the (shared) host shows as one long call; every call's time
        # and the mean are reported beside it
        mean = max_over_ranks(evs[0].elapsed_time(evs[-1]) / e2e_steps, dist)
        return max_over_ranks(float(np.median(calls[-e2e_steps:])), dist), mean

    e2e_calls, e2e_seq_calls = [], []
    e2e_ms, e2e_mean = time_e2e(e2e_step, e2e_calls)
    out_pipelined = pin_out.numpy().copy()
    e2e_seq_ms, e2e_seq_mean = time_e2e(e2e_sequential_step, e2e_seq_calls)
    # the pipelined call's result is the device path's, bit for bit
    e2e_same = bool(np.array_equal(out_pipelined, pin_out.numpy()))
    del out_pipelined

    # measured FMA throughput of the two pipes (the rooflines' measured denominators)
    probe = {"fp64_tflops": lq.peak_probe(lq.LQ_F64), "fp32_tflops": lq.peak_probe(lq.LQ_F32),
             "how": "lq_peak_probe: 8 CTAs x 256 threads per SM, 8 independent FMA chains per thread, CUDA events"}

    # secondary configurations (64-lattice batch, 24^3x48 gradient, 16^3x32 micro-suite)
    h2d_bytes, d2h_bytes = int(pin_in.numel() * 4), int(pin_out.numel() * 4)
    del f32, f64, pin_in, pin_out
    torch.cuda.empty_cache()
    secondary = {}
    if rank == 0 and not args.no_secondary:
        import types
        import bench_workloads
        sargs = types.SimpleNamespace(steps=max(1, min(args.steps, 5)), warmup=max(3, args.warmup), dims=None,
                                      prec="both", fd_links=args.fd_links)
        secondary = run_secondary(sargs, torch, lq, fieldgen, bench_workloads, probe)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, dt, n = time_oracle_sample()
        Ua = fieldgen.near_identity_su3_torch((24, 24, 24, 96), SEED, device="cuda").cpu().numpy()
        torch.cuda.empty_cache()
        va, dta, na, procs = time_oracle_all_cores(Ua)
        del Ua
        cpu = {"value": v, "unit": "link-updates/s", "cores": 1, "kind": "oracle",
               "sample": f"1 FP64 stout step, 4 dirs, on 16^3x32 (same generator and rho): {n} link updates in {dt:.1f} s",
               "all_cores": {"value": va, "unit": "link-updates/s", "cores": procs, "kind": "oracle",
                             "sample": f"1 FP64 stout step, 4 dirs, on 24^3x96 as {procs} t-slabs with one-slice "
                                       f"halos in a spawned process pool: {na} link updates in {dta:.2f} s"}}

    if rank == 0:
        value = weak_scaling_value(links_per_step, world, step32 * 1e-3)
        value64 = weak_scaling_value(links_per_step, world, step64 * 1e-3)
        links_per_launch = V * len(DIRS)
        mhz = clocks.get("sm_mhz") or 2070.0
        kernel_names = {1: "k_stout_global_f{b}", 2: "k_stout_smem<float,reproject>",
                        3: "k_wfield<{t}> + k_stout_wf<{t}>"}
        tuned32 = lq.tune_lookup(lq.LQ_F32, DIMS, DIRS)
        var32 = args.variant or (tuned32[2] if tuned32 else 1)
        roof32 = roofline(kern32, links_per_launch, "f32", hbm, mhz, ch_flops_per_link(ch32), var32)
        roof32["ch_stats"] = {"link_updates": ch32[0], "series": ch32[1], "mean_K": ch32[2] / max(1, ch32[1])}
        roof32["kernel"] = kernel_names[var32].format(b="32<reproject>", t="float")
        roof32["launch"] = {"variant": var32, "tuned": tuned32}
        if var32 == 2:
            roof32["traffic"] = None   # DRAM counters of the shared-memory kernel not captured at this revision
        tuned64 = lq.tune_lookup(lq.LQ_F64, DIMS, DIRS)
        var64 = (args.variant if args.variant in (1, 3) else 0) or (tuned64[2] if tuned64 else 1)
        roof64 = roofline(kern64, links_per_launch, "f64", hbm, mhz, ch_flops_per_link(ch64), var64)
        roof64["ch_stats"] = {"link_updates": ch64[0], "series": ch64[1], "mean_K": ch64[2] / max(1, ch64[1])}
        roof64["kernel"] = kernel_names[var64].format(b="64", t="double")
        roof64["launch"] = {"variant": var64, "tuned": tuned64}
        roof64w = roofline(kern64w, links_per_launch, "f64", hbm, mhz, ch_flops_per_link(ch64), 3)
        roof64w["kernel"] = kernel_names[3].format(t="double")
        out = {
            "metric": METRIC, "value": value, "unit": "link-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step32, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "precision": "FP32 matrix algebra and storage; FP64 Cayley-Hamilton coefficients, SU(3) re-projection and plaquette accumulation",
            "config": {"workload": WORKLOAD, "lattice": list(DIMS), "n_smear": N_SMEAR, "rho": RHO, "dirs": "xyzt",
                       "l2": "inputs larger than L2 (3.06 GB FP32 links)", "per_rank": "independent lattice per rank",
                       "input_per_step": "the same thin links every step, restored by a device copy outside the step's CUDA-event interval"},
            "roofline": roof32,
            "fp64": {"value": value64, "ms_per_step": step64, "kernel_ms": kern64, "roofline": roof64},
            "fp64_two_link_products": {
                "value": weak_scaling_value(links_per_step, world, step64w * 1e-3), "ms_per_step": step64w,
                "kernel_ms": kern64w, "roofline": roof64w, "vs_oracle_sampled_max_abs": e64wo,
                "vs_fp64_one_kernel_max_abs": err_w_64,
                "note": "opts variant=3: k_wfield + k_stout_wf, 9 staple products per link instead of 12"},
            "fp32_speedup_vs_fp64": value / value64,
            "accuracy": {"fp32_vs_fp64_gpu_max_abs": err_32_64, "fp32_vs_oracle_sampled_max_abs": e32o,
                         "fp64_vs_oracle_sampled_max_abs": e64o, "plaquette_fp32": p32[0], "plaquette_fp64": p64[0],
                         "plaquette_abs_diff": abs(p32[0] - p64[0])},
            "e2e": {"value": weak_scaling_value(links_per_step, world, e2e_ms * 1e-3), "unit": "link-updates/s",
                    "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": d2h_bytes,
                    "ms_per_step": e2e_ms, "statistic": "median over the timed calls", "ms_mean": e2e_mean,
                    "ms_calls": e2e_calls,
                    "call": "lq_stout_smear_host (16 t-slabs, transfers overlapped)",
                    "matches_device_path": e2e_same,
                    "sequential": {"value": weak_scaling_value(links_per_step, world, e2e_seq_ms * 1e-3),
                                   "ms_per_step": e2e_seq_ms, "ms_mean": e2e_seq_mean, "ms_calls": e2e_seq_calls,
                                   "call": "lq_field_upload + lq_stout_smear + lq_plaquette + lq_field_download"}},
            "gpu_launches": args.steps * (N_SMEAR + 2),
            "clocks": clocks,
            "cpu_baseline": cpu,
            "peaks_measured": probe,
        }
        out["roofline"]["frac_of_measured_fp64"] = roof32["achieved"] / probe["fp64_tflops"]
        out["fp64"]["roofline"]["frac_of_measured_fp64"] = roof64["achieved"] / probe["fp64_tflops"]
        out.update(secondary)
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
