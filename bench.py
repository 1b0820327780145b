"""Benchmark: GStencil/s and HBM-roofline fraction of the stencil sweep on GB300.

One "step" is one full solve of the workload through the C ABI: the 2D radius-2
box stencil (25 points) on an 8192 x 8192 FP32 grid, random normalised
coefficients, periodic boundary, 100 time steps (stencil_apply with inputs
resident in HBM).  The grid (256 MiB) is larger than L2, so no flush is needed
between steps.  Beside it the line reports the CUDA-core gather form at equal
error, the error of both against the FP64 oracle at sampled points, p50/p99,
the roofline of the dominant kernel and the oracle's own speed on the host.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank solves its own copy of the workload (independent
problems, no data exchange: weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import dataclasses

import numpy as np

from paper_2310_16298_gb300 import replicas

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GStencil/s and % HBM roofline, matrixized vs gather at equal error; p50/p99"
UNIT = "GStencil/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="box25-8192",
                    choices=["box25-8192", "star7-512", "box27-512", "box125-512", "sine7-512", "sine27-512", "jacobi-256",
                             "batch-1024", "serve-2000", "error-growth", "cover-study", "ablation"])
    ap.add_argument("--batch", type=int, default=1024, help="problems in the batch workload")
    ap.add_argument("--side", type=int, default=0, help="grid side (0 = the workload's own)")
    ap.add_argument("--tsteps", type=int, default=0, help="stencil time steps per solve (0 = the workload's own)")
    ap.add_argument("--bc", default="", choices=["", "dirichlet", "periodic"],
                    help="boundary condition ('' = the workload's own)")
    ap.add_argument("--dtype", default="", choices=["", "f32", "f64"], help="storage type ('' = the workload's own)")
    ap.add_argument("--prec", default="native", choices=["native", "tf32", "tf32x3", "bf16", "bf16x2", "bf16x3", "bf16w2"],
                    help="matrixized arithmetic (native = TF32x3 for FP32)")
    ap.add_argument("--cover", default="auto", choices=["auto", "parallel", "hybrid"],
                    help="line cover of star stencils on the matrixized kernel")
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-f64", action="store_true", help="skip the FP64 leg of the 2D workload")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def base_workload(args):
    import stencil_inputs as si
    w = args.workload
    if w == "box25-8192":
        return si.box25_8192(args.dtype or "f32", args.tsteps or 100, args.side or 8192)
    if w == "star7-512":
        return si.cube_512(si.STAR, args.dtype or "f32", args.tsteps or 50, args.side or 512)
    if w == "box27-512":
        return si.cube_512(si.BOX, args.dtype or "f32", args.tsteps or 50, args.side or 512)
    if w == "box125-512":
        return si.cube_512(si.BOX, args.dtype or "f32", args.tsteps or 50, args.side or 512, r=2)
    if w == "sine7-512":
        return si.sine_cube_512(si.STAR, args.tsteps or 1000, args.side or 512)
    if w == "sine27-512":
        return si.sine_cube_512(si.BOX, args.tsteps or 1000, args.side or 512)
    return si.jacobi_256(args.tsteps or 10)


def workload(args):
    import dataclasses
    p = base_workload(args)
    return dataclasses.replace(p, bc=args.bc) if args.bc else p


def workload_config(p, args, extra=None):
    desc = {"box25-8192": "2D box r=2 (25-point)", "star7-512": "3D 7-point star", "box27-512": "3D 27-point box",
            "box125-512": "3D box r=2 (125-point)",
            "sine7-512": "3D 7-point star (centre 0.4, neighbours 0.1)",
            "sine27-512": "3D 27-point separable box ((1/4,1/2,1/4)^3)",
            "jacobi-256": "2D 5-point Jacobi star"}[args.workload]
    grid_bytes = p.points * (4 if p.dtype == "f32" else 8)
    fdesc = ("lowest sine mode field (exact result known in closed form)" if p.field_kind == "sine"
             else "seeded synthetic field and coefficients")
    cfg = {"workload": f"{desc} {'x'.join(str(s) for s in p.shape)} {p.dtype.upper()}, {p.bc}, "
                       f"{p.steps} time steps per solve, {fdesc}",
           "grid": list(p.shape), "radius": p.r, "kind": p.kind, "boundary": p.bc,
           "time_steps_per_solve": p.steps,
           "l2_policy": (f"inputs larger than L2 (grid {grid_bytes / 2**20:.0f} MiB > 129 MB L2); no flush"
                         if grid_bytes > 129e6 else
                         f"grid {grid_bytes / 2**20:.1f} MiB is L2-resident: latency workload, no HBM claim")}
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained"), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


# Sources that build each kernel family (the ncu traffic of a kernel stays
# valid while these files are unchanged).
KERNEL_SOURCES = {
    "matrixized-f32-2d": ("mx.cu", "mxutil.cuh", "ptx.cuh", "common.cuh", "mx.h", "plan.cpp", "plan.h"),
    "matrixized-f32-3d": ("mx3d.cu", "mxutil.cuh", "ptx.cuh", "common.cuh", "mx.h", "plan.cpp", "plan.h"),
    "gather": ("gather.cu", "common.cuh", "kernels.h"),
}


def kernel_source_hash(kernel_key):
    fam = next((k for k in KERNEL_SOURCES if kernel_key.startswith(k)), None)
    csrc = os.path.join(ROOT, "paper_2310_16298_gb300", "csrc")
    files = KERNEL_SOURCES[fam] if fam else sorted(f for f in os.listdir(csrc) if f.endswith((".cu", ".cuh", ".h", ".cpp")))
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key):
    """Per-launch DRAM bytes for the kernel from the committed ncu summary,
    valid only while the kernel's sources are unchanged."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    e = d.get(kernel_key)
    if not e or e.get("source_hash") != kernel_source_hash(kernel_key):
        return None
    return e.get("dram_bytes_per_launch")


def oracle_baseline(p, field, max_seconds=20.0):
    """Time the FP64 oracle on a bounded sample of the workload: the full grid,
    as many whole time steps as fit in about max_seconds (at least one)."""
    import oracle
    oracle.build()
    cores = oracle.threads()
    t0 = time.perf_counter()
    oracle.gather(field, p.r, p.coeffs, p.bc, 1)
    t1 = time.perf_counter() - t0
    nsteps = max(1, min(p.steps, int(max_seconds / max(t1, 1e-6)) - 1))
    if nsteps > 1:
        t0 = time.perf_counter()
        oracle.gather(field, p.r, p.coeffs, p.bc, nsteps)
        dt = time.perf_counter() - t0
    else:
        nsteps, dt = 1, t1
    gst = p.points * nsteps / dt / 1e9
    return {"value": gst, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"full {'x'.join(str(s) for s in p.shape)} grid, {nsteps} of {p.steps} time steps, "
                      f"{dt:.1f} s, FP64 gather definition, OpenMP over rows"}


# Tile periods of the matrixized kernels along each axis (slowest first):
# 2D tiles are 4 lane quarters of 2 (32 - 2 ceil(r/2)) rows by 2 items of 16
# columns; 3D work units are 32-plane chunks by 4 quarters of 32 - 2r rows by
# 16 or 32 columns.  Seams between them are sampled on purpose.
def tile_periods(ndim, r):
    if ndim == 2:
        q = 2 * (32 - 2 * ((r + 1) // 2))
        return [(q, 4 * q), (16, 32)]
    q = 32 - 2 * r
    return [(32,), (q, 4 * q), (16, 32)]


def sample_points(shape, r, n=64, n_random=8, seed=77):
    """Output points checked against the oracle: every corner (the periodic
    wrap in every axis), then points whose coordinates sit on either side of
    tile, quarter and item seams, near both edges and mid-grid, then a few
    uniform random points."""
    rng = np.random.default_rng(seed)
    ndim = len(shape)
    cands = []
    for ax, (nax, periods) in enumerate(zip(shape, tile_periods(ndim, r))):
        c = {0, 1, 2, nax // 2, nax - 3, nax - 2, nax - 1}
        for P in periods:
            for k in (1, 2, max(1, nax // P // 2), nax // P):
                c.update((k * P - 1, k * P))
        cands.append(sorted(v for v in c if 0 <= v < nax))
    pts = [list(p) for p in np.ndindex(*([2] * ndim))]
    pts = [[0 if b == 0 else shape[d] - 1 for d, b in enumerate(p)] for p in pts]
    seen = {tuple(p) for p in pts}
    want = min(n, int(np.prod([len(c) for c in cands])))
    for _ in range(20 * n):   # bounded: small grids hold fewer candidate points
        if len(pts) >= want:
            break
        p = tuple(int(rng.choice(c)) for c in cands)
        if p not in seen:
            seen.add(p)
            pts.append(list(p))
    for _ in range(n_random):
        pts.append([int(rng.integers(0, s)) for s in shape])
    return np.array(pts, dtype=np.int64)


def sine_closed_form(p, field, pts):
    """lam^T times the initial sine mode at the sampled points, with
    lam = sum_o C^g[o] prod_k cos(pi (o_k - r) / (n_k + 1)) (exact for C^g
    symmetric in every axis and zero Dirichlet boundaries)."""
    phi = [np.pi / (n + 1) for n in p.shape]
    w = 2 * p.r + 1
    lam = 0.0
    for o in np.ndindex(*([w] * p.ndim)):
        lam += p.coeffs[o] * np.prod([np.cos(ph * (ok - p.r)) for ph, ok in zip(phi, o)])
    return lam ** p.steps * field[tuple(pts.T)]


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import stencil_inputs as si
    p = workload(args)
    field = p.field()
    # each "step" is a bounded sample: one time step of the full grid
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle.gather(field, p.r, p.coeffs, p.bc, 1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.gather(field, p.r, p.coeffs, p.bc, 1)
        times.append(time.perf_counter() - t0)
    t = float(np.median(times))
    v = p.points / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(p, args, {"sample": "one time step of the full grid per bench step"}),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": "one of the workload's time steps on the full grid per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ batch workload
def run_batch_workload(args):
    """Many independent 2D 9-point box problems (sides log-uniform in [64, 2048],
    steps uniform in 20..200, FP32, zero Dirichlet) advanced by one graph
    replay of a packed persistent schedule."""
    rank, world, local = dist_env()
    import torch
    import paper_2310_16298_gb300 as sx
    import stencil_inputs as si
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    # the batch of every rank is its shard of world x n problems (independent units)
    allp = si.batch_1024(args.batch * world)
    probs = [allp[i] for i in replicas.shard(len(allp), rank, world)]
    plans, xs, ys = [], [], []
    for p in probs:
        plans.append(sx.stencil_plan_create(p.shape, p.r, p.kind, p.coeffs, "f32",
                                            sx.make_options("native", p.bc, "gather", 0)))
        x = torch.tensor(p.field(), dtype=torch.float32, device=dev)
        xs.append(x)
        ys.append(torch.empty_like(x))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = sx.stencil_batch_create(plans, [x.data_ptr() for x in xs], [y.data_ptr() for y in ys],
                                [p.steps for p in probs], 0)
    create_s = time.perf_counter() - t0
    info = sx.stencil_batch_info(b)
    stream = torch.cuda.Stream(device=dev)
    for _ in range(args.warmup):
        sx.stencil_batch_launch(b, stream.cuda_stream)
    stream.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    for a, e in ev:
        a.record(stream)
        sx.stencil_batch_launch(b, stream.cuda_stream)
        e.record(stream)
    stream.synchronize()
    clk = sampler.stop()
    ms = [a.elapsed_time(e) for a, e in ev]
    tot = sum(ms) / 1e3
    tot = replicas.max_over_ranks(tot, dev)
    value = replicas.sum_over_ranks(info["updates"] * args.steps, dev) / tot / 1e9
    # accuracy: a few problems against the oracle at sampled points
    import oracle
    errs = []
    if rank == 0:
        for i in (0, len(probs) // 2, len(probs) - 1):
            p = probs[i]
            pts = sample_points(p.shape, p.r, n=8, n_random=2, seed=i)
            want = oracle.sample(p.field(), p.r, p.coeffs, p.bc, p.steps, pts)
            got = ys[i][tuple(torch.as_tensor(c, device=dev) for c in pts.T)].double().cpu().numpy()
            errs.append(oracle.error_norms(got, want))
    npts = sum(p.points for p in probs)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"batch of {len(probs)} independent 2D 9-point box problems, sides "
                                       f"log-uniform in [64, 2048], steps uniform in [20, 200], FP32, zero Dirichlet; "
                                       f"one CUDA-graph replay of packed persistent launches per step",
                           "points": npts, "updates_per_run": info["updates"], "tb": info["tb"],
                           "tile_shape": ["64x128", "32x64"][info["tile_shape"]],
                           "launches_per_run": info["launches"], "tiles_per_run": info["tiles"],
                           "create_s": create_s, "parallelism": f"replicas x{world}",
                           "l2_policy": f"{npts * 8 / 2**30:.1f} GiB of grids per run > L2; no flush"},
                "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
                "err_vs_oracle": [{"rel_l2": a, "rel_max": b2} for a, b2 in errs],
                "gpu_launches": info["launches"] * args.steps, "clocks": clk}
        print(json.dumps(line), flush=True)
    sx.stencil_batch_destroy(b)
    for p in plans:
        sx.stencil_plan_destroy(p)
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------ serving workload
def run_error_growth(args):
    """Error against the FP64 oracle (full grid) after 10, 100 and 1000 steps
    for every precision mode of the matrixized kernel and for the FP32 gather
    kernel: 2D r=2 box, 512^2 FP32, periodic, the coefficients and field of
    the 8192^2 workload's recipe."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    import torch
    import paper_2310_16298_gb300 as sx
    import stencil_inputs as si
    import oracle
    torch.cuda.set_device(local)
    p = si.box25_8192("f32", 1, args.side or 512)
    field = p.field()
    x = torch.tensor(field, dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    modes = [("gather", "native"), ("matrixized", "tf32x3"), ("matrixized", "bf16x3"), ("matrixized", "bf16x2"),
             ("matrixized", "tf32"), ("matrixized", "bf16"), ("matrixized", "bf16w2")]
    table = {}
    for steps in (10, 100, 1000):
        ref = oracle.gather(field, p.r, p.coeffs, p.bc, steps)
        for impl, prec in modes:
            plan = sx.Plan(p.shape, p.r, p.kind, p.coeffs, "f32", bc=p.bc, impl=impl, prec=prec)
            plan.apply(x, y, steps)
            torch.cuda.synchronize()
            l2, mx = oracle.error_norms(y.double().cpu().numpy(), ref)
            table.setdefault(f"{impl}-{prec}", {})[str(steps)] = {"rel_l2": l2, "rel_max": mx}
            plan.close()
    line = {"metric": "rel-L2 / rel-max error vs the FP64 oracle after T steps", "value": None, "unit": "",
            "workload": f"2D box r=2 (25-point) {p.shape[0]}x{p.shape[1]} FP32, periodic, full-grid comparison",
            "errors": table}
    print(json.dumps(line), flush=True)


def run_cover_study(args):
    """The line-cover study of the paper's Sec. 5.2 on this GPU: one sweep of a
    3D star of order 1..3 (512^3 FP32 by default, zero Dirichlet, seeded
    coefficients) with each cover -- all lines on the tensor cores (parallel)
    or the contiguous-axis line there and the off-axis weights on the CUDA
    cores (hybrid) -- and the cover COVER_AUTO picks, for TF32x3 and TF32."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    import torch
    import paper_2310_16298_gb300 as sx
    import stencil_inputs as si
    torch.cuda.set_device(local)
    side = args.side or 512
    shape = (side, side, side)
    x = torch.rand(shape, device="cuda") * 2 - 1
    y = torch.empty_like(x)
    stream = torch.cuda.Stream()
    rows = []
    for r in (1, 2, 3):
        cg = si.coeffs_random(3, r, si.STAR, 103, dtype="f32")
        for prec in ("tf32x3", "tf32"):
            row = {"radius": r, "points": 6 * r + 1, "prec": prec}
            for cover in ("parallel", "hybrid", "auto"):
                plan = sx.Plan(shape, r, "star", cg, "f32", bc="dirichlet", impl="matrixized", prec=prec, cover=cover)
                for _ in range(2):
                    plan.apply(x, y, 1, stream)
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
                for a_, b_ in ev:
                    a_.record(stream)
                    plan.apply(x, y, 1, stream)
                    b_.record(stream)
                stream.synchronize()
                ms = float(np.median([a_.elapsed_time(b_) for a_, b_ in ev]))
                row[cover] = {"ms_per_sweep": ms, "gstencil_s": x.numel() / ms / 1e6,
                              "n_lines": plan.info["n_lines"], "n_scalar": plan.info["n_scalar"],
                              "tile_n": plan.info["tile_n"], "cover": plan.info["cover"]}
                plan.close()
            rows.append(row)
    line = {"metric": "line-cover study: GStencil/s of one sweep per cover", "value": None, "unit": "GStencil/s",
            "workload": f"3D star r=1..3, {side}^3 FP32, zero Dirichlet, matrixized kernel",
            "covers": rows}
    print(json.dumps(line), flush=True)


def run_ablation(args):
    """Scheduling ablation of the 3D matrixized kernel (the unrolling study of
    the paper's Sec. 4.2 on this GPU): one sweep of the 7-point star (hybrid
    cover) and of the 27-point box, 512^3 FP32 TF32x3, for work units of
    1 .. 128 output planes.  A unit streams its planes plus 2r halo planes,
    so deeper units re-read fewer planes (operand reuse across planes) but
    leave fewer units to balance across the SMs."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    import torch
    import paper_2310_16298_gb300 as sx
    import stencil_inputs as si
    torch.cuda.set_device(local)
    side = args.side or 512
    shape = (side, side, side)
    x = torch.rand(shape, device="cuda") * 2 - 1
    y = torch.empty_like(x)
    stream = torch.cuda.Stream()
    rows = []
    for kind in ("star", "box"):
        cg = si.coeffs_random(3, 1, kind, 103, dtype="f32")
        for up in (1, 2, 4, 8, 16, 32, 64, 128):
            plan = sx.Plan(shape, 1, kind, cg, "f32", bc="dirichlet", impl="matrixized", prec="tf32x3",
                           cover="hybrid" if kind == "star" else "auto", unit_planes=up)
            for _ in range(2):
                plan.apply(x, y, 1, stream)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
            for a_, b_ in ev:
                a_.record(stream)
                plan.apply(x, y, 1, stream)
                b_.record(stream)
            stream.synchronize()
            ms = float(np.median([a_.elapsed_time(b_) for a_, b_ in ev]))
            tile_n = plan.info["tile_n"]
            units = -(-side // up) * -(-side // 120) * -(-side // tile_n)
            rows.append({"kind": kind, "unit_planes": up, "input_planes_per_output_plane": (up + 2) / up,
                         "units": units, "ms_per_sweep": ms, "gstencil_s": x.numel() / ms / 1e6})
            plan.close()
    line = {"metric": "scheduling ablation: GStencil/s of one 3D sweep per work-unit depth", "value": None,
            "unit": "GStencil/s", "workload": f"3D r=1 {side}^3 FP32 TF32x3, zero Dirichlet, matrixized kernel",
            "rows": rows}
    print(json.dumps(line), flush=True)


def run_serving_workload(args):
    """Poisson arrivals of mixed stencil solves (70% 2D 128^2..4096^2 r=1..3
    star|box, 30% 3D 64^3..384^3 7/27-point, 10% FP64, steps 10..500) served
    with continuous batching under a 120 GB budget.  The saturated rate is
    measured first (all requests queued at once); then the same requests
    arrive as Poisson streams at 0.5x and 0.8x that rate and the latency
    (arrival to result on the host) is reported."""
    rank, world, local = dist_env()
    import torch
    import paper_2310_16298_gb300 as sx
    import stencil_inputs as si
    torch.cuda.set_device(local)
    n = args.batch if args.batch != 1024 else 2000
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    # every rank serves the requests a round-robin router sends it from a
    # stream of world x n requests (independent units, no data exchange)
    base = replicas.routed(si.serving_stream(n * world, rate_per_s=1.0), rank, world)

    def serve(arrivals):
        srv = sx.stencil_server_create(120 * 10**9, 64, 16, 8)
        keep, ids = [], []
        t0 = time.perf_counter()
        for (t_arr, rq) in arrivals:
            dt = t0 + t_arr - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            p = rq.problem
            r, ref = sx.make_request(p.shape, p.r, p.kind, p.coeffs, p.dtype, p.steps, bc=p.bc,
                                     seed=p.field_seed, lo=p.field_lo, hi=p.field_hi)
            keep.append((r, ref))
            ids.append(sx.stencil_server_submit(srv, r))
        lat, upd, first, last = [], 0, None, 0.0
        for rid in ids:
            assert sx.stencil_server_wait(srv, rid, -1) == sx.OK, sx.stencil_last_error()
            st = sx.stencil_server_result(srv, rid, None)
            lat.append(st["done_s"] - st["submit_s"])
            upd += st["updates"]
            first = st["submit_s"] if first is None else min(first, st["submit_s"])
            last = max(last, st["done_s"])
        stats = sx.stencil_server_stats(srv)
        sx.stencil_server_destroy(srv)
        return np.array(lat), upd, last - first, stats

    sampler = ClockSampler(local)
    sampler.start()
    lat_s, upd, span, st_s = serve([(0.0, q) for q in base])
    sat_rate = n / span   # this rank's saturated rate
    span_all = replicas.max_over_ranks(span, dev)
    results = {"saturated": {"requests_per_s": replicas.sum_over_ranks(n, dev) / span_all,
                             "gstencil_s": replicas.sum_over_ranks(upd, dev) / span_all / 1e9, "makespan_s": span_all,
                             "p50_latency_s": float(np.percentile(lat_s, 50)),
                             "p99_latency_s": float(np.percentile(lat_s, 99)), "peak_resident": st_s["peak_resident"],
                             "peak_bytes": st_s["peak_bytes"]}}
    for frac in (0.5, 0.8):
        stream = replicas.routed(si.serving_stream(n * world, rate_per_s=frac * sat_rate * world), rank, world)
        lat, upd_f, span_f, st_f = serve([(q.arrival_s, q) for q in stream])
        span_f = replicas.max_over_ranks(span_f, dev)
        results[f"load_{frac}"] = {"offered_requests_per_s": replicas.sum_over_ranks(frac * sat_rate, dev),
                                   "gstencil_s": replicas.sum_over_ranks(upd_f, dev) / span_f / 1e9,
                                   "p50_latency_s": float(np.percentile(lat, 50)),
                                   "p99_latency_s": float(np.percentile(lat, 99)),
                                   "peak_resident": st_f["peak_resident"], "peak_bytes": st_f["peak_bytes"]}
    clk = sampler.stop()
    if rank == 0:
        head = results["load_0.8"]
        line = {"metric": METRIC, "value": head["gstencil_s"], "unit": UNIT, "n_gpus": world, "steps": 1,
                "warmup": 0, "ms_per_step": span_all * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"serving: {n} Poisson-arrival requests, 70% 2D (128^2..4096^2, r 1..3, "
                                       f"star|box), 30% 3D (64^3..384^3, 7/27-point), FP32 with 10% FP64, steps "
                                       f"10..500, 120 GB admission budget, 64 slots, quantum 16 steps",
                           "value_is": "GStencil/s over the makespan at offered load 0.8 x saturated rate",
                           "parallelism": f"replicas x{world}"},
                "p50_ms": head["p50_latency_s"] * 1e3, "p99_ms": head["p99_latency_s"] * 1e3,
                "serving": results, "clocks": clk}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------ our arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch-1024":
        return run_batch_workload(args)
    if args.workload == "serve-2000":
        return run_serving_workload(args)
    if args.workload == "error-growth":
        return run_error_growth(args)
    if args.workload == "cover-study":
        return run_cover_study(args)
    if args.workload == "ablation":
        return run_ablation(args)
    rank, world, local = dist_env()
    import torch
    import paper_2310_16298_gb300 as sx
    import stencil_inputs as si

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    p = workload(args)
    if world > 1:   # every rank solves its own independent grid (a replica with its own field)
        p = dataclasses.replace(p, field_seed=replicas.field_seed(p.field_seed, rank))
    field = p.field()
    td = torch.float32 if p.dtype == "f32" else torch.float64
    x = torch.tensor(field, dtype=td, device=dev)
    y = torch.empty_like(x)
    stream = torch.cuda.Stream(device=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    results = {}
    for impl in ("matrixized", "gather"):
        try:
            plan = sx.Plan(p.shape, p.r, p.kind, p.coeffs, p.dtype, bc=p.bc, impl=impl,
                           prec=args.prec if impl == "matrixized" else "native",
                           cover=args.cover if impl == "matrixized" else "auto")
        except sx.StencilError as e:
            results[impl] = {"unavailable": str(e)}
            continue
        results[impl] = {"plan": plan}

    main_impl = "matrixized" if "plan" in results.get("matrixized", {}) else "gather"

    # accuracy of each implementation at sampled points (oracle on the dependency cone)
    import oracle
    pts = sample_points(p.shape, p.r)
    if p.field_kind == "sine":
        # long runs: every point depends on the whole grid, so the check is
        # the closed form (the field is an eigenvector of the symmetric stencil)
        want = sine_closed_form(p, field, pts)
    else:
        want = oracle.sample(field, p.r, p.coeffs, p.bc, p.steps, pts) if rank == 0 else None
    for impl, res in results.items():
        if "plan" not in res:
            continue
        with torch.cuda.stream(stream):
            res["plan"].apply(x, y, p.steps, stream)
        stream.synchronize()
        if rank == 0:
            idx = tuple(torch.as_tensor(c, device=dev) for c in pts.T)
            got = y[idx].double().cpu().numpy()
            l2, mx = oracle.error_norms(got, want)
            res["err"] = {"rel_l2": l2, "rel_max": mx, "points": len(pts)}

    def time_solves(plan, k, w, sampler=None):
        for _ in range(w):
            plan.apply(x, y, p.steps, stream)
        stream.synchronize()
        barrier()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        if sampler:
            sampler.start()
        t_host = time.perf_counter()
        for i in range(k):
            ev[i][0].record(stream)
            plan.apply(x, y, p.steps, stream)
            ev[i][1].record(stream)
        stream.synchronize()
        t_host = time.perf_counter() - t_host
        clk = sampler.stop() if sampler else None
        torch.cuda.synchronize()
        barrier()
        ms = [a.elapsed_time(b) for a, b in ev]
        return ms, t_host, clk

    # --- the timed region: K solves of the main implementation
    plan = results[main_impl]["plan"]
    sampler = ClockSampler(local)
    ms, t_host, clk = time_solves(plan, args.steps, args.warmup, sampler)
    tot = float(np.sum(ms)) / 1e3
    tot = replicas.max_over_ranks(tot, dev)
    updates = replicas.sum_over_ranks(p.updates * args.steps, dev)
    value = updates / tot / 1e9
    per_solve = np.array(ms)
    results[main_impl]["timing"] = ms

    # --- the baseline form at equal error (gather), same protocol, untimed for `value`
    other = "gather" if main_impl == "matrixized" else None
    if other and "plan" in results[other]:
        oms, _, _ = time_solves(results[other]["plan"], max(2, args.steps // 2), 1)
        results[other]["timing"] = oms

    # --- the paper's own precision (FP64) on the same 2D workload: the CUDA-core
    # gather kernel (no FP64 tensor-core kind on this GPU), its error at
    # sampled points and its fraction of the nominal FP64 FMA rate
    f64_leg = None
    if (rank == 0 and args.workload == "box25-8192" and p.dtype == "f32" and not args.no_f64):
        p64 = dataclasses.replace(p, dtype="f64", coeffs=si.coeffs_random(2, p.r, p.kind, 102, dtype="f64"))
        f64f = p64.field()
        x64 = torch.tensor(f64f, dtype=torch.float64, device=dev)
        y64 = torch.empty_like(x64)
        plan64 = sx.Plan(p64.shape, p64.r, p64.kind, p64.coeffs, "f64", bc=p64.bc, impl="gather")
        plan64.apply(x64, y64, p64.steps, stream)
        stream.synchronize()
        fev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(2)]
        for a_, b_ in fev:
            a_.record(stream)
            plan64.apply(x64, y64, p64.steps, stream)
            b_.record(stream)
        stream.synchronize()
        t64 = float(np.median([a_.elapsed_time(b_) for a_, b_ in fev])) / 1e3
        pts64 = pts[:16]
        want64 = oracle.sample(f64f, p64.r, p64.coeffs, p64.bc, p64.steps, pts64)
        got64 = y64[tuple(torch.as_tensor(c, device=dev) for c in pts64.T)].cpu().numpy()
        l2_64, mx_64 = oracle.error_norms(got64, want64)
        g64 = p64.updates / t64 / 1e9
        nterms = int(np.count_nonzero(p64.coeffs))
        f64_leg = {"impl": "gather", "dtype": "f64", "gstencil_s": g64, "ms_per_solve": t64 * 1e3,
                   "err_vs_oracle": {"rel_l2": l2_64, "rel_max": mx_64, "points": len(pts64)},
                   "fp64_tflops": g64 * 2 * nterms / 1e3, "fp64_peak_tflops_nominal": 1.25,
                   "fp64_frac_of_nominal": g64 * 2 * nterms / 1e3 / 1.25,
                   "note": "FP64 runs on CUDA-core FMAs (tcgen05 has no FP64 kind); bound by the FP64 FMA rate"}
        plan64.close()
        del x64, y64

    # --- dominant kernel, live: the timed region's median solve over its sweeps
    # (CUDA events on the launching stream around each solve; consecutive
    # sweeps overlap each launch's set-up with the previous kernel's tail).
    # An isolated single-sweep launch (events around it, no overlap) is
    # reported beside it.
    info = plan.info
    tb = info["tb"]
    kernels = info.get("kernels_per_sweep", 1)   # 2: tensor-core kernel + periodic boundary terms
    sweeps_per_solve = (p.steps + tb - 1) // tb
    launches_per_solve = sweeps_per_solve * kernels
    kms = float(np.percentile(per_solve, 50)) / sweeps_per_solve
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(20)]
    for i in range(20):
        kev[i][0].record(stream)
        plan.apply(x, y, tb, stream)
        kev[i][1].record(stream)
    stream.synchronize()
    kms_isolated = float(np.median([a.elapsed_time(b) for a, b in kev[3:]]))
    es = 4 if p.dtype == "f32" else 8
    alg_bytes = 2 * es * p.points  # read the grid once, write it once per launch
    pk = peaks()
    achieved = alg_bytes / (kms / 1e3) / 1e9
    kernel_key = f"{main_impl}-{p.dtype}-{p.ndim}d-r{p.r}-{p.kind}-tb{tb}"
    roofline = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": ncu_traffic(kernel_key),
                "kernel": kernel_key, "launch_ms": kms, "launch_ms_isolated": kms_isolated,
                "launch_timing": "median solve of the timed region / sweeps per solve",
                "algorithmic_bytes_per_launch": alg_bytes,
                "time_steps_per_launch": tb, "peak_source": f"{pk['source']} (copy bandwidth, burst)"}
    if kernels > 1:
        roofline["timed_region"] = ("one sweep: the tensor-core kernel, then the kernel that adds the "
                                    "periodic boundary's wrapped terms over the boundary strips")

    # --- end to end through the host-buffer C-ABI call
    e2e = None
    if not args.no_e2e:
        h_in = torch.from_numpy(field.astype(np.float32 if p.dtype == "f32" else np.float64)).pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        sx.stencil_apply_host(plan.handle, h_in.numpy(), h_out.numpy(), p.steps)  # warm
        et = []
        for _ in range(max(2, args.steps // 2)):
            t0 = time.perf_counter()
            sx.stencil_apply_host(plan.handle, h_in.numpy(), h_out.numpy(), p.steps)
            et.append(time.perf_counter() - t0)
        e2e_t = replicas.max_over_ranks(float(np.median(et)), dev)
        e2e = {"value": replicas.sum_over_ranks(p.updates, dev) / e2e_t / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(h_in.numel() * h_in.element_size()),
               "d2h_bytes_per_step": int(h_out.numel() * h_out.element_size()),
               "api": "stencil_apply_host (pinned host buffers, H2D + solve + D2H)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_baseline:
        cpu = oracle_baseline(p, field)

    if rank == 0:
        comp = {}
        for impl, res in results.items():
            if "plan" not in res:
                comp[impl] = res
                continue
            d = {"plan": {k: v for k, v in res["plan"].info.items()}, "err_vs_oracle": res.get("err")}
            if "timing" in res:
                t = np.array(res["timing"]) / 1e3
                d["gstencil_s_p50"] = p.updates / float(np.percentile(t, 50)) / 1e9
                d["ms_per_solve_p50"] = float(np.percentile(t, 50) * 1e3)
                d["ms_per_solve_p99"] = float(np.percentile(t, 99) * 1e3)
            comp[impl] = d
        if f64_leg:
            comp["gather_f64"] = f64_leg
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": p.dtype, "data": "synthetic",
                "config": workload_config(p, args, {"impl": main_impl, "prec": info["prec"], "tb": tb, "cover": args.cover,
                                                    "parallelism": f"replicas x{world}"}),
                "p50_ms": float(np.percentile(per_solve, 50)), "p99_ms": float(np.percentile(per_solve, 99)),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches_per_solve * args.steps * world, "clocks": clk, "compare": comp,
                "host_s": t_host}
        print(json.dumps(line), flush=True)
    for res in results.values():
        if "plan" in res:
            res["plan"].close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
