"""Benchmark: Wilson-Clover apply GFlop/s and HBM roofline fraction at
24^3x32 (FP32), plus mixed-precision RAS-BiCGStab vs plain FP64 BiCGStab
time to 1e-10 on the same lattice.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one application of M = (1 + T) - kappa H to an FP32 colour-spinor
field on the 24^3x32 lattice (Haar-like SU(3) links, csw = 1.0,
kappa = 0.125, antiperiodic time, Z2 source), inputs resident in HBM.
GFlop/s counts 1320 (hopping) + 504 (clover) = 1824 flops per site.  Every
step reads links + clover + input spinor = 297 MB (> 129 MB L2) and steps
rotate over 4 input/output field pairs.

Under torchrun (N > 1) every rank runs an independent replica of the
workload (the path has no data exchange between lattices: weak scaling);
the timed region is bracketed by barriers and the max over ranks is taken.

--impl reference times the CPU oracle (plain FP64 C, OpenMP) on the host
cores on a bounded sample of the same apply.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOPS_PER_SITE = 1320 + 504
# compulsory bytes per site of one M apply: in + out spinor, 4 forward links,
# clover (FP32 and FP16: 12-real links; FP16: per-site FP32 scale with each
# spinor; FP64: 18-real links)
BYTES_PER_SITE = {"f32": 96 + 96 + 192 + 288, "f16": 52 + 52 + 96 + 144, "f64": 192 + 192 + 576 + 576}
CFG = 2  # the 24^3x32 FP32 workload
METRIC = "Wilson-Clover apply GFlop/s & % HBM roofline; mixed vs FP64 solve time to 1e-10"

# DRAM bytes per launch of the timed kernel from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum), valid only while the kernel source is unchanged.
NCU_TRAFFIC = {
    # dram__bytes_read.sum + dram__bytes_write.sum of one k_apply<P32, M>
    # launch at 24^3x32 (shape #20: persistent, programmatic dependent launch;
    # the other lexicographic shapes run the same kernel body), from the
    # capture summarised in profiles/apply_fp32_24x24x24x32.md; valid while
    # the operator's device sources hash to sources_sha
    "sources_sha": "b010e33ca36fe672",
    "bytes_per_launch": 292184064,
}


def kernel_sources_sha() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1612_06556_gb300", "csrc")
    for f in ("wc_dslash.cu", "wc_stencil.cuh", "wc_device.cuh", "wc_df.cuh", "wc_df2.cuh", "wc_check.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples every 200 ms while running (clocks, throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank: int):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        self.gpu = ids[local_rank] if local_rank < len(ids) else str(local_rank)
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(float(r[2]) for r in rows),
                "reasons": reasons, "samples": len(rows)}


def reduce_max(x: float, world: int, device: str = "cuda") -> float:
    """Max of x over all ranks (all_reduce MAX); x itself when world == 1."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Throughput of the whole job: every rank's units over the slowest
    rank's time (weak scaling: each rank runs its own replica)."""
    return units_per_rank * world / (max_ms * 1e-3)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class OracleSampler:
    """The CPU oracle's M apply on a contiguous sample of sites of the same
    lattice.  The oracle's clover field is built once, outside the timing;
    the sample size is calibrated so that one timed call takes ~target_s."""

    def __init__(self, dims, U, src, csw, kappa, tbc, target_s):
        import oracle
        self.oracle = oracle
        self.args = (dims, tbc, kappa, csw, U, src)
        self.T = oracle.clover_field(dims, csw, kappa, U)
        self.V = int(np.prod(dims))
        n = min(self.V, 4096)
        dt = self._time(n, 1)
        want = n * target_s / max(dt, 1e-6)      # sites that take target_s
        self.n = int(min(self.V, max(256, want)))
        self.reps = max(1, int(round(want / self.V))) if want > self.V else 1
        self.cores = int(os.environ.get("OMP_NUM_THREADS", len(os.sched_getaffinity(0))))

    def _time(self, n, reps):
        dims, tbc, kappa, csw, U, src = self.args
        sites = np.arange(n)
        t0 = time.perf_counter()
        for _ in range(reps):
            self.oracle.apply_M(dims, tbc, kappa, csw, U, src, T=self.T, sites=sites)
        return time.perf_counter() - t0

    def step(self):
        """One timed sample: (GFlop/s, seconds)."""
        dt = self._time(self.n, self.reps)
        return FLOPS_PER_SITE * self.n * self.reps / dt / 1e9, dt

    def describe(self, dt):
        what = (f"{self.reps} full-lattice applies" if self.n == self.V
                else f"sites 0..{self.n - 1} of the {self.V}-site lattice")
        return f"oracle FP64 M apply (C, OpenMP): {what}, {dt:.2f} s per sample"


def run_reference(args, world, rank):
    import synth
    if rank != 0:
        return
    dims, U, src, csw, kappa, tbc = synth.config_inputs(CFG)
    V = int(np.prod(dims))
    per_step = max(0.02, min(args.ref_seconds, 150.0 / (args.steps + args.warmup)))
    smp = OracleSampler(dims, U, src, csw, kappa, tbc, per_step)
    vals, secs = [], []
    for i in range(args.warmup + args.steps):
        g, dt = smp.step()
        if i >= args.warmup:
            vals.append(g)
            secs.append(dt)
    value = statistics.median(vals)
    desc = smp.describe(statistics.median(secs))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFlop/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * FLOPS_PER_SITE * V / (value * 1e9),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Haar-like SU(3) links, Z2 source)",
        "config": {"workload": "Wilson-Clover M apply, 24^3x32, csw=1.0, kappa=0.125, antiperiodic t",
                   "lattice": list(dims), "sample": desc},
        "cpu_baseline": {"value": value, "unit": "GFlop/s", "cores": smp.cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "GFlop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1612_06556_gb300 as wc
    import synth

    stream = torch.cuda.current_stream()
    dims, U, src, csw, kappa, tbc = synth.config_inputs(CFG)
    V = int(np.prod(dims))
    lat = wc.Lattice(dims, tbc, stream=stream).load_gauge(U).load_clover(csw, kappa)
    nring = 4
    ins = [lat.field(wc.F32).load(src) for _ in range(nring)]
    outs = [lat.field(wc.F32) for _ in range(nring)]

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return reduce_max(x, world, "cuda")

    if args.apply_shape >= 0:   # pin one launch shape instead of the autotuner's pick
        lat.apply_shape(wc.F32, 0, args.apply_shape)
    for i in range(args.warmup):
        lat.apply_M(outs[i % nring], ins[i % nring])
    with ClockSampler(local) as clocks:
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(args.steps):
            lat.apply_M(outs[i % nring], ins[i % nring])
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        ms = max_over_ranks(ms)
        # end to end through the public API with host buffers: canonical
        # complex64 in (pinned, the FP32 apply's own precision) -> import ->
        # apply -> export -> host; the complex128 round trip beside it
        fin, fout = lat.field(wc.F32), lat.field(wc.F32)

        def e2e(host_in):
            host_out = torch.empty_like(host_in).pin_memory()
            for _ in range(2):
                fin.load(host_in)
                lat.apply_M(fout, fin)
                fout.store(host_out)
            barrier()
            t0 = time.perf_counter()
            for _ in range(args.e2e_steps):
                fin.load(host_in)
                lat.apply_M(fout, fin)
                fout.store(host_out)
            torch.cuda.synchronize()
            return max_over_ranks(1000 * (time.perf_counter() - t0) / args.e2e_steps)

        def e2e_pipelined(host_in):
            # asynchronous calls: the next step's host-to-device copy overlaps
            # this step's kernels and device-to-host copy
            host_out = torch.empty_like(host_in).pin_memory()
            for _ in range(2):
                fin.load_async(host_in)
                lat.apply_M(fout, fin)
                fout.store_async(host_out)
            lat.sync()
            barrier()
            t0 = time.perf_counter()
            for _ in range(args.e2e_steps):
                fin.load_async(host_in)
                lat.apply_M(fout, fin)
                fout.store_async(host_out)
            lat.sync()
            return max_over_ranks(1000 * (time.perf_counter() - t0) / args.e2e_steps)

        host64 = torch.from_numpy(src.astype(np.complex64)).pin_memory()
        e2e_ms = e2e_pipelined(host64)
        e2e_sync_ms = e2e(host64)
        e2e128_ms = e2e(torch.from_numpy(src).pin_memory())
        solve = solve_comparison(wc, lat, src, args) if not args.skip_solves else None
    clk = clocks.summary()
    shape = lat.apply_shape(wc.F32, 0)
    mdag_ms = time_applies(lat, outs, ins, "Mdag", 500, stream)
    fp64_apply = fp64_apply_timing(wc, lat, dims, src, stream)
    copy_gbs = copy_rate(BYTES_PER_SITE["f32"] * V, stream)
    multi = multi_rhs_apply(wc, lat, dims, ms / args.steps, stream)
    ras = ras_timing(wc, lat, dims, src, stream)
    split = split_mult_timing(wc, dims, U, src, csw, kappa, tbc, stream, ms / args.steps)
    point = point_source_solve(wc)
    large = large_lattice(wc, args) if not args.skip_large else None
    batch = batch_comparison(wc, args) if not args.skip_batch else None
    force = force_timing(wc, args) if not args.skip_force else None

    per_launch_ms = ms / args.steps
    flops = FLOPS_PER_SITE * V
    value = whole_job_rate(flops, world, per_launch_ms) / 1e9
    peak, peak_kind = measured_peaks()
    bytes_alg = BYTES_PER_SITE["f32"] * V
    achieved = bytes_alg / (per_launch_ms * 1e-3) / 1e9
    traffic = None
    if NCU_TRAFFIC["sources_sha"] == kernel_sources_sha():
        traffic = NCU_TRAFFIC["bytes_per_launch"]
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "GFlop/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_launch_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded Haar-like SU(3) links, Z2 source)",
        "config": {"workload": "Wilson-Clover M apply, 24^3x32, FP32 storage and arithmetic, csw=1.0, "
                               "kappa=0.125, antiperiodic t",
                   "lattice": list(dims), "l2": "inputs 297 MB per step > 129 MB L2; 4 rotating field pairs",
                   "parallelism": f"replicas{world}",
                   "launch_shape": {"threads": shape[0], "tile": list(shape[1]), "reg_cap": shape[2] % 4,
                                    "persistent": (shape[2] // 4) % 4, "pdl": shape[2] // 16,
                                    "chosen_by": "pinned" if args.apply_shape >= 0 else "autotuner"}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "k_apply<P32, M>",
                     "peak_kind": peak_kind, "algorithmic_bytes_per_launch": bytes_alg,
                     "same_size_copy_gbs": copy_gbs, "frac_of_same_size_copy": achieved / copy_gbs},
        "e2e": {"value": whole_job_rate(flops, world, e2e_ms) / 1e9, "unit": "GFlop/s",
                "h2d_bytes_per_step": V * 12 * 8, "d2h_bytes_per_step": V * 12 * 8,
                "ms_per_step": e2e_ms, "host_data": "complex64, page-locked",
                "calls": "wc_field_import_async -> wc_apply_M -> wc_field_export_async per step, wc_sync at the end",
                "synchronous_calls_ms_per_step": e2e_sync_ms, "complex128_synchronous_ms_per_step": e2e128_ms},
        "gpu_launches": args.steps,
        "clocks": clk,
    }
    if solve is not None:
        line["solve"] = solve
    line["apply_mdag"] = {"ms": mdag_ms, "gflops": flops / (mdag_ms * 1e-3) / 1e9,
                          "roofline_frac": bytes_alg / (mdag_ms * 1e-3) / 1e9 / peak}
    line["apply_fp64"] = fp64_apply
    if large is not None:
        line["large_32x32x32x64"] = large
    if batch is not None:
        line["batch"] = batch
    if force is not None:
        line["force"] = force
    line["apply_multi"] = multi
    line["ras"] = ras
    line["split_mult"] = split
    line["point_source_8x8x8x8"] = point
    if world == 1 and not args.skip_cpu:
        smp = OracleSampler(dims, U, src, csw, kappa, tbc, args.ref_seconds)
        g, dt = smp.step()
        line["cpu_baseline"] = {"value": g, "unit": "GFlop/s", "cores": smp.cores, "kind": "oracle",
                                "sample": smp.describe(dt),
                                "point_source_solve_8x8x8x8": oracle_point_source_solve()}
    print(json.dumps(line), flush=True)


def small_batch(wc):
    """The same 36-RHS structure on small lattices (8^4, 8^3x12, 8^3x16),
    where one BiCGStab step is tens of microseconds of GPU work and the
    per-step host read-back of a sequential solve is of the same order: the
    graph-driven batch (device-side loop, no host round trips) against 36
    sequential solves, even-odd reliable update to 1e-10."""
    import synth
    lats, bs = [], []
    for i, dims in enumerate([(8, 8, 8, 8), (8, 8, 8, 12), (8, 8, 8, 16)]):
        U = synth.exp_links(dims, 0.3, 1200 + 10 * i)
        lat = wc.Lattice(dims, -1).load_gauge(U).load_clover(1.0, 0.124)
        for spin in range(4):
            for colour in range(3):
                lats.append(lat)
                bs.append(lat.field(wc.F64).load(synth.point_source(dims, spin, colour)))
    prm = wc.solve_params(tol=1e-10, max_iter=5000, precond=wc.PRECOND_NONE, solver=wc.SOLVER_RELIABLE,
                          delta=0.01, even_odd=True)

    def batch():
        xs = [lat.field(wc.F64) for lat in lats]
        t0 = time.perf_counter()
        infos = wc.solve_batch(lats, xs, bs, prm, check=False)
        dt = time.perf_counter() - t0
        for x in xs:
            x.close()
        return infos, dt

    def sequential():
        t0 = time.perf_counter()
        infos = []
        for lat, b in zip(lats, bs):
            x = lat.field(wc.F64)
            infos.append(lat.solve(x, b, prm, check=False))
            x.close()
        return infos, time.perf_counter() - t0

    batch()
    sequential()
    ib, tb = batch()
    iseq, ts = sequential()
    return {"rhs": len(lats), "lattices": [[8, 8, 8, 8], [8, 8, 8, 12], [8, 8, 8, 16]],
            "solver": "even-odd reliable update, tol 1e-10", "batch_seconds": tb, "sequential_seconds": ts,
            "speedup_vs_sequential": ts / tb, "all_ok": all(i.status == 0 for i in ib + iseq)}


def batch_comparison(wc, args):
    """36 right-hand sides (12 spin-colour point sources on each of
    24^3x48, 16^3x32 and 32^3x32, each lattice with its own exp(0.3 iH)
    gauge field) to 1e-10 with FP32 RAS (block shapes from the autotuner):
    one graph-launched batch (reliable-update solver; also the flexible FP64
    outer solver, and the even-odd reliable-update solver without RAS, whose
    12 sources per lattice step in lockstep groups with FP32 Krylov vectors
    and in one branch each with FP16 vectors, each timed also with the other
    schedule) vs 36 sequential solves on the same GPU."""
    import synth
    cfg = synth.CONFIGS[4]
    lats, bs, srcs = [], [], []
    for i, dims in enumerate(cfg["dims"]):
        U = synth.gauge_for(cfg["gauge"], dims, 1100 + 10 * i)
        lat = wc.Lattice(dims, cfg["tbc"]).load_gauge(U).load_clover(cfg["csw"], cfg["kappa"])
        del U
        for spin in range(4):
            for colour in range(3):
                lats.append(lat)
                bs.append(lat.field(wc.F64).load(synth.point_source(dims, spin, colour)))
    params = wc.solve_params(tol=1e-10, max_iter=2000, precond=wc.PRECOND_RAS, inner_prec=wc.F32,
                             block=(0, 0, 0, 0), solver=wc.SOLVER_RELIABLE, delta=0.01)
    shapes = {}
    for lat, b in zip(lats[::12], bs[::12]):
        shapes["x".join(map(str, lat.dims))] = list(lat.ras_autotune(b, params)[0])

    def run_batch(prm):
        xs = [lat.field(wc.F64) for lat in lats]
        t0 = time.perf_counter()
        infos = wc.solve_batch(lats, xs, bs, prm, check=False)
        dt = time.perf_counter() - t0
        for x in xs:
            x.close()
        return infos, dt

    run_batch(params)                       # warm-up: allocations, launch-shape tuning
    infos, t_batch = run_batch(params)
    flex = wc.solve_params(tol=1e-10, max_iter=2000, precond=wc.PRECOND_RAS, inner_prec=wc.F32,
                           block=(0, 0, 0, 0), solver=wc.SOLVER_FLEXIBLE)
    infos_flex, t_flex = run_batch(flex)
    eo = wc.solve_params(tol=1e-10, max_iter=5000, precond=wc.PRECOND_NONE, solver=wc.SOLVER_RELIABLE,
                         delta=0.01, even_odd=True)
    run_batch(eo)                           # warm-up: clover inverses, half-lattice fields
    infos_eo, t_eo = run_batch(eo)
    # the same batch with one graph branch per right-hand side instead of
    # lockstep groups (one multi-RHS Schur launch per group and step)
    os.environ["WC_BATCH_LOCKSTEP"] = "0"
    try:
        infos_eo_br, t_eo_br = run_batch(eo)
    finally:
        del os.environ["WC_BATCH_LOCKSTEP"]
    eo_h16 = wc.solve_params(tol=1e-10, max_iter=5000, precond=wc.PRECOND_NONE, solver=wc.SOLVER_RELIABLE,
                             delta=0.01, krylov_prec=wc.F16, even_odd=True)
    run_batch(eo_h16)
    infos_eo_h16, t_eo_h16 = run_batch(eo_h16)
    # FP16 vectors take one branch per right-hand side by default; the
    # lockstep schedule for comparison
    os.environ["WC_BATCH_LOCKSTEP"] = "1"
    try:
        infos_eo_h16_ls, t_eo_h16_ls = run_batch(eo_h16)
    finally:
        del os.environ["WC_BATCH_LOCKSTEP"]
    # the same with the FP64 operator steps in double-FP32 arithmetic
    for lat in lats[::12]:
        lat.set_fp64_arith(wc.ARITH_DF32)
    run_batch(eo_h16)
    infos_eo_h16_df, t_eo_h16_df = run_batch(eo_h16)
    for lat in lats[::12]:
        lat.set_fp64_arith(wc.ARITH_F64)
    eo_ras = wc.solve_params(tol=1e-10, max_iter=5000, precond=wc.PRECOND_RAS, inner_prec=wc.F32,
                             block=(4, 4, 4, 4), solver=wc.SOLVER_RELIABLE, delta=0.01, even_odd=True)
    run_batch(eo_ras)
    infos_eo_ras, t_eo_ras = run_batch(eo_ras)
    # the same with RAS on the blocks' own Schur complements
    eo_ras_schur = wc.solve_params(tol=1e-10, max_iter=5000, precond=wc.PRECOND_RAS, inner_prec=wc.F32,
                                   block=(4, 4, 4, 4), solver=wc.SOLVER_RELIABLE, delta=0.01, even_odd=True,
                                   ras_schur=True)
    run_batch(eo_ras_schur)
    infos_eo_ras_s, t_eo_ras_s = run_batch(eo_ras_schur)
    t0 = time.perf_counter()
    seq_eo = []
    for lat, b in zip(lats, bs):
        x = lat.field(wc.F64)
        seq_eo.append(lat.solve(x, b, eo, check=False))
        x.close()
    t_seq_eo = time.perf_counter() - t0
    t0 = time.perf_counter()
    seq = []
    for lat, b in zip(lats, bs):
        x = lat.field(wc.F64)
        blk = shapes["x".join(map(str, lat.dims))]
        seq.append(lat.solve(x, b, tol=1e-10, max_iter=2000, precond=wc.PRECOND_RAS, inner_prec=wc.F32,
                             block=blk, solver=wc.SOLVER_RELIABLE, delta=0.01, check=False))
        x.close()
    t_seq = time.perf_counter() - t0
    return {"rhs": len(lats), "lattices": [list(d) for d in cfg["dims"]],
            "solver": "reliable update (FP32 BiCGStab + FP32 RAS, FP64 refreshes, delta 0.01), tol 1e-10",
            "batch_seconds": t_batch, "sequential_seconds": t_seq, "speedup_vs_sequential": t_seq / t_batch,
            "max_true_rel_resid": max(i.true_rel_resid for i in infos),
            "all_ok": all(i.status == 0 for i in infos),
            "steps": [min(i.iters for i in infos), max(i.iters for i in infos)],
            "sequential_all_ok": all(i.status == 0 for i in seq),
            "flexible_batch_seconds": t_flex, "flexible_all_ok": all(i.status == 0 for i in infos_flex),
            "flexible_steps": [min(i.iters for i in infos_flex), max(i.iters for i in infos_flex)],
            "even_odd_batch_seconds": t_eo, "even_odd_all_ok": all(i.status == 0 for i in infos_eo),
            "even_odd_branch_per_rhs_batch_seconds": t_eo_br,
            "even_odd_branch_per_rhs_all_ok": all(i.status == 0 for i in infos_eo_br),
            "even_odd_fp16_vectors_lockstep_batch_seconds": t_eo_h16_ls,
            "even_odd_fp16_vectors_lockstep_all_ok": all(i.status == 0 for i in infos_eo_h16_ls),
            "even_odd_sequential_seconds": t_seq_eo, "even_odd_sequential_all_ok": all(i.status == 0 for i in seq_eo),
            "even_odd_fp16_vectors_batch_seconds": t_eo_h16,
            "even_odd_fp16_vectors_all_ok": all(i.status == 0 for i in infos_eo_h16),
            "even_odd_fp16_vectors_df32_batch_seconds": t_eo_h16_df,
            "even_odd_fp16_vectors_df32_all_ok": all(i.status == 0 for i in infos_eo_h16_df),
            "even_odd_ras_batch_seconds": t_eo_ras, "even_odd_ras_all_ok": all(i.status == 0 for i in infos_eo_ras),
            "even_odd_ras_schur_batch_seconds": t_eo_ras_s,
            "even_odd_ras_schur_all_ok": all(i.status == 0 for i in infos_eo_ras_s),
            "even_odd_ras_schur_steps": [min(i.iters for i in infos_eo_ras_s), max(i.iters for i in infos_eo_ras_s)],
            "even_odd_ras_steps": [min(i.iters for i in infos_eo_ras), max(i.iters for i in infos_eo_ras)],
            "even_odd_steps": [min(i.iters for i in infos_eo), max(i.iters for i in infos_eo)],
            "even_odd_max_true_rel_resid": max(i.true_rel_resid for i in infos_eo),
            "ras_blocks_autotuned": shapes,
            "small_lattices": small_batch(wc)}


def multi_rhs_apply(wc, lat, dims, single_ms, stream, n=12, reps=100):
    """The 12 spin-colour sources of a propagator through one multi-RHS
    launch (wc_apply_multi) on the same lattice: links and clover read once
    per site for all 12 fields, 192 + 480/12 = 232 B per site and field."""
    import torch
    import synth
    V = int(np.prod(dims))
    ins = [lat.field(wc.F32).load(synth.z2_source(dims, 3000 + r)) for r in range(n)]
    outs = [lat.field(wc.F32) for _ in range(n)]
    for _ in range(3):
        lat.apply_multi(outs, ins)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        lat.apply_multi(outs, ins)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    for f in ins + outs:
        f.close()
    bps = 192 + 480 / n
    peak, _ = measured_peaks()
    gbs = bps * n * V / (ms * 1e-3) / 1e9
    return {"rhs": n, "ms_per_launch": ms, "gflops": FLOPS_PER_SITE * V * n / (ms * 1e-3) / 1e9,
            "bytes_per_site_per_rhs": bps, "algorithmic_gbs": gbs, "roofline_frac": gbs / peak,
            "speedup_vs_single_applies": n * single_ms / ms}


def fp32_fma_peak():
    """Measured FP32 FMA throughput (TFLOP/s): cuBLAS FP32 GEMM (TF32 off, so
    it runs on the FMA pipe, not the tensor cores), 8192^3, best of 5 --
    the denominator of the RAS block solver's effective rate."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        n = 8192
        a = torch.randn(n, n, device="cuda")
        b = torch.randn(n, n, device="cuda")
        torch.mm(a, b)
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.mm(a, b)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return 2.0 * n ** 3 / (best * 1e-3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def ras_timing(wc, lat, dims, src, stream, reps=50):
    """One RAS application (4^4 blocks, overlap 1, 4 MR steps) at 24^3x32 on
    FP32 and FP16 storage: seconds per application and the effective rate
    4 MR steps x 1296 extended sites x blocks x (1824 + 96) flop."""
    import torch
    V = int(np.prod(dims))
    blocks = V // 256
    flops = 4 * 1296 * blocks * (FLOPS_PER_SITE + 96)
    peak = fp32_fma_peak()
    out = {"blocks": blocks, "fp32_fma_peak_tflops_measured": peak}
    for name, prec in (("f32", wc.F32), ("f16", wc.F16)):
        a, z = lat.field(prec).load(src), lat.field(prec)
        for _ in range(3):
            lat.ras(z, a)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            lat.ras(z, a)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        tf = flops / (ms * 1e-3) / 1e12
        out[name] = {"ms": ms, "effective_tflops": tf, "frac_of_fp32_fma_peak": tf / peak}
        # the same blocks on the even-odd system: MR on each block's
        # even-site Schur complement (648 even sites per extended block; the
        # time includes the split of the input and the merge of the output)
        for _ in range(3):
            lat.ras_schur(z, a)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            lat.ras_schur(z, a)
        e1.record(stream)
        torch.cuda.synchronize()
        out["schur_" + name] = {"ms": e0.elapsed_time(e1) / reps}
        a.close()
        z.close()
    return out


def periodic_box(dims, a, start, extents):
    """The box [start, start + extents) of a canonical [V, ...] array,
    coordinates periodic (input slicing for the sub-domains)."""
    lx, ly, lz, lt = dims
    g = a.reshape((lt, lz, ly, lx) + a.shape[1:])
    for m in range(4):
        idx = np.arange(start[m], start[m] + extents[m]) % dims[m]
        g = np.take(g, idx, axis=3 - m)
    return np.ascontiguousarray(g).reshape((-1,) + a.shape[1:])


def split_mult_timing(wc, dims, U, src, csw, kappa, tbc, stream, whole_ms, reps=100):
    """The overlapped MULT (paper Sec. 2.2) on one GPU: the lattice cut in two
    along t into sub-domains of half the time extent, each step timed by
    itself on the stream -- halo pack of both sub-domains, the device copies
    standing in for the exchange, interior and surface launches -- against
    the whole-lattice FP32 apply.  On a multi-GPU machine the interior launch
    would run while the buffers travel."""
    import torch
    lt = dims[3] // 2
    local = (dims[0], dims[1], dims[2], lt)
    subs, fin, fout, send, recv = [], [], [], [], []
    for r in range(2):
        off = (0, 0, 0, r * lt)
        s = wc.SubDomain(local, dims, off, tbc, stream=stream)
        s.load_gauge(periodic_box(dims, U, (0, 0, 0, off[3] - 1), (dims[0], dims[1], dims[2], lt + 2)))
        s.load_clover(csw, kappa)
        subs.append(s)
        fin.append(s.field(wc.F32).load(periodic_box(dims, src, off, local)))
        fout.append(s.field(wc.F32))
        nb = s.halo_bytes(3)
        send.append([None] * 6 + [torch.empty(nb // 4, dtype=torch.float32, device="cuda") for _ in range(2)])
        recv.append([None] * 6 + [torch.empty(nb // 4, dtype=torch.float32, device="cuda") for _ in range(2)])

    def pack():
        for r in range(2):
            subs[r].halo_pack(fin[r], send[r])

    def exchange():
        for r in range(2):
            recv[r][7].copy_(send[1 - r][6])   # from the upper neighbour: its lower-face data
            recv[r][6].copy_(send[1 - r][7])   # from the lower neighbour: its upper-face data

    def interior():
        for r in range(2):
            subs[r].apply_interior(fout[r], fin[r])

    def surface():
        for r in range(2):
            subs[r].apply_surface(fout[r], fin[r], recv[r])

    out = {"cut": "t in two", "sub_domain": list(local), "face_bytes_per_direction": subs[0].halo_bytes(3)}
    for name, fn in (("pack", pack), ("exchange_copies", exchange), ("interior", interior), ("surface", surface)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        out[name + "_us"] = 1000 * e0.elapsed_time(e1) / reps
    out["split_total_us"] = out["pack_us"] + out["exchange_copies_us"] + out["interior_us"] + out["surface_us"]
    out["whole_lattice_apply_us"] = 1000 * whole_ms
    out["interior_share"] = out["interior_us"] / (out["pack_us"] + out["interior_us"] + out["surface_us"])
    for f in fin + fout:
        f.close()
    for s in subs:
        s.close()
    return out


def copy_rate(total_bytes, stream, reps=200):
    """Read+write GB/s of a plain device copy (torch) that moves the same
    bytes per launch as one apply, rotating over 4 buffer pairs: context for
    the roofline fraction, since the measured peak comes from 4.3 GB copies
    and a 55 us launch pays its ramp-up and drain on every call."""
    import torch
    n = int(total_bytes // 8)   # float32 elements per buffer (half read, half written)
    gen = torch.Generator(device="cuda").manual_seed(1)
    # random contents: a constant buffer could be moved faster than real data
    src = [torch.randn(n, device="cuda", generator=gen) for _ in range(4)]
    dst = [torch.empty(n, device="cuda") for _ in range(4)]
    for i in range(8):
        dst[i % 4].copy_(src[i % 4])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(reps):
        dst[i % 4].copy_(src[i % 4])
    e1.record(stream)
    torch.cuda.synchronize()
    return 8 * n / (e0.elapsed_time(e1) / reps * 1e-3) / 1e9


def time_applies(lat, outs, ins, kind, steps, stream):
    """Average device time (ms) of `steps` applies rotating over the field
    pairs, CUDA events on the lattice's stream."""
    import torch
    fn = {"M": lat.apply_M, "Mdag": lat.apply_Mdag}[kind]
    for i in range(3):
        fn(outs[i % len(outs)], ins[i % len(ins)])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):
        fn(outs[i % len(outs)], ins[i % len(ins)])
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def large_lattice(wc, args):
    """The 32^3x64 workload (exp(0.25 iH) links, csw 1.6, kappa 0.128,
    Gaussian source): FP32 and FP16-storage applies with their roofline
    fractions and errors against this library's FP64 apply (the oracle
    parity of all three precisions is the tests' job); nested solves to
    1e-10 (FP16-storage RAS inner, and even-odd FP32 inner) with their FP64
    true residuals; with --large-solve N also the even-odd reliable-update
    solve within N steps (it stagnates here)."""
    import torch
    import synth
    dims, U, src, csw, kappa, tbc = synth.config_inputs(3)
    V = int(np.prod(dims))
    stream = torch.cuda.current_stream()
    lat = wc.Lattice(dims, tbc, stream=stream).load_gauge(U).load_clover(csw, kappa)
    peak, _ = measured_peaks()
    out = {"lattice": list(dims)}
    f64_in, f64_out = lat.field(wc.F64).load(src), lat.field(wc.F64)
    lat.apply_M(f64_out, f64_in)
    ref = f64_out.store(np.zeros_like(src))
    f64_in.close()
    f64_out.close()
    for name, prec, bps in (("f32", wc.F32, BYTES_PER_SITE["f32"]), ("f16", wc.F16, BYTES_PER_SITE["f16"])):
        if args.apply_shape >= 0:
            lat.apply_shape(prec, 0, args.apply_shape)
        ins = [lat.field(prec).load(src) for _ in range(2)]
        outs = [lat.field(prec) for _ in range(2)]
        ms = time_applies(lat, outs, ins, "M", 200, stream)
        lat.apply_M(outs[0], ins[0])
        res = outs[0].store(np.zeros_like(src))
        err = float(np.linalg.norm(res - ref) / np.linalg.norm(ref))
        gbs = bps * V / (ms * 1e-3) / 1e9
        out["apply_" + name] = {"ms": ms, "gflops": FLOPS_PER_SITE * V / (ms * 1e-3) / 1e9, "algorithmic_gbs": gbs,
                                "roofline_frac": gbs / peak, "bytes_per_site": bps,
                                "rel_err_vs_fp64_apply": err}
        for f in ins + outs:
            f.close()
    # near-critical (kappa 0.128, csw 1.6): plain and reliable-update
    # BiCGStab stagnate near 1e-8 here; the paper's three-level structure
    # (FP64 flexible outer, FP32 inner BiCGStab) converges.  FP16 storage as
    # prescribed: inner BiCGStab + RAS with FP16 spinors, links and clover,
    # on the full lattice and on the even-odd operator (the paper's inner
    # configuration); fastest: inner BiCGStab on the even-odd operator.
    b = lat.field(wc.F64).load(src)
    solves = [("solve_nested_ras_f16", dict(precond=wc.PRECOND_RAS, inner_prec=wc.F16, max_iter=20)),
              ("solve_eo_nested_ras_f16", dict(precond=wc.PRECOND_RAS, inner_prec=wc.F16, even_odd=True,
                                               max_iter=20)),
              ("solve_eo_nested_f32", dict(precond=wc.PRECOND_NONE, even_odd=True, max_iter=60)),
              ("solve_eo_nested_h16", dict(precond=wc.PRECOND_NONE, even_odd=True, krylov_prec=wc.F16,
                                           max_iter=60))]
    if args.large_solve:
        solves.append(("solve_eo_reliable_f32", dict(precond=wc.PRECOND_NONE, even_odd=True, max_iter=args.large_solve,
                                                     solver=wc.SOLVER_RELIABLE, delta=0.01)))
    for name, kw in solves:
        kw.setdefault("solver", wc.SOLVER_NESTED)
        x = lat.field(wc.F64)
        info = lat.solve(x, b, tol=1e-10, inner_tol=0.01, inner_iters=100, check=False, **kw)
        out[name] = {"seconds": info.seconds, "steps": info.iters, "true_rel_resid": info.true_rel_resid,
                     "status": wc.STATUS.get(info.status, info.status)}
        x.close()
    return out


def force_timing(wc, args):
    """S = phi^+ (M^+ M)^-1 phi and its force on 16^3x32 (kappa 0.12,
    csw 1.0, exp(0.3 iH) links, Gaussian phi): two solves to 1e-12 (FP64
    flexible BiCGStab + FP32 RAS, or even-odd reliable update), then the
    force kernels."""
    import torch
    import synth
    dims, U, phi, csw, kappa, tbc = synth.config_inputs(5)
    lat = wc.Lattice(dims, tbc).load_gauge(U).load_clover(csw, kappa)
    f_phi = lat.field(wc.F64).load(phi)
    # the force stays on the device (a CUDA tensor), as an HMC update would use it
    F = torch.zeros((int(np.prod(dims)), 4, 3, 3), dtype=torch.complex128, device="cuda")
    out = {"lattice": list(dims), "force_buffer": "device"}
    for name, kw, what in (
            ("flexible_ras", dict(tol=1e-12, precond=wc.PRECOND_RAS, inner_prec=wc.F32),
             "FP64 flexible BiCGStab + FP32 RAS"),
            ("eo_reliable", dict(tol=1e-12, precond=wc.PRECOND_NONE, even_odd=True, solver=wc.SOLVER_RELIABLE),
             "even-odd FP32 BiCGStab with FP64 reliable updates"),
            ("eo_reliable_df32", dict(tol=1e-12, precond=wc.PRECOND_NONE, even_odd=True, solver=wc.SOLVER_RELIABLE),
             "even-odd FP32 BiCGStab with reliable updates, FP64 operator steps in double-FP32")):
        lat.set_fp64_arith(wc.ARITH_DF32 if name.endswith("_df32") else wc.ARITH_F64)
        lat.action_force(f_phi, F, **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        torch.cuda.nvtx.range_push("force_" + name)   # lets a profiler select the timed call
        S = lat.action_force(f_phi, F, **kw)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[name] = {"seconds": dt, "S": S, "solves": f"M^+ Y = phi then M X = Y, {what}, tol 1e-12"}
    return out


def solve_comparison(wc, lat, src, args):
    """Mixed-precision RAS-BiCGStab (FP32 and FP16 inner; flexible, reliable
    update, nested) and even-odd (Schur complement) solves vs plain FP64
    BiCGStab, all to 1e-10 from x0 = 0, on the same GPU and lattice."""
    import torch
    b = lat.field(wc.F64).load(src)
    out = {}
    for name, kw in (("mixed_ras_f32", dict(precond=wc.PRECOND_RAS, inner_prec=wc.F32)),
                     ("mixed_ras_f16", dict(precond=wc.PRECOND_RAS, inner_prec=wc.F16)),
                     ("reliable_ras_f32", dict(precond=wc.PRECOND_RAS, inner_prec=wc.F32,
                                               solver=wc.SOLVER_RELIABLE, delta=0.01)),
                     ("reliable_ras_f16", dict(precond=wc.PRECOND_RAS, inner_prec=wc.F16,
                                               solver=wc.SOLVER_RELIABLE, delta=0.01)),
                     ("nested_ras_f16", dict(precond=wc.PRECOND_RAS, inner_prec=wc.F16,
                                             solver=wc.SOLVER_NESTED, inner_tol=0.01, inner_iters=100)),
                     ("fp64_plain", dict(precond=wc.PRECOND_NONE)),
                     ("eo_fp64_plain", dict(precond=wc.PRECOND_NONE, even_odd=True)),
                     ("eo_reliable_f32", dict(precond=wc.PRECOND_NONE, solver=wc.SOLVER_RELIABLE, delta=0.01,
                                              even_odd=True)),
                     ("eo_reliable_f32_delta1e-4", dict(precond=wc.PRECOND_NONE, solver=wc.SOLVER_RELIABLE,
                                                        delta=1e-4, even_odd=True)),
                     ("eo_nested_f32", dict(precond=wc.PRECOND_NONE, solver=wc.SOLVER_NESTED, inner_tol=0.01,
                                            inner_iters=100, even_odd=True)),
                     ("eo_reliable_ras_f16", dict(precond=wc.PRECOND_RAS, inner_prec=wc.F16,
                                                  solver=wc.SOLVER_RELIABLE, delta=0.01, even_odd=True)),
                     ("eo_reliable_ras_schur_f16", dict(precond=wc.PRECOND_RAS, inner_prec=wc.F16,
                                                        solver=wc.SOLVER_RELIABLE, delta=0.01, even_odd=True,
                                                        ras_schur=True)),
                     ("eo_reliable_ras_schur_f32", dict(precond=wc.PRECOND_RAS, inner_prec=wc.F32,
                                                        solver=wc.SOLVER_RELIABLE, delta=0.01, even_odd=True,
                                                        ras_schur=True)),
                     ("eo_reliable_h16", dict(precond=wc.PRECOND_NONE, solver=wc.SOLVER_RELIABLE, delta=0.01,
                                              krylov_prec=wc.F16, even_odd=True)),
                     ("eo_nested_h16", dict(precond=wc.PRECOND_NONE, solver=wc.SOLVER_NESTED, inner_tol=0.01,
                                            inner_iters=100, krylov_prec=wc.F16, even_odd=True)),
                     # the same solvers with their FP64 operator steps in double-FP32 arithmetic
                     ("fp64_plain_df32", dict(precond=wc.PRECOND_NONE)),
                     ("mixed_ras_f32_df32", dict(precond=wc.PRECOND_RAS, inner_prec=wc.F32)),
                     ("eo_fp64_plain_df32", dict(precond=wc.PRECOND_NONE, even_odd=True)),
                     ("reliable_ras_f16_df32", dict(precond=wc.PRECOND_RAS, inner_prec=wc.F16,
                                                    solver=wc.SOLVER_RELIABLE, delta=0.01)),
                     ("eo_reliable_f32_df32", dict(precond=wc.PRECOND_NONE, solver=wc.SOLVER_RELIABLE, delta=0.01,
                                                   even_odd=True)),
                     ("eo_reliable_h16_df32", dict(precond=wc.PRECOND_NONE, solver=wc.SOLVER_RELIABLE,
                                                   delta=0.01, krylov_prec=wc.F16, even_odd=True)),
                     ("eo_reliable_h16_delta1e-4_df32", dict(precond=wc.PRECOND_NONE, solver=wc.SOLVER_RELIABLE,
                                                             delta=1e-4, krylov_prec=wc.F16, even_odd=True)),
                     ("eo_nested_h16_df32", dict(precond=wc.PRECOND_NONE, solver=wc.SOLVER_NESTED,
                                                 inner_tol=0.01, inner_iters=100, krylov_prec=wc.F16,
                                                 even_odd=True))):
        if args.solves and name not in args.solves.split(","):
            continue
        lat.set_fp64_arith(wc.ARITH_DF32 if name.endswith("_df32") else wc.ARITH_F64)
        x = lat.field(wc.F64)
        lat.solve(x, b, tol=1e-10, max_iter=20000, check=False, **kw)   # warm-up (allocations)
        x.close()
        x = lat.field(wc.F64)
        torch.cuda.nvtx.range_push(name)   # lets a profiler select the timed solve
        info = lat.solve(x, b, tol=1e-10, max_iter=20000, check=False, **kw)
        torch.cuda.nvtx.range_pop()
        out[name] = {"seconds": info.seconds, "iters": info.iters, "true_rel_resid": info.true_rel_resid,
                     "status": wc.STATUS.get(info.status, info.status)}
        x.close()
    lat.set_fp64_arith(wc.ARITH_F64)
    if "fp64_plain" in out and "mixed_ras_f32" in out:
        out["speedup_mixed_f32_vs_fp64"] = out["fp64_plain"]["seconds"] / out["mixed_ras_f32"]["seconds"]
    # mixed-precision solvers only (not the FP64-only ones, in either arithmetic)
    ok = [k for k, v in out.items() if isinstance(v, dict) and "fp64_plain" not in k and v["status"] == "WC_OK"]
    if ok and "fp64_plain" in out:
        best = min(ok, key=lambda k: out[k]["seconds"])
        out["fastest_mixed"] = best
        out["speedup_fastest_mixed_vs_fp64"] = out["fp64_plain"]["seconds"] / out[best]["seconds"]
    out["ras"] = ("4^4 blocks, overlap 1, 4 MR iterations; _ras_schur_: RAS on block Schur complements "
                  "(wc_ras_params.schur)")
    out["df32"] = "suffix _df32: FP64 operator steps in double-FP32 arithmetic (wc_set_fp64_arith)"
    return out


def point_source_solve(wc):
    """The 8^3x8 point-source system (exp(0.3 iH) links, csw 1.0, kappa
    0.12, antiperiodic t): plain FP64 BiCGStab to 1e-12 on the GPU, second of
    two identical solves."""
    import synth
    dims, U, src, csw, kappa, tbc = synth.config_inputs(1)
    lat = wc.Lattice(dims, tbc).load_gauge(U).load_clover(csw, kappa)
    b = lat.field(wc.F64).load(src)
    out = {"lattice": list(dims), "solver": "plain FP64 BiCGStab, tol 1e-12"}
    for _ in range(2):
        x = lat.field(wc.F64)
        info = lat.solve(x, b, tol=1e-12, check=False)
        x.close()
    out.update({"seconds": info.seconds, "iters": info.iters, "true_rel_resid": info.true_rel_resid,
                "status": wc.STATUS.get(info.status, info.status)})
    # the same solve as a one-right-hand-side graph batch: the BiCGStab loop
    # runs on the device, no host read-back per step
    for _ in range(2):
        x = lat.field(wc.F64)
        t0 = time.perf_counter()
        binfo = wc.solve_batch([lat], [x], [b], tol=1e-12, check=False)[0]
        dt = time.perf_counter() - t0
        x.close()
    out["graph_batch"] = {"seconds": dt, "iters": binfo.iters, "true_rel_resid": binfo.true_rel_resid,
                          "status": wc.STATUS.get(binfo.status, binfo.status)}
    lat.close()
    return out


def oracle_point_source_solve():
    """The same system solved by the CPU oracle's FP64 BiCGStab (host
    cores), for the reported CPU baseline."""
    import oracle
    import synth
    dims, U, src, csw, kappa, tbc = synth.config_inputs(1)
    op = oracle.Operator(dims, U, csw, kappa, tbc)
    t0 = time.perf_counter()
    res = oracle.bicgstab(op.M, src, tol=1e-12)
    return {"seconds": time.perf_counter() - t0, "iters": int(res.iters)}


def fp64_apply_timing(wc, lat, dims, src, stream, steps=60):
    """The FP64 operator on FP64 fields at the bench lattice: FP64
    arithmetic against double-FP32 arithmetic (each value a pair of floats,
    FP32 pipes), same 1536 B per site; rate in FP64-equivalent flops and the
    largest difference between the two results relative to the largest
    output."""
    import torch
    V = int(np.prod(dims))
    ins = [lat.field(wc.F64).load(src * (1.0 + 0.1 * k)) for k in range(4)]
    outs = [lat.field(wc.F64) for _ in range(4)]
    res = {}
    got = {}
    for name, mode in (("f64", wc.ARITH_F64), ("df32", wc.ARITH_DF32)):
        lat.set_fp64_arith(mode)
        ms = time_applies(lat, outs, ins, "M", steps, stream)
        lat.apply_M(outs[0], ins[0])
        got[name] = outs[0].store(np.zeros_like(src))
        # gbs: on the 1536 B this layout moves (18-real links); gbs_1344: on
        # 1344 B per site, the compulsory bytes with 12-real links
        res[name] = {"ms": ms, "fp64_equiv_tflops": FLOPS_PER_SITE * V / (ms * 1e-3) / 1e12,
                     "gbs": BYTES_PER_SITE["f64"] * V / (ms * 1e-3) / 1e9,
                     "gbs_1344": 1344 * V / (ms * 1e-3) / 1e9}
    lat.set_fp64_arith(wc.ARITH_F64)
    for f in ins + outs:
        f.close()
    res["speedup_df32_vs_f64"] = res["f64"]["ms"] / res["df32"]["ms"]
    res["df32_max_diff_rel"] = float(np.max(np.abs(got["df32"] - got["f64"])) / np.max(np.abs(got["f64"])))
    return res


def profile_run(args):
    """A small, self-contained workload for ncu captures: the config-2 input
    recipe on --profile-dims, warm-ups, then --steps launches of one kernel
    (applies through the autotuned or pinned shape, or RAS with 4^4 blocks,
    overlap 1, 4 MR steps)."""
    import torch
    import paper_1612_06556_gb300 as wc
    import synth
    dims = tuple(int(d) for d in args.profile_dims.split(","))
    U = synth.haar_links(dims, 1002)
    src = synth.z2_source(dims, 2002)
    lat = wc.Lattice(dims, -1).load_gauge(U).load_clover(1.0, 0.125)
    which = (args.profile_apply or args.profile_ras or args.profile_schur_multi or args.profile_ras_schur or
             args.profile_apply_multi)
    prec = {"f32": wc.F32, "f16": wc.F16, "f64": wc.F64}[which]
    if args.profile_apply and args.apply_shape >= 0:
        lat.apply_shape(prec, 0, args.apply_shape)
    a, b = lat.field(prec).load(src), lat.field(prec)
    if args.profile_schur_multi or args.profile_apply_multi:
        ins = [lat.field(prec).load(synth.point_source(dims, spin=k % 4, colour=k // 4)) for k in range(12)]
        outs = [lat.field(prec) for _ in range(12)]
        if args.profile_apply_multi:
            step = lambda: lat.apply_multi(outs, ins)   # noqa: E731
        else:
            step = lambda: lat.apply_schur_multi(outs, ins)   # noqa: E731
    elif args.profile_apply:
        step = lambda: lat.apply_M(b, a)   # noqa: E731
    elif args.profile_ras_schur:
        step = lambda: lat.ras_schur(b, a)   # noqa: E731
    else:
        step = lambda: lat.ras(b, a)   # noqa: E731
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    kind = ("apply" if args.profile_apply else "ras" if args.profile_ras else
            "ras_schur" if args.profile_ras_schur else "apply_multi" if args.profile_apply_multi else "schur_multi")
    print(json.dumps({"profile": kind, "prec": which,
                      "dims": list(dims), "steps": args.steps}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--ref-seconds", type=float, default=12.0)
    ap.add_argument("--skip-solves", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-force", action="store_true")
    ap.add_argument("--skip-large", action="store_true")
    ap.add_argument("--solves", default="",
                    help="comma-separated subset of the solve comparison (default: all)")
    ap.add_argument("--apply-shape", type=int, default=-1,
                    help="pin launch shape #N (0..21) of the timed applies instead of autotuning it")
    ap.add_argument("--large-solve", type=int, default=0,
                    help="also run the even-odd reliable-update solve of the 32^3x64 system (max steps)")
    ap.add_argument("--profile-apply", choices=["f32", "f16", "f64"], default=None,
                    help="run only --steps M applies of this precision on --profile-dims (for ncu captures)")
    ap.add_argument("--profile-ras", choices=["f32", "f16"], default=None,
                    help="run only --steps RAS applications on --profile-dims (for ncu captures)")
    ap.add_argument("--profile-schur-multi", choices=["f32", "f16"], default=None,
                    help="run only --steps multi-RHS Schur applications (12 fields) on --profile-dims")
    ap.add_argument("--profile-apply-multi", choices=["f32"], default=None,
                    help="run only --steps multi-RHS M applications (12 fields) on --profile-dims")
    ap.add_argument("--profile-ras-schur", choices=["f32", "f16"], default=None,
                    help="run only --steps block-Schur RAS applications on --profile-dims")
    ap.add_argument("--profile-dims", default="24,24,24,32")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if (args.profile_apply or args.profile_ras or args.profile_schur_multi or args.profile_ras_schur or
            args.profile_apply_multi):
        profile_run(args)
        return
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
