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
BYTES_PER_SITE = {"f32": 96 + 96 + 192 + 288, "f16": 52 + 52 + 96 + 144, "f64": 1344}
CFG = 2  # the 24^3x32 FP32 workload
METRIC = "Wilson-Clover apply GFlop/s & % HBM roofline; mixed vs FP64 solve time to 1e-10"

# DRAM bytes per launch of the timed kernel from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum), valid only while the kernel source is unchanged.
NCU_TRAFFIC = {
    "sources_sha": None,
    "bytes_per_launch": None,
}


def kernel_sources_sha() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1612_06556_gb300", "csrc")
    for f in ("wc_dslash.cu", "wc_stencil.cuh", "wc_internal.cuh"):
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
        if world == 1:
            return x
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

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
        # complex128 in (pinned) -> import -> apply -> export -> host
        host_in = torch.from_numpy(src).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        fin, fout = lat.field(wc.F32), lat.field(wc.F32)
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
        e2e_ms = max_over_ranks(1000 * (time.perf_counter() - t0) / args.e2e_steps)
        solve = solve_comparison(wc, lat, src, args) if not args.skip_solves else None
    clk = clocks.summary()

    per_launch_ms = ms / args.steps
    flops = FLOPS_PER_SITE * V
    gflops_rank = flops / (per_launch_ms * 1e-3) / 1e9
    value = gflops_rank * world
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
                   "parallelism": f"replicas{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "k_apply<P32, M>",
                     "peak_kind": peak_kind, "algorithmic_bytes_per_launch": bytes_alg},
        "e2e": {"value": flops * world / (e2e_ms * 1e-3) / 1e9, "unit": "GFlop/s",
                "h2d_bytes_per_step": V * 12 * 16, "d2h_bytes_per_step": V * 12 * 16,
                "ms_per_step": e2e_ms},
        "gpu_launches": args.steps,
        "clocks": clk,
    }
    if solve is not None:
        line["solve"] = solve
    if world == 1 and not args.skip_cpu:
        smp = OracleSampler(dims, U, src, csw, kappa, tbc, args.ref_seconds)
        g, dt = smp.step()
        line["cpu_baseline"] = {"value": g, "unit": "GFlop/s", "cores": smp.cores, "kind": "oracle",
                                "sample": smp.describe(dt)}
    print(json.dumps(line), flush=True)


def solve_comparison(wc, lat, src, args):
    """Mixed-precision RAS-BiCGStab (FP32 and FP16 inner) vs plain FP64
    BiCGStab, both to 1e-10 from x0 = 0, on the same GPU and lattice."""
    b = lat.field(wc.F64).load(src)
    out = {}
    for name, kw in (("mixed_ras_f32", dict(precond=wc.PRECOND_RAS, inner_prec=wc.F32)),
                     ("mixed_ras_f16", dict(precond=wc.PRECOND_RAS, inner_prec=wc.F16)),
                     ("fp64_plain", dict(precond=wc.PRECOND_NONE))):
        x = lat.field(wc.F64)
        lat.solve(x, b, tol=1e-10, max_iter=20000, check=False, **kw)   # warm-up (allocations)
        x.close()
        x = lat.field(wc.F64)
        info = lat.solve(x, b, tol=1e-10, max_iter=20000, check=False, **kw)
        out[name] = {"seconds": info.seconds, "iters": info.iters, "true_rel_resid": info.true_rel_resid,
                     "status": wc.STATUS.get(info.status, info.status)}
        x.close()
    out["speedup_mixed_f32_vs_fp64"] = out["fp64_plain"]["seconds"] / out["mixed_ras_f32"]["seconds"]
    out["ras"] = "4^4 blocks, overlap 1, 4 MR iterations"
    return out


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
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
