"""Benchmark: even-odd Wilson Dslash GB/s on GB300 (16^3 x 32 workload), plus solver numbers.

python bench.py [--gpus N --steps K --warmup W] [--impl reference]

One step = 100 applications of the even-odd Dslash D_eo (FP32 spinors and
18-real FP32 links, SoA) on a 16^3 x 32 lattice over 10 independent (links,
spinor) sets (~630 MB > 129 MB L2), issued as 10 batched launches of the 10
sets each (lqcd_dslash_batch), so that every application streams from HBM. value = algorithmic bytes (each input read once, output written once:
(8*18 + 48) reals = 768 B per output site) / device time. Under torchrun each
rank runs its own copy of the workload (independent lattices, no collective):
weak scaling, value summed over ranks and divided by the slowest rank's time.

--impl reference times the FP64 CPU oracle (the correctness reference, run as
it stands) on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import multiprocessing as mp
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (16, 16, 16, 32)
KAPPA = 0.15
EPS = 0.5
NSETS = 10
APPS_PER_STEP = 100
METRIC = "Dslash GB/s vs HBM peak; solves/s and p99 latency at 1e-10 resid vs FP64 CG"
WORKLOAD = "16^3x32 even-odd Wilson Dslash, FP32 SoA spinors + 18-real FP32 links, 100 applications/step (10 batched launches x 10 field sets)"


def algorithmic_bytes_per_site(prec_bytes: int, link_reals: int) -> int:
    """Each input read once, output written once: 8 links + in spinor + out spinor."""
    return (8 * link_reals + 24 + 24) * prec_bytes


def _gen_set(k):
    from paper_1112_5280_gb300 import synth
    U = synth.random_links(DIMS, EPS, seed=synth.SEED_LINKS + k)
    psi = synth.gaussian_spinor(DIMS, seed=synth.SEED_SOURCE + k)
    return U, psi


def generate_sets(n):
    """Seeded inputs, generated in a spawn pool before any GPU call."""
    ctx = mp.get_context("spawn")
    workers = min(n, max(1, (os.cpu_count() or 2) // 2))
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
        return list(ex.map(_gen_set, range(n)))


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.t:
            self.t.join(timeout=2)

    def summary(self, t0, t1):
        sm, smax, reasons = [], [], set()
        for ts, line in self.lines:
            if not (t0 <= ts <= t1):
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ helpers

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def profile_traffic(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        from paper_1112_5280_gb300 import build as libbuild
        ent = d.get(kernel_key)
        if ent and ent.get("source_hash") == libbuild.source_hash():
            return ent.get("dram_bytes_per_launch")
    except Exception:
        return None
    return None


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ oracle arm

def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import oracle
    from paper_1112_5280_gb300 import synth
    U = synth.random_links(DIMS, EPS, seed=synth.SEED_LINKS)
    psi = synth.gaussian_spinor(DIMS, seed=synth.SEED_SOURCE)
    cores = oracle.get_threads()
    Vh = synth.volume(DIMS) // 2
    bytes_per_app = algorithmic_bytes_per_site(8, 18) * Vh
    # one step = one oracle application (a bounded sample of the 100-application step)
    for _ in range(max(1, args.warmup)):
        oracle.hop_eo(DIMS, U, psi, 0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.hop_eo(DIMS, U, psi, 0)
    dt = time.perf_counter() - t0
    gbs = bytes_per_app * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded exp(i eps H) links, Gaussian spinors)",
        "config": {"workload": WORKLOAD, "dims": list(DIMS), "eps": EPS,
                   "note": "oracle computes the FP64 operator; bytes counted at FP64 (1536 B/site)"},
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} oracle D_eo applications at 16^3x32 (1 per step)"},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def cpu_baseline_oracle(budget_s=12.0):
    import oracle
    from paper_1112_5280_gb300 import synth
    U = synth.random_links(DIMS, EPS, seed=synth.SEED_LINKS)
    psi = synth.gaussian_spinor(DIMS, seed=synth.SEED_SOURCE)
    Vh = synth.volume(DIMS) // 2
    oracle.hop_eo(DIMS, U, psi, 0)
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        oracle.hop_eo(DIMS, U, psi, 0)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": algorithmic_bytes_per_site(8, 18) * Vh * n / dt / 1e9, "unit": "GB/s",
            "cores": oracle.get_threads(), "kind": "oracle",
            "sample": f"{n} FP64 oracle D_eo applications at 16^3x32 in {dt:.1f} s "
                      "(FP64 operator, bytes counted at 1536 B/site)"}


# ------------------------------------------------------------------ GPU arm

def run_ours(args, world, rank, local):
    sets = generate_sets(NSETS)
    import torch
    from paper_1112_5280_gb300 import lqcd, synth

    dev = local if world > 1 else 0
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    ctx = lqcd.Context(dev, stream)
    Vh = synth.volume(DIMS) // 2

    def make(prec):
        gs, fi, fo = [], [], []
        for U, psi in sets:
            gs.append(ctx.gauge(DIMS, U, prec=prec, compress=18, t_bc=-1))
            fi.append(ctx.field(DIMS, prec, lqcd.ODD, data=psi))
            fo.append(ctx.field(DIMS, prec, lqcd.EVEN))
        return gs, fi, fo

    def step_single(gs, fi, fo):
        for j in range(APPS_PER_STEP):
            k = j % NSETS
            lqcd.dslash_eo(gs[k], fi[k], fo[k], 0)

    def step_batched(batch):
        for _ in range(APPS_PER_STEP // NSETS):
            batch.apply()

    def timed(prec, steps, warmup, batched=True):
        """One step = 100 applications captured once as a CUDA graph, replayed `steps` times."""
        gs, fi, fo = make(prec)
        batch = lqcd.DslashBatch(gs, fi, fo, 0) if batched else None
        run = (lambda: step_batched(batch)) if batched else (lambda: step_single(gs, fi, fo))
        run()  # eager pass: link copies and launch configuration exist before capture
        ctx.sync()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            run()
        for _ in range(warmup):
            graph.replay()
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(steps):
                graph.replay()
            e1.record(stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        barrier(world)
        ms = e0.elapsed_time(e1)
        del graph
        if batch:
            batch.close()
        for o in gs + fi + fo:
            o.close()
        launches = steps * (APPS_PER_STEP // NSETS if batched else APPS_PER_STEP)
        return ms, launches, (t0, t1)

    sampler = ClockSampler(dev)
    sampler.start()
    time.sleep(0.3)
    ms32, launches, (t0, t1) = timed("f32", args.steps, args.warmup)
    clocks = sampler.summary(t0, t1)
    steps64 = max(3, args.steps // 8)
    ms64, _, _ = timed("f64", steps64, args.warmup)
    single = {}
    if not args.no_variants:
        for prec, nb in (("f32", 4), ("f64", 8)):
            st = max(3, args.steps // (4 if prec == "f32" else 16))
            ms, n, _ = timed(prec, st, args.warmup, batched=False)
            us = ms * 1e3 / n
            single[prec] = {"us_per_launch": us,
                            "GBps": algorithmic_bytes_per_site(nb, 18) * Vh / (us * 1e-6) / 1e9}
    sampler.stop()

    apps = args.steps * APPS_PER_STEP
    b32 = algorithmic_bytes_per_site(4, 18) * Vh
    b64 = algorithmic_bytes_per_site(8, 18) * Vh
    ms_max = max_over_ranks(ms32, world)
    gbs_rank = b32 * apps / (ms32 * 1e-3) / 1e9
    value = b32 * apps * world / (ms_max * 1e-3) / 1e9
    us_per_launch = ms32 * 1e3 / launches
    apps64 = steps64 * APPS_PER_STEP
    gbs64 = b64 * apps64 / (ms64 * 1e-3) / 1e9
    flops_site = 1320

    # end to end through the C ABI with host buffers: upload, 100 applications, download
    e2e = run_e2e(ctx, lqcd, sets, args, world)

    peak, peak_kind = measured_peaks()
    kname = f"k_dslash<F32,F32,18,nodag,LIN> x{NSETS} slots"
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic: seeded exp(i*0.5*H) SU(3) links, Gaussian spinors",
        "config": {"workload": WORKLOAD, "dims": list(DIMS), "kappa": KAPPA, "eps": EPS,
                   "l2": f"inputs larger than L2: rotating {NSETS} independent field sets (~500 MB)",
                   "bytes_per_site": algorithmic_bytes_per_site(4, 18),
                   "timing": "each step captured once as a CUDA graph and replayed; CUDA events on the launch stream",
                   "parallelism": f"replicas x{world} (independent lattices per GPU)"},
        "roofline": {"bound": "hbm", "achieved": gbs_rank, "peak": peak, "unit": "GB/s",
                     "frac": gbs_rank / peak, "peak_kind": f"{peak_kind} copy bandwidth (burst)",
                     "traffic": profile_traffic("dslash_f32_18_16x32"),
                     "kernel": kname, "us_per_launch": us_per_launch,
                     "us_per_application": ms32 * 1e3 / apps},
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": launches,
        "extra": {
            "dslash_f32_gflops": flops_site * Vh * apps / (ms32 * 1e-3) / 1e9,
            "dslash_f32_effective_GBps_conventional_1440B": 1440 * Vh * apps / (ms32 * 1e-3) / 1e9,
            "dslash_f64_GBps": gbs64, "dslash_f64_us_per_application": ms64 * 1e3 / apps64,
            "dslash_f64_gflops": flops_site * Vh * apps64 / (ms64 * 1e-3) / 1e9,
            "one_application_per_launch": single,
        },
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_oracle()
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    return 0


def run_e2e(ctx, lqcd, sets, args, world):
    import torch
    from paper_1112_5280_gb300 import synth
    U, psi = sets[0]
    g = ctx.gauge(DIMS, U, prec="f32", compress=18, t_bc=-1)
    fi = ctx.field(DIMS, "f32", lqcd.ODD)
    fo = ctx.field(DIMS, "f32", lqcd.EVEN)
    host_in = torch.from_numpy(psi).pin_memory().numpy()
    host_out = torch.zeros(psi.shape, dtype=torch.complex128).pin_memory().numpy()
    Vh = synth.volume(DIMS) // 2
    steps = max(3, args.steps // 10)
    for _ in range(2):
        fi.upload(host_in)
        for _ in range(APPS_PER_STEP):
            lqcd.dslash_eo(g, fi, fo, 0)
        fo.download(host_out)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(steps):
        fi.upload(host_in)
        for _ in range(APPS_PER_STEP):
            lqcd.dslash_eo(g, fi, fo, 0)
        fo.download(host_out)
    dt = max_over_ranks(time.perf_counter() - t0, world)
    bytes_step = algorithmic_bytes_per_site(4, 18) * Vh * APPS_PER_STEP
    for o in (g, fi, fo):
        o.close()
    return {"value": bytes_step * steps * world / dt / 1e9, "unit": "GB/s",
            "h2d_bytes_per_step": int(psi.nbytes), "d2h_bytes_per_step": int(psi.nbytes),
            "steps": steps, "note": "host FP64 spinor upload + 100 applications + download"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the one-application-per-launch timings")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
