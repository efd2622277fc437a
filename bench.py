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


def _gen_links(args):
    dims, eps, seed = args
    from paper_1112_5280_gb300 import synth
    return synth.random_links(dims, eps, seed=seed)


def _gen_spinor(args):
    dims, seed = args
    from paper_1112_5280_gb300 import synth
    return synth.gaussian_spinor(dims, seed=seed)


# solver workloads
SOLVE_DIMS = (32, 32, 32, 64)    # kappa 0.155, eps 0.8: mixed FP16 CG vs plain FP64 CG
SOLVE_KAPPA, SOLVE_EPS = 0.155, 0.8
SOLVE_MU = 0.01                   # twisted mass of the tm_* solve variants
MRHS_DIMS = (24, 24, 24, 48)     # 12 point sources, kappa 0.15
MRHS_KAPPA = 0.15
MLAT_SIZES = ((8, 8, 8, 8), (12, 12, 12, 24), (16, 16, 16, 32))  # 64 uneven lattices
MLAT_N = 64
SERVE_POOL = 2                   # resident gauge fields / sources per serving lattice size
HB_DIMS, HB_BETA = (32, 32, 32, 64), 6.0  # pure-gauge SU(3) heatbath
HB_FLOPS_PER_LINK = 3500         # FP64 flops of one link update (staple 2484, U W 198, 3 subgroups ~810)
FP64_PEAK_TFLOPS = 152 * 2.07e9 * 2 * 2 / 1e12  # SMs x max clock x FP64 FMA/clk/SM x 2 (1.26)


def generate_inputs(full: bool):
    """All seeded inputs, generated in one spawn pool before any GPU call."""
    from paper_1112_5280_gb300 import serve, synth
    ctx = mp.get_context("spawn")
    workers = max(1, (os.cpu_count() or 2) - 1)
    jobs = {}
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
        jobs["sets"] = [ex.submit(_gen_set, k) for k in range(NSETS)]
        if full:
            jobs["solve_U"] = ex.submit(_gen_links, (SOLVE_DIMS, SOLVE_EPS, synth.SEED_LINKS))
            jobs["solve_b"] = ex.submit(_gen_spinor, (SOLVE_DIMS, synth.SEED_SOURCE))
            jobs["mrhs_U"] = ex.submit(_gen_links, (MRHS_DIMS, 0.5, synth.SEED_LINKS))
            rng = np.random.default_rng(synth.SEED_ARRIVALS + 1)
            sizes = [MLAT_SIZES[i] for i in rng.integers(0, len(MLAT_SIZES), MLAT_N)]
            kappas = rng.uniform(0.12, 0.155, MLAT_N)
            jobs["mlat"] = [(sizes[i], float(kappas[i]),
                             ex.submit(_gen_links, (sizes[i], 0.5, synth.SEED_LINKS + 100 + i)),
                             ex.submit(_gen_spinor, (sizes[i], synth.SEED_SOURCE + 100 + i)))
                            for i in range(MLAT_N)]
            jobs["serve"] = [([ex.submit(_gen_links, (d, 0.5, synth.SEED_LINKS + 200 + 10 * li + k))
                               for k in range(SERVE_POOL)],
                              [ex.submit(_gen_spinor, (d, synth.SEED_SOURCE + 200 + 10 * li + k))
                               for k in range(SERVE_POOL)])
                             for li, d in enumerate(serve.LATTICES)]
        out = {"sets": [f.result() for f in jobs["sets"]]}
        if full:
            out["solve"] = (jobs["solve_U"].result(), jobs["solve_b"].result())
            out["mrhs_U"] = jobs["mrhs_U"].result()
            out["mlat"] = [(d, k, fu.result(), fb.result()) for d, k, fu, fb in jobs["mlat"]]
            out["serve"] = ([[f.result() for f in gp] for gp, _ in jobs["serve"]],
                            [[f.result() for f in sp] for _, sp in jobs["serve"]])
    return out


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

TUNE = True  # autotune launch shapes before timing (off with --no-autotune)


def run_ours(args, world, rank, local):
    global TUNE
    TUNE = not args.no_autotune
    inputs = generate_inputs(full=not args.dslash_only)
    sets = inputs["sets"]
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

    tuned = {}

    def timed(prec, steps, warmup, batched=True):
        """One step = 100 applications captured once as a CUDA graph, replayed `steps` times."""
        gs, fi, fo = make(prec)
        if not args.no_autotune:  # launch shape of this precision and slot count, measured
            tuned[f"{prec}_x{NSETS if batched else 1}"] = lqcd.autotune_dslash(
                gs if batched else gs[:1], prec)
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
    msdf, _, _ = timed("df64", steps64, args.warmup)
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
                   "autotune": tuned or "off",
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
            "dslash_df64_GBps": b64 * apps64 / (msdf * 1e-3) / 1e9,
            "dslash_df64_us_per_application": msdf * 1e3 / apps64,
            "dslash_f64_gflops": flops_site * Vh * apps64 / (ms64 * 1e-3) / 1e9,
            "one_application_per_launch": single,
        },
    }
    if not args.dslash_only:
        line["solve"] = run_solve_section(ctx, lqcd, inputs, world)
        line["dslash32"] = run_dslash32_section(ctx, lqcd, world, U=inputs["solve"][0])
        line["multi_rhs"] = run_mrhs_section(ctx, lqcd, inputs, world)
        line["multi_lattice"] = run_mlat_section(ctx, lqcd, inputs, world)
        line["serve"] = run_serve_section(ctx, lqcd, inputs, world, rank)
        line["heatbath"] = run_heatbath_section(ctx, lqcd, world)
        line["hmc"] = run_hmc_section(ctx, lqcd, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_oracle()
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    return 0


def _lat_stats(ms_list):
    a = np.asarray(ms_list, dtype=np.float64)
    return {"n": int(a.size), "solves_per_s": float(1e3 / a.mean()), "p50_ms": float(np.percentile(a, 50)),
            "p99_ms": float(np.percentile(a, 99)), "mean_ms": float(a.mean())}


def run_solve_section(ctx, lqcd, inputs, world):
    """32^3x64, kappa 0.155, eps 0.8: mixed precision vs plain FP64 CG, each to 1e-10."""
    import torch
    U, b = inputs["solve"]
    g = ctx.gauge(SOLVE_DIMS, U, prec="f64")
    src = ctx.field(SOLVE_DIMS, "f64", lqcd.FULL, data=b)
    x = ctx.field(SOLVE_DIMS, "f64", lqcd.FULL)
    out = {"workload": "32^3x64 kappa=0.155 eps=0.8, Gaussian source, tol 1e-10 (full-M FP64 residual); "
                       f"tm_*: twisted mass mu={SOLVE_MU}"}
    if TUNE:
        out["autotune"] = {f"{p_}_{c_}": lqcd.autotune_dslash([g], p_, c_)
                           for p_, c_ in (("f16", 12), ("bf16", 12), ("f32", 12), ("f64", 18), ("df64", 18))}
    variants = [
        ("cg_mixed_f16_12", dict(sloppy_prec="f16", sloppy_compress=12), 6),
        ("cg_mixed_f16_12_truef64", dict(sloppy_prec="f16", sloppy_compress=12, true_prec="f64"), 3),
        ("cg_mixed_bf16_12", dict(sloppy_prec="bf16", sloppy_compress=12), 3),
        ("cg_mixed_f32_12", dict(sloppy_prec="f32", sloppy_compress=12), 3),
        ("bicgstab_mixed_f32_12", dict(sloppy_prec="f32", sloppy_compress=12, solver=lqcd.BICGSTAB), 6),
        ("cg_fp64", dict(sloppy_prec="f64"), 3),
        ("cg_df64", dict(sloppy_prec="df64"), 3),
        ("bicgstab_fp64", dict(sloppy_prec="f64", solver=lqcd.BICGSTAB), 2),
        # N_f = 2 twisted mass, one flavour (mu = 0.01): the same launches with A, A^-1 fused
        ("tm_cg_mixed_f16_12", dict(sloppy_prec="f16", sloppy_compress=12, mu=SOLVE_MU), 3),
        ("tm_bicgstab_mixed_f32_12", dict(sloppy_prec="f32", sloppy_compress=12, solver=lqcd.BICGSTAB,
                                          mu=SOLVE_MU), 3),
    ]
    for name, kw, reps in variants:
        o = lqcd.solve_opts(**kw)
        lqcd.solve_fields(g, src, SOLVE_KAPPA, 1e-10, x, o)  # warm-up (graph capture, link copies)
        ms, infos = [], []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = lqcd.solve_fields(g, src, SOLVE_KAPPA, 1e-10, x, o)
            ms.append((time.perf_counter() - t0) * 1e3)
            infos.append(info)
        st = _lat_stats(ms)
        st.update(ms_each=[round(v, 2) for v in ms], iters=infos[-1]["iters"],
                  reliable_updates=infos[-1]["reliable_updates"],
                  true_resid=max(i["true_resid"] for i in infos),
                  converged=all(i["status"] == 0 for i in infos))
        out[name] = st
    base = out["cg_fp64"]["solves_per_s"]
    for name in list(out):
        if isinstance(out[name], dict) and "solves_per_s" in out[name]:
            out[name]["speedup_vs_cg_fp64"] = out[name]["solves_per_s"] / base
    for o_ in (g, src, x):
        o_.close()
    return out


def run_mrhs_section(ctx, lqcd, inputs, world):
    """24^3x48, kappa 0.15: 12 point sources (spin x colour) solved together vs one by one."""
    import torch
    from paper_1112_5280_gb300 import synth
    U = inputs["mrhs_U"]
    d = MRHS_DIMS
    g = ctx.gauge(d, U, prec="f64")
    site = synth.point_site(d)
    srcs = [ctx.field(d, "f64", lqcd.FULL, data=synth.point_source(d, site, s_, c_))
            for s_ in range(4) for c_ in range(3)]
    xs = [ctx.field(d, "f64", lqcd.FULL) for _ in srcs]
    o = lqcd.solve_opts(sloppy_prec="f32", sloppy_compress=12)
    tuned = {}
    if TUNE:  # the 12-slot sloppy launch and the FP64-class update launch
        tuned = {"f32_12_x12": lqcd.autotune_dslash([g] * 12, "f32", 12),
                 "df64_18_x12": lqcd.autotune_dslash([g] * 12, "df64", 18)}
    lqcd.solve_multi(g, srcs, MRHS_KAPPA, 1e-10, xs, o)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    infos = lqcd.solve_multi(g, srcs, MRHS_KAPPA, 1e-10, xs, o)
    t_multi = time.perf_counter() - t0
    t0 = time.perf_counter()
    for s_, x_ in zip(srcs, xs):
        lqcd.solve_fields(g, s_, MRHS_KAPPA, 1e-10, x_, o)
    t_seq = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    corr = lqcd.meson_correlator(xs, list(range(10)))
    t_corr = time.perf_counter() - t0
    res = {"workload": "24^3x48 kappa=0.15, 12 point sources at a seeded site, FP32 inner / FP64 outer",
           "meson_correlator_ms": t_corr * 1e3,
           "pion_correlator_t0_t1": [float(corr[1, 0].real), float(corr[1, 1].real)],
           "multi_ms": t_multi * 1e3, "sequential_ms": t_seq * 1e3,
           "solves_per_s": 12 / t_multi, "speedup_vs_sequential": t_seq / t_multi,
           "max_true_resid": max(i["true_resid"] for i in infos),
           "converged": all(i["status"] == 0 for i in infos),
           "iters": [i["iters"] for i in infos], "autotune": tuned or "off"}
    for o_ in [g] + srcs + xs:
        o_.close()
    return res


def run_mlat_section(ctx, lqcd, inputs, world):
    """64 uneven lattices (8^4, 12^3x24, 16^3x32), own links and kappa, in one engine."""
    import torch
    items = inputs["mlat"]
    o = lqcd.solve_opts(sloppy_prec="f32", sloppy_compress=12)
    gs = [ctx.gauge(d, U, prec="f64") for d, _, U, _ in items]
    srcs = [ctx.field(d, "f64", lqcd.FULL, data=b) for d, _, _, b in items]
    xs = {d: ctx.field(d, "f64", lqcd.FULL) for d in MLAT_SIZES}
    tuned = {}
    if TUNE:  # all 64 slots in one launch: the sloppy and the FP64-class operator
        tuned = {"f32_12_x64": lqcd.autotune_dslash(gs, "f32", 12),
                 "df64_18_x64": lqcd.autotune_dslash(gs, "df64", 18)}

    def batched():
        eng = lqcd.Engine(ctx, o, max_slots=MLAT_N)
        ids = [eng.submit(g_, s_, k, 1e-10) for g_, s_, (_, k, _, _) in zip(gs, srcs, items)]
        while eng.step() > 0:
            pass
        infos = [eng.result(i, xs[d]) for i, (d, _, _, _) in zip(ids, items)]
        eng.close()
        return infos

    batched()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    infos = batched()
    t_b = time.perf_counter() - t0
    t0 = time.perf_counter()
    for g_, s_, (d, k, _, _) in zip(gs, srcs, items):
        lqcd.solve_fields(g_, s_, k, 1e-10, xs[d], o)
    t_s = time.perf_counter() - t0
    sites = sum(int(np.prod(d)) for d, _, _, _ in items)
    res = {"workload": f"{MLAT_N} lattices from 8^4 / 12^3x24 / 16^3x32, kappa U[0.12,0.155], eps 0.5, "
                       "FP32 inner / FP64 outer, one engine (all slots in every launch, CUDA-graph chunks)",
           "total_sites": sites, "batched_ms": t_b * 1e3, "sequential_ms": t_s * 1e3,
           "solves_per_s": MLAT_N / t_b, "speedup_vs_sequential": t_s / t_b,
           "max_true_resid": max(i["true_resid"] for i in infos),
           "converged": all(i["status"] == 0 for i in infos), "autotune": tuned or "off"}
    for o_ in gs + srcs + list(xs.values()):
        o_.close()
    return res


def run_heatbath_section(ctx, lqcd, world):
    """SU(3) heatbath sweeps at 32^3x64, beta 6.0, from a cold start (unit links): link
    updates/s, FP64 ALU roofline, plaquette."""
    import torch
    from paper_1112_5280_gb300 import synth
    g = ctx.gauge(HB_DIMS, synth.unit_links(HB_DIMS), prec="f64")
    g.heatbath(HB_BETA, nsweeps=3, seed=synth.SEED_LINKS)  # warm-up sweeps (part of thermalisation)
    n = 10
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    fails = g.heatbath(HB_BETA, nsweeps=n, seed=synth.SEED_LINKS, sweep0=3)
    dt = max_over_ranks(time.perf_counter() - t0, world)
    links = 4 * synth.volume(HB_DIMS)
    rate = links * n / dt
    achieved = rate * HB_FLOPS_PER_LINK / 1e12
    res = {"workload": f"{'x'.join(map(str, HB_DIMS))} Wilson gauge action beta={HB_BETA}, cold start, "
                       "Cabibbo-Marinari + Creutz, reunitarised every sweep",
           "sweeps": n, "ms_per_sweep": dt / n * 1e3, "link_updates_per_s": rate * world,
           "plaquette_after": g.plaquette(), "attempt_limit_hits": fails,
           "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": achieved / FP64_PEAK_TFLOPS,
                        "peak_kind": "derived FP64: 152 SMs x 2.07 GHz x 2 FMA/clk/SM x 2 flop",
                        "flops_per_link_update": HB_FLOPS_PER_LINK}}
    g.close()
    return res


HMC_DIMS, HMC_BETA, HMC_KAPPA, HMC_MU = (16, 16, 16, 32), 5.6, 0.14, 0.01


def run_dslash32_section(ctx, lqcd, world, U=None):
    """The solvers' sloppy operator at 32^3x64: one even-odd Dslash application per launch
    (FP16 and FP32 spinors, 12-real links), 200 launches replayed from a CUDA graph."""
    import torch
    from paper_1112_5280_gb300 import synth
    d = SOLVE_DIMS
    if U is None:
        U = synth.random_links(d, SOLVE_EPS, seed=synth.SEED_LINKS)
    Vh = synth.volume(d) // 2
    psi = synth.gaussian_spinor(d, seed=synth.SEED_SOURCE)
    out = {"workload": "32^3x64 even-odd Dslash, 12- and 18-real links, one application per launch"}
    peak, _ = measured_peaks()
    for prec, nb, nr in (("f16", 2, 12), ("f32", 4, 12), ("f16", 2, 18), ("f32", 4, 18)):
        g = ctx.gauge(d, U, prec=prec, compress=nr)
        fi = ctx.field(d, prec, lqcd.ODD, data=psi)
        fo = ctx.field(d, prec, lqcd.EVEN)
        lqcd.dslash_eo(g, fi, fo, 0)
        ctx.sync()
        st = ctx._stream  # the context's launch stream (a torch stream)
        graph = torch.cuda.CUDAGraph()
        n = 200
        with torch.cuda.graph(graph, stream=st):
            for _ in range(n):
                lqcd.dslash_eo(g, fi, fo, 0)
        for _ in range(3):
            graph.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            e0.record(st)
            graph.replay()
            e1.record(st)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / n
        gbs = algorithmic_bytes_per_site(nb, nr) * Vh / (us * 1e-6) / 1e9
        out[prec if nr == 12 else f"{prec}_18"] = {
            "us_per_application": us, "GBps": gbs, "frac_of_measured_hbm": gbs / peak,
            "bytes_per_site": algorithmic_bytes_per_site(nb, nr)}
        del graph
        for o_ in (g, fi, fo):
            o_.close()
    return out


def run_hmc_section(ctx, lqcd, world):
    """One N_f = 2 twisted-mass HMC trajectory (2MN, tau 1, 8 outer x 4 gauge steps, force
    solves to 1e-10 with FP16-12 sloppy CG) at 16^3x32 on links thermalised by 20 heatbath
    sweeps at beta 5.6."""
    import torch
    from paper_1112_5280_gb300 import synth
    d = HMC_DIMS
    g = ctx.gauge(d, synth.unit_links(d))
    g.heatbath(HMC_BETA, nsweeps=20, seed=synth.SEED_LINKS)
    ev = (synth.parity_of_sites(d) == 0)[:, None, None]
    eta = ctx.field(d, "f64", lqcd.FULL)
    phi = ctx.field(d, "f64", lqcd.FULL)

    def refresh(k):
        """Momentum and pseudofermion heatbath of trajectory k: phi = Mhat^dag eta at the current links."""
        eta.upload(synth.gaussian_spinor(d, seed=synth.SEED_SOURCE + 10 + k) * ev)
        lqcd.apply_Mhat(g, HMC_KAPPA, eta, phi, dagger=True, mu=HMC_MU)
        m.upload(synth.gaussian_momenta(d, seed=synth.SEED_SOURCE + 20 + k))

    m = ctx.mom(d)
    p = lqcd.hmc_params(beta=HMC_BETA, kappa=HMC_KAPPA, mu=HMC_MU, tau=1.0, nsteps=8, ngauge=4,
                        scheme=lqcd.TWO_MN, tol=1e-10)
    opts = lqcd.solve_opts(sloppy_prec="f16", sloppy_compress=12)
    warm = []
    for k in range(2):  # towards the dynamical ensemble (accepted unconditionally)
        refresh(k)
        warm.append(lqcd.hmc_trajectory(g, p, m, phi, opts)["dH"])
    refresh(2)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    info = lqcd.hmc_trajectory(g, p, m, phi, opts)
    dt = max_over_ranks(time.perf_counter() - t0, world)
    res = {"workload": f"{'x'.join(map(str, d))} N_f=2 twisted mass kappa={HMC_KAPPA} mu={HMC_MU}, "
                       f"beta={HMC_BETA} (links: 20 heatbath sweeps, then 2 HMC trajectories), 2MN tau=1 8x4 steps, "
                       "force solves 1e-10 (FP16-12 sloppy CG, double-float updates)",
           "ms_per_trajectory": dt * 1e3, "trajectories_per_s": world / dt,
           "dH": info["dH"], "dH_warmup": warm, "force_evals": info["force_evals"],
           "solver_iters": info["solver_iters"],
           "plaquette": info["plaquette"], "fermion_action_start": info["fermion0"]}
    for o_ in (g, m, eta, phi):
        o_.close()
    return res


def run_serve_section(ctx, lqcd, inputs, world, rank):
    """Poisson stream over {8^4, 16^3x32, 24^3x48, 32^3x64} (0.4/0.3/0.2/0.1), resident gauge
    fields, admission by HBM budget, continuous batching; closed-loop capacity, then open loop
    at 0.5x and 0.9x of it."""
    from paper_1112_5280_gb300 import serve, synth
    gpools, spools = inputs["serve"]
    opts = lqcd.solve_opts(sloppy_prec="f16", sloppy_compress=12, chunk=16)
    budget = 64 << 30
    srv = serve.GpuServer(ctx, serve.LATTICES, gpools, spools, opts=opts, hbm_budget=budget,
                          max_slots=64)
    n = 120
    mk = lambda rate, seed: serve.shard(serve.poisson_stream(
        n, rate, seed=seed, gauge_pool=SERVE_POOL, source_pool=SERVE_POOL), rank, world)  # noqa: E731
    warm = serve.poisson_stream(8, 0, seed=1, gauge_pool=SERVE_POOL, source_pool=SERVE_POOL)
    srv.scheduler().run(warm, realtime=False)
    res, wall = srv.scheduler().run(mk(0, synth.SEED_ARRIVALS), realtime=False)
    cap = serve.summarize(res, wall)
    out = {"workload": "Poisson stream, lattices 8^4/16^3x32/24^3x48/32^3x64 weights 0.4/0.3/0.2/0.1, "
                       "kappa U[0.12,0.155], tol 1e-10, FP16-12 sloppy CG + FP64 reliable updates, "
                       f"budget {budget >> 30} GiB, up to 64 concurrent requests",
           "closed_loop": cap}
    for frac in (0.5, 0.9):
        rate = frac * cap["solves_per_s"] * world
        sch = srv.scheduler()
        res, wall = sch.run(mk(rate, synth.SEED_ARRIVALS), realtime=True)
        s_ = serve.summarize(res, wall)
        s_["rate_per_s"] = rate
        s_["max_concurrent"] = sch.max_active
        out[f"open_loop_{frac}"] = s_
    srv.close()
    return out


def run_e2e(ctx, lqcd, sets, args, world):
    import torch
    from paper_1112_5280_gb300 import synth
    U, psi = sets[0]
    g = ctx.gauge(DIMS, U, prec="f32", compress=18, t_bc=-1)
    # full-lattice fields: the host arrays of a user's call; D_eo reads the odd half of fi
    # and writes the even half of fo
    fi = ctx.field(DIMS, "f32", lqcd.FULL)
    fo = ctx.field(DIMS, "f32", lqcd.FULL)
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
    ap.add_argument("--no-autotune", action="store_true", help="default launch shapes (no autotuner)")
    ap.add_argument("--no-variants", action="store_true", help="skip the one-application-per-launch timings")
    ap.add_argument("--dslash-only", action="store_true", help="skip the solver, multi-RHS, multi-lattice and serving sections")
    ap.add_argument("--section", choices=["heatbath", "hmc", "dslash32", "solve", "mrhs"],
                    help="run one section alone and print its JSON (profiling); no contract line")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.section:
        return run_one_section(args, world, rank, local)
    return run_ours(args, world, rank, local)


def run_one_section(args, world, rank, local):
    import torch
    from paper_1112_5280_gb300 import lqcd
    dev = local if world > 1 else 0
    torch.cuda.set_device(dev)
    ctx = lqcd.Context(dev, torch.cuda.Stream(device=dev))
    if args.section == "solve":
        from paper_1112_5280_gb300 import synth
        inputs = {"solve": (synth.random_links(SOLVE_DIMS, SOLVE_EPS, seed=synth.SEED_LINKS),
                            synth.gaussian_spinor(SOLVE_DIMS, seed=synth.SEED_SOURCE))}
        res = run_solve_section(ctx, lqcd, inputs, world)
    elif args.section == "mrhs":
        from paper_1112_5280_gb300 import synth
        inputs = {"mrhs_U": synth.random_links(MRHS_DIMS, EPS, seed=synth.SEED_LINKS)}
        res = run_mrhs_section(ctx, lqcd, inputs, world)
    else:
        fn = {"heatbath": run_heatbath_section, "hmc": run_hmc_section,
              "dslash32": run_dslash32_section}[args.section]
        res = fn(ctx, lqcd, world)
    if rank == 0:
        print(json.dumps({"section": args.section, **res}))
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
