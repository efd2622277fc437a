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
SERVE_POOL = 4                   # resident gauge fields / sources per serving lattice size
SERVE_N = 240                    # requests per serving run (after a separate warm-up stream)
HB_DIMS, HB_BETA = (32, 32, 32, 64), 6.0  # pure-gauge SU(3) heatbath


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
    """nvidia-smi clock and throttle-reason samples, each stamped with nvidia-smi's own
    timestamp (its output reaches the pipe in blocks, so the time a line is read says
    nothing about when it was taken)."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 100

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.t:
            self.t.join(timeout=2)

    @staticmethod
    def _stamp(text):
        import datetime
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.datetime.strptime(text.strip(), fmt).timestamp()
            except ValueError:
                pass
        return None

    def summary(self, t0, t1):
        """Samples stamped within [t0, t1] (time.time() seconds)."""
        sm, smax, power, reasons = [], [], [], set()
        for line in list(self.lines):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            ts = self._stamp(parts[0])
            if ts is None or not (t0 <= ts <= t1):
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "sm_mhz_min": float(min(sm)), "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": float(np.median(power))}

    def windows_min(self, windows):
        """Lowest SM clock sampled inside each (t0, t1) window, None where no sample fell."""
        return [self.summary(a, b).get("sm_mhz_min") for a, b in windows]


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


def profile_counts(key: str):
    """A per-unit count (instructions per site, ...) from an ncu capture, as committed in
    profiles/counts.json, if it was taken on the current sources of the files it names."""
    p = os.path.join(ROOT, "profiles", "counts.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        from paper_1112_5280_gb300 import build as libbuild
        ent = d.get(key)
        if ent and ent.get("source_hash") == libbuild.source_hash(tuple(ent["files"])):
            return ent.get("value")
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


def _time_oracle(fn, budget_s, min_n=1):
    fn()
    n, t0 = 0, time.perf_counter()
    while n < min_n or time.perf_counter() - t0 < budget_s:
        fn()
        n += 1
    return n, time.perf_counter() - t0


def cpu_baseline_oracle(solve_inputs=None, budget_s=12.0):
    """The FP64 oracle timed on the host cores (a reported baseline): the headline's D_eo at
    16^3x32 on all cores for about budget_s, plus the oracle at one thread, the 32^3x64
    D_eo and the 4^4 CG on M^dag M (the small workload), each bounded to a few seconds."""
    import oracle
    from paper_1112_5280_gb300 import synth
    U = synth.random_links(DIMS, EPS, seed=synth.SEED_LINKS)
    psi = synth.gaussian_spinor(DIMS, seed=synth.SEED_SOURCE)
    Vh = synth.volume(DIMS) // 2
    b64 = algorithmic_bytes_per_site(8, 18)
    cores = oracle.get_threads()
    n, dt = _time_oracle(lambda: oracle.hop_eo(DIMS, U, psi, 0), budget_s)
    out = {"value": b64 * Vh * n / dt / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
           "sample": f"{n} FP64 oracle D_eo applications at 16^3x32 in {dt:.1f} s "
                     "(FP64 operator, bytes counted at 1536 B/site)"}
    plan = {}
    oracle.set_threads(1)
    try:
        n1, dt1 = _time_oracle(lambda: oracle.hop_eo(DIMS, U, psi, 0), 3.0)
    finally:
        oracle.set_threads(cores)
    plan["deo_16x32_1thread"] = {"GBps": b64 * Vh * n1 / dt1 / 1e9, "ms_per_application": dt1 / n1 * 1e3,
                                 "gflops": 1320 * Vh * n1 / dt1 / 1e9, "threads": 1}
    plan["deo_16x32_all_cores"] = {"GBps": out["value"], "ms_per_application": dt / n * 1e3,
                                   "gflops": 1320 * Vh * n / dt / 1e9, "threads": cores}
    if solve_inputs is not None:
        U2, b2 = solve_inputs
        Vh2 = synth.volume(SOLVE_DIMS) // 2
        n2, dt2 = _time_oracle(lambda: oracle.hop_eo(SOLVE_DIMS, U2, b2, 0), 3.0)
        plan["deo_32x64_all_cores"] = {"GBps": b64 * Vh2 * n2 / dt2 / 1e9, "ms_per_application": dt2 / n2 * 1e3,
                                       "gflops": 1320 * Vh2 * n2 / dt2 / 1e9, "threads": cores}
    d0 = (4, 4, 4, 4)
    U0 = synth.random_links(d0, 0.3, seed=synth.SEED_LINKS)
    s0 = synth.gaussian_spinor(d0, seed=synth.SEED_SOURCE)
    t0 = time.perf_counter()
    _, st0, it0, r0 = oracle.solve(d0, U0, 0.12, s0, tol=1e-10, method=oracle.METHOD_CG_FULL)
    plan["solve_4x4_cg_full_MdagM"] = {"ms": (time.perf_counter() - t0) * 1e3, "iters": it0,
                                       "true_resid": r0, "converged": st0 == 0, "threads": cores}
    out["plan"] = plan
    return out


# ------------------------------------------------------------------ GPU arm

TUNE = True  # autotune launch shapes before timing (off with --no-autotune)


CLOCK_WINDOW_S = 2.0  # the sampler needs load of at least this length around a timed region


def run_ours(args, world, rank, local):
    global TUNE
    import torch
    from paper_1112_5280_gb300 import lqcd, synth
    loaded = []
    if args.load_tune:  # a saved table stands in for the tuner (same choices, no tuning launches)
        lqcd.tune_load(args.load_tune)
        args.no_autotune = True
        loaded = [e for e in lqcd.tune_entries() if e["nrhs"] == 0]
    TUNE = not args.no_autotune
    inputs = generate_inputs(full=not args.dslash_only)
    sets = inputs["sets"]

    dev = local if world > 1 else 0
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    ctx = lqcd.Context(dev, stream)
    Vh = synth.volume(DIMS) // 2
    # FMA rates of this GPU (the FP64 and double-float rooflines), measured before any
    # sampled region
    alu = {"f64_fma_tflops": ctx.alu_peak("f64"), "f32_fma_tflops": ctx.alu_peak("f32"),
           "f32x2_fma_tflops": ctx.alu_peak("f32x2")}

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
        """One step = 100 applications captured once as a CUDA graph, replayed `steps` times.
        Returns the event time of the timed replays, the launches in them and the clock
        window: the timed region, extended by further (untimed) replays of the same graph
        to CLOCK_WINDOW_S when it is shorter than the sampling period allows."""
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
        t0 = time.time()
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(steps):
                graph.replay()
            e1.record(stream)
        torch.cuda.synchronize()
        t1 = time.time()
        barrier(world)
        ms = e0.elapsed_time(e1)
        if t1 - t0 < CLOCK_WINDOW_S:
            with torch.cuda.stream(stream):
                while time.time() - t0 < CLOCK_WINDOW_S:
                    for _ in range(20):
                        graph.replay()
                    torch.cuda.synchronize()
        t2 = time.time()
        del graph
        if batch:
            batch.close()
        for o in gs + fi + fo:
            o.close()
        launches = steps * (APPS_PER_STEP // NSETS if batched else APPS_PER_STEP)
        return ms, launches, (t0, t1, t2)

    sampler = ClockSampler(dev)
    sampler.start()
    time.sleep(0.5)
    ms32, launches, (t0, t1, t2) = timed("f32", args.steps, args.warmup)
    clocks = sampler.summary(t0 - 0.05, t2 + 0.05)
    clocks["window"] = (f"timed region {t1 - t0:.3f} s" + (
        f", extended to {t2 - t0:.2f} s by replaying the same graph (untimed)" if t2 > t1 else ""))
    clocks["samples_in_timed_region"] = sampler.summary(t0 - 0.05, t1 + 0.05)["samples"]
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
    f64_tflops = flops_site * Vh * apps64 / (ms64 * 1e-3) / 1e12
    df_tflops = flops_site * Vh * apps64 / (msdf * 1e-3) / 1e12

    # end to end through the C ABI with host buffers: the headline workload (10 sets, 10-slot
    # launches) with every set's input uploaded and output downloaded in every step
    e2e = run_e2e(ctx, lqcd, sets, args, world, stream)

    peak, peak_kind = measured_peaks()
    # the timed kernel: the tuner's form for the 10-slot key (0: default register budget, 3: 8
    # CTAs per SM); its ncu traffic is keyed by form in profiles/traffic.json
    if loaded:  # the loaded table's entry for this launch size (FP32, 18 reals)
        ent = [e for e in loaded if e["prec"] == 1 and e["nr"] == 18 and
               int(np.log2(e["ntiles"])) == int(np.log2(NSETS * (Vh // 64)))]
        tuned = {f"f32_x{NSETS}": ent[0]} if ent else {}
        tuned["loaded_from"] = args.load_tune
    form32 = tuned.get(f"f32_x{NSETS}", {}).get("form", 0) if tuned else 0
    kname = (f"k_dslash<F32,F32,18,nodag,EPI_PLAIN> x{NSETS} slots, form {form32} "
             f"({'8 CTAs per SM, 128 registers' if form32 == 3 else '6 CTAs per SM'})")
    df_ops = profile_counts("dslash_df64_16x32_fp32_ops_per_site")
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
                     "traffic": profile_traffic("dslash_f32_18_16x32" + ("_form3" if form32 == 3 else "")),
                     "kernel": kname, "us_per_launch": us_per_launch,
                     "us_per_application": ms32 * 1e3 / apps},
        # the paper's precision (Section 3: FP64): bound by the FP64 pipe on this part
        "roofline_f64": {"bound": "alu", "achieved": f64_tflops, "peak": alu["f64_fma_tflops"],
                         "unit": "TFLOP/s", "frac": f64_tflops / alu["f64_fma_tflops"],
                         "peak_kind": "measured FP64 FMA rate of this GPU (lqcd_alu_peak, same run)",
                         "flops_per_site": flops_site,
                         "kernel": f"k_dslash<F64,F64,18,nodag,EPI_PLAIN> x{NSETS} slots",
                         "us_per_application": ms64 * 1e3 / apps64,
                         "hbm_frac": gbs64 / peak},
        # FP64-class storage, arithmetic in double-float on the FP32 pipes
        "roofline_df64": {"bound": "alu",
                          "achieved": None if df_ops is None else df_ops * Vh * apps64 / (msdf * 1e-3) / 1e12,
                          "peak": alu["f32_fma_tflops"] / 2, "unit": "T FP32 instructions/s",
                          "frac": None if df_ops is None else
                          df_ops * Vh * apps64 / (msdf * 1e-3) / 1e12 / (alu["f32_fma_tflops"] / 2),
                          "peak_kind": "measured FP32 FMA rate / 2 (one FP32 instruction per lane and cycle)",
                          "fp32_instructions_per_site": df_ops,
                          "kernel": f"k_dslash3<DF64,DF64,nodag,EPI_PLAIN> x{NSETS} slots",
                          "us_per_application": msdf * 1e3 / apps64,
                          "hbm_frac": b64 * apps64 / (msdf * 1e-3) / 1e9 / peak},
        "alu_peaks": alu,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": launches,
        "extra": {
            "dslash_f32_gflops": flops_site * Vh * apps / (ms32 * 1e-3) / 1e9,
            "dslash_f32_effective_GBps_conventional_1440B": 1440 * Vh * apps / (ms32 * 1e-3) / 1e9,
            "dslash_f64_GBps": gbs64, "dslash_f64_us_per_application": ms64 * 1e3 / apps64,
            "dslash_df64_GBps": b64 * apps64 / (msdf * 1e-3) / 1e9,
            "dslash_df64_us_per_application": msdf * 1e3 / apps64,
            "dslash_f64_gflops": f64_tflops * 1e3,
            "dslash_df64_gflops_double_float": df_tflops * 1e3,
            "one_application_per_launch": single,
        },
    }
    if "f32" in single:
        # per-application cost inside a launch: t(10 sets) = 10 a + X and t(1 set) = a + X
        a = (us_per_launch - single["f32"]["us_per_launch"]) / (NSETS - 1)
        line["extra"]["dslash_f32_in_launch"] = {
            "us_per_application": a, "us_per_launch_fixed": us_per_launch - NSETS * a,
            "GBps": b32 / (a * 1e-6) / 1e9, "frac_of_measured_hbm": b32 / (a * 1e-6) / 1e9 / peak,
            "note": "from the 10-set and 1-set launch timings: launch, ramp-up and tail excluded"}
    if not args.dslash_only:
        def section(name, fn):
            """run one section; its clock samples (median, lowest) go with its results"""
            t_a = time.time()
            res = fn()
            res["clocks"] = sampler.summary(t_a, time.time())
            line[name] = res

        section("solve", lambda: run_solve_section(ctx, lqcd, inputs, world))
        section("dslash32", lambda: run_dslash32_section(ctx, lqcd, world, U=inputs["solve"][0]))
        section("multi_rhs", lambda: run_mrhs_section(ctx, lqcd, inputs, world, sampler))
        section("multi_lattice", lambda: run_mlat_section(ctx, lqcd, inputs, world))
        section("serve", lambda: run_serve_section(ctx, lqcd, inputs, world, rank))
        section("heatbath", lambda: run_heatbath_section(ctx, lqcd, world, alu))
        section("hmc", lambda: run_hmc_section(ctx, lqcd, world))
    sampler.stop()
    if args.save_tune and rank == 0:
        lqcd.tune_save(args.save_tune)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_oracle(inputs.get("solve"))
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
    # the FP64-class comparator on this part is the double-float CG (FP64-class storage and
    # arithmetic on the FP32 pipes); plain FP64 CG is bound by GB300's narrow FP64 pipe
    base_df = out["cg_df64"]["solves_per_s"]
    base = out["cg_fp64"]["solves_per_s"]
    for name in list(out):
        if isinstance(out[name], dict) and "solves_per_s" in out[name]:
            out[name]["speedup_vs_cg_df64"] = out[name]["solves_per_s"] / base_df
            out[name]["speedup_vs_cg_fp64"] = out[name]["solves_per_s"] / base
    out["comparators"] = ("speedup_vs_cg_df64: against the double-float CG, the fair FP64-class "
                          "comparator on GB300; speedup_vs_cg_fp64: against plain FP64 CG (FP64 pipe bound)")
    for o_ in (g, src, x):
        o_.close()
    return out


def run_mrhs_section(ctx, lqcd, inputs, world, sampler=None):
    """24^3x48, kappa 0.15: 12 point sources (spin x colour) solved together vs one by one.
    With a running clock sampler, the lowest SM clock seen during each solve is reported."""
    import torch
    from paper_1112_5280_gb300 import synth
    U = inputs["mrhs_U"]
    d = MRHS_DIMS
    g = ctx.gauge(d, U, prec="f64")
    site = synth.point_site(d)
    srcs = [ctx.field(d, "f64", lqcd.FULL, data=synth.point_source(d, site, s_, c_))
            for s_ in range(4) for c_ in range(3)]
    xs = [ctx.field(d, "f64", lqcd.FULL) for _ in srcs]
    o = lqcd.solve_opts(sloppy_prec="f32", sloppy_compress=12)  # shared links if tuned faster
    o_shared = lqcd.solve_opts(sloppy_prec="f32", sloppy_compress=12, multi_rhs_links=1)
    tuned = {}
    if TUNE:  # the sloppy and the FP64-class update launch, 12 slots and one (the comparator)
        tuned = {"f32_12_x12": lqcd.autotune_dslash([g] * 12, "f32", 12),
                 "df64_18_x12": lqcd.autotune_dslash([g] * 12, "df64", 18),
                 "f32_12_x1": lqcd.autotune_dslash([g], "f32", 12),
                 "df64_18_x1": lqcd.autotune_dslash([g], "df64", 18)}

    st = ctx._stream
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def timed_call(fn):
        """wall and device (events on the context stream) time of one synchronous call, ms"""
        e0, e1 = ev(), ev()
        torch.cuda.synchronize()
        w0 = time.time()
        t0 = time.perf_counter()
        e0.record(st)
        out = fn()
        e1.record(st)
        e1.synchronize()
        windows.append((w0, time.time()))
        return (time.perf_counter() - t0) * 1e3, e0.elapsed_time(e1), out

    windows = []

    def together(opts):
        lqcd.solve_multi(g, srcs, MRHS_KAPPA, 1e-10, xs, opts)  # warm-up (engine, graph)
        return timed_call(lambda: lqcd.solve_multi(g, srcs, MRHS_KAPPA, 1e-10, xs, opts))

    sh_wall, sh_dev, _ = together(o_shared)
    multi_wall, multi_dev, infos = together(o)
    t_shared, t_multi = sh_wall * 1e-3, multi_wall * 1e-3
    lqcd.solve_fields(g, srcs[0], MRHS_KAPPA, 1e-10, xs[0], o)  # warm-up of the one-slot engine
    each, each_dev = [], []
    for s_, x_ in zip(srcs, xs):
        w_, d_, _ = timed_call(lambda: lqcd.solve_fields(g, s_, MRHS_KAPPA, 1e-10, x_, o))
        each.append(w_)
        each_dev.append(d_)
    t_seq = sum(each) * 1e-3
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    corr = lqcd.meson_correlator(xs, list(range(10)))
    t_corr = time.perf_counter() - t0
    res = {"workload": "24^3x48 kappa=0.15, 12 point sources at a seeded site, FP32-12 inner / FP64-class outer",
           "meson_correlator_ms": t_corr * 1e3,
           "pion_correlator_t0_t1": [float(corr[1, 0].real), float(corr[1, 1].real)],
           "multi_ms": t_multi * 1e3, "multi_shared_links_ms": t_shared * 1e3, "sequential_ms": t_seq * 1e3,
           "sequential_ms_each": [round(v, 2) for v in each],
           "sequential_device_ms_each": [round(v, 2) for v in each_dev],
           "multi_device_ms": multi_dev, "multi_shared_links_device_ms": sh_dev,
           "solves_per_s": 12 / t_multi, "speedup_vs_sequential": t_seq / t_multi,
           "shared_links_vs_default": t_multi / t_shared,
           "max_true_resid": max(i["true_resid"] for i in infos),
           "converged": all(i["status"] == 0 for i in infos),
           "iters": [i["iters"] for i in infos], "autotune": tuned or "off",
           "note": "multi: one batch with the default link sharing (the tuner's measured choice for "
                   "this key); multi_shared_links: one batch with each site block's links loaded once "
                   "for a group of sources (k_dslash_mrhs) regardless of tuning"}
    if sampler is not None:  # windows: shared, default, then the 12 single solves
        time.sleep(0.3)  # the last samples reach the pipe in blocks
        lows = sampler.windows_min(windows)
        res["sm_mhz_min_multi"] = lows[1]
        res["sm_mhz_min_multi_shared_links"] = lows[0]
        res["sm_mhz_min_sequential_each"] = lows[2:]
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
    if TUNE:  # all 64 slots in one launch, and one slot of each size (the comparator)
        tuned = {"f32_12_x64": lqcd.autotune_dslash(gs, "f32", 12),
                 "df64_18_x64": lqcd.autotune_dslash(gs, "df64", 18)}
        for d in MLAT_SIZES:
            g1 = next(g_ for g_, (d_, _, _, _) in zip(gs, items) if d_ == d)
            tag = "x".join(str(v) for v in d)
            tuned[f"f32_12_{tag}"] = lqcd.autotune_dslash([g1], "f32", 12)
            tuned[f"df64_18_{tag}"] = lqcd.autotune_dslash([g1], "df64", 18)

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


def run_heatbath_section(ctx, lqcd, world, alu=None):
    """SU(3) heatbath sweeps at 32^3x64, beta 6.0, from a cold start (unit links): link
    updates/s and the FP64 pipe's share. The update's arithmetic is partly double-float on
    the FP32 pipes and partly FP64 (Creutz's draw, the accept test); its FP64 roofline takes
    the FP64 operations one link update executes, counted by ncu on the current sources."""
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
    res = {"workload": f"{'x'.join(map(str, HB_DIMS))} Wilson gauge action beta={HB_BETA}, cold start, "
                       "Cabibbo-Marinari + Creutz, reunitarised every sweep",
           "sweeps": n, "ms_per_sweep": dt / n * 1e3, "link_updates_per_s": rate * world,
           "plaquette_after": g.plaquette(), "attempt_limit_hits": fails}
    f64_ops = profile_counts("heatbath_32x64_fp64_flop_per_link")
    if f64_ops and alu:
        ach = rate * f64_ops / 1e12
        res["roofline"] = {"bound": "alu", "achieved": ach, "peak": alu["f64_fma_tflops"],
                           "unit": "TFLOP/s", "frac": ach / alu["f64_fma_tflops"],
                           "peak_kind": "measured FP64 FMA rate of this GPU (lqcd_alu_peak, same run)",
                           "fp64_flop_per_link_update": f64_ops,
                           "note": "FP64 flop executed per link update (2 per DFMA), from an ncu capture "
                                   "of k_heatbath on the current sources; the rest runs on the FP32 pipes"}
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


HMC_NSTEPS, HMC_NGAUGE, HMC_TRAJ = 20, 4, 4
HMC_CHRONO = 2  # force solves start from the linear extrapolation of the last two solutions


def run_hmc_section(ctx, lqcd, world):
    """N_f = 2 twisted-mass HMC (2MN, tau 1, 20 outer x 4 gauge steps, force solves to 1e-10
    with FP16-12 sloppy CG) at 16^3x32 on links thermalised by 20 heatbath sweeps at beta
    5.6 and 2 HMC trajectories; then 4 timed trajectories with the Metropolis test. The step
    count keeps |dH| near or below 1 (8 steps gave dH ~ 4)."""
    import torch
    from paper_1112_5280_gb300 import synth
    d = HMC_DIMS
    g = ctx.gauge(d, synth.unit_links(d))
    g.heatbath(HMC_BETA, nsweeps=20, seed=synth.SEED_LINKS)
    ev = (synth.parity_of_sites(d) == 0)[:, None, None]
    eta = ctx.field(d, "f64", lqcd.FULL)
    phi = ctx.field(d, "f64", lqcd.FULL)
    m = ctx.mom(d)

    def refresh(k):
        """Momentum and pseudofermion heatbath of trajectory k: phi = Mhat^dag eta at the current links."""
        eta.upload(synth.gaussian_spinor(d, seed=synth.SEED_SOURCE + 10 + k) * ev)
        lqcd.apply_Mhat(g, HMC_KAPPA, eta, phi, dagger=True, mu=HMC_MU)
        m.upload(synth.gaussian_momenta(d, seed=synth.SEED_SOURCE + 20 + k))

    kw = dict(beta=HMC_BETA, kappa=HMC_KAPPA, mu=HMC_MU, tau=1.0, nsteps=HMC_NSTEPS, ngauge=HMC_NGAUGE,
              scheme=lqcd.TWO_MN, tol=1e-10, chrono=HMC_CHRONO)
    opts = lqcd.solve_opts(sloppy_prec="f16", sloppy_compress=12)
    warm = []
    for k in range(2):  # towards the dynamical ensemble (accepted unconditionally)
        refresh(k)
        warm.append(lqcd.hmc_trajectory(g, lqcd.hmc_params(**kw), m, phi, opts)["dH"])
    rng = np.random.default_rng(synth.SEED_ARRIVALS + 7)
    ms, infos = [], []
    for k in range(HMC_TRAJ):
        refresh(2 + k)
        p = lqcd.hmc_params(accept_u=float(1.0 - rng.random()), **kw)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        infos.append(lqcd.hmc_trajectory(g, p, m, phi, opts))
        ms.append(max_over_ranks(time.perf_counter() - t0, world) * 1e3)
    dH = [i["dH"] for i in infos]
    res = {"workload": f"{'x'.join(map(str, d))} N_f=2 twisted mass kappa={HMC_KAPPA} mu={HMC_MU}, "
                       f"beta={HMC_BETA} (links: 20 heatbath sweeps, then 2 HMC trajectories), 2MN tau=1 "
                       f"{HMC_NSTEPS}x{HMC_NGAUGE} steps, force solves 1e-10 (FP16-12 sloppy CG, "
                       f"double-float updates, initial guess by linear extrapolation of the last two "
                       f"solutions), {HMC_TRAJ} timed trajectories with the Metropolis test",
           "ms_per_trajectory": float(np.mean(ms)), "ms_each": [round(v, 1) for v in ms],
           "trajectories_per_s": world * 1e3 / float(np.mean(ms)),
           "dH": dH, "dH_warmup": warm, "acceptance": float(np.mean([i["accepted"] for i in infos])),
           "exp_minus_dH_mean": float(np.mean(np.exp(-np.asarray(dH)))),
           "force_evals": infos[-1]["force_evals"], "solver_iters": infos[-1]["solver_iters"],
           "plaquette": infos[-1]["plaquette"]}
    for o_ in (g, m, eta, phi):
        o_.close()
    return res


def run_serve_section(ctx, lqcd, inputs, world, rank):
    """Poisson stream over {8^4, 16^3x32, 24^3x48, 32^3x64} (0.4/0.3/0.2/0.1), 4 resident gauge
    fields and sources per size, admission by HBM budget, continuous batching; closed-loop
    capacity, then open loop at 0.5x, 0.8x and 0.9x of it, 240 requests each after a warm-up
    stream, with p50/p99 per lattice size. Near the closed-loop capacity (0.9x) the queue can
    grow over a run: a batch of fewer concurrent requests does less per launch than the full
    queue the capacity was measured with."""
    from paper_1112_5280_gb300 import serve, synth
    gpools, spools = inputs["serve"]
    opts = lqcd.solve_opts(sloppy_prec="f16", sloppy_compress=12)
    budget = 64 << 30
    srv = serve.GpuServer(ctx, serve.LATTICES, gpools, spools, opts=opts, hbm_budget=budget,
                          max_slots=64)
    n = SERVE_N
    mk = lambda rate, seed: serve.shard(serve.poisson_stream(
        n, rate, seed=seed, gauge_pool=SERVE_POOL, source_pool=SERVE_POOL), rank, world)  # noqa: E731
    warm = serve.poisson_stream(16, 0, seed=1, gauge_pool=SERVE_POOL, source_pool=SERVE_POOL)
    srv.scheduler().run(warm, realtime=False)
    res, wall = srv.scheduler().run(mk(0, synth.SEED_ARRIVALS), realtime=False)
    cap = serve.summarize(res, wall)
    out = {"workload": "Poisson stream, lattices 8^4/16^3x32/24^3x48/32^3x64 weights 0.4/0.3/0.2/0.1, "
                       f"kappa U[0.12,0.155], tol 1e-10, {SERVE_POOL} resident gauge fields and sources per "
                       "size, FP16-12 sloppy CG + FP64-class reliable updates, "
                       f"budget {budget >> 30} GiB, up to 64 concurrent requests, {n} requests per run",
           "closed_loop": cap}
    for frac in (0.5, 0.8, 0.9):
        rate = frac * cap["solves_per_s"] * world
        sch = srv.scheduler()
        res, wall = sch.run(mk(rate, synth.SEED_ARRIVALS), realtime=True)
        s_ = serve.summarize(res, wall)
        s_["rate_per_s"] = rate
        s_["max_concurrent"] = sch.max_active
        out[f"open_loop_{frac}"] = s_
    srv.close()
    return out


def run_e2e(ctx, lqcd, sets, args, world, stream):
    """The headline workload through the C ABI with host buffers: every step uploads each
    set's input spinor from pinned host memory (full-lattice FP64, the host layout), runs the
    10 batched launches of 10 applications and downloads each set's output. CUDA events on
    the context stream around the steps; the downloads synchronise the host."""
    import torch
    from paper_1112_5280_gb300 import synth
    gs = [ctx.gauge(DIMS, U, prec="f32", compress=18, t_bc=-1) for U, _ in sets]
    # full-lattice fields: the host arrays of a user's call; D_eo reads the odd half of fi
    # and writes the even half of fo
    fi = [ctx.field(DIMS, "f32", lqcd.FULL) for _ in sets]
    fo = [ctx.field(DIMS, "f32", lqcd.FULL) for _ in sets]
    host_in = [torch.from_numpy(psi).pin_memory().numpy() for _, psi in sets]
    host_out = [torch.zeros(psi.shape, dtype=torch.complex128).pin_memory().numpy() for _, psi in sets]
    batch = lqcd.DslashBatch(gs, fi, fo, 0)
    Vh = synth.volume(DIMS) // 2

    def step():
        for f, h in zip(fi, host_in):
            f.upload(h)
        for _ in range(APPS_PER_STEP // NSETS):
            batch.apply()
        for f, h in zip(fo, host_out):
            f.download(h)

    steps = max(3, args.steps // 20)
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    bytes_step = algorithmic_bytes_per_site(4, 18) * Vh * APPS_PER_STEP
    nbytes = sum(h.nbytes for h in host_in)
    batch.close()
    for o in gs + fi + fo:
        o.close()
    # the copy bound of such a step: plain pinned-host <-> device copies of the same bytes
    # (one buffer each way, CUDA events), plus the device-timed compute of the headline
    hbuf = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    dbuf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    rates = {}
    with torch.cuda.stream(stream):
        for name, dst, src in (("h2d", dbuf, hbuf), ("d2h", hbuf, dbuf)):
            dst.copy_(src, non_blocking=True)
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            for _ in range(3):
                dst.copy_(src, non_blocking=True)
            c1.record(stream)
            c1.synchronize()
            rates[name] = 3 * nbytes / (c0.elapsed_time(c1) * 1e-3) / 1e9
    del hbuf, dbuf
    copy_ms = (nbytes / rates["h2d"] + nbytes / rates["d2h"]) / 1e6
    return {"value": bytes_step * steps * world / (ms * 1e-3) / 1e9, "unit": "GB/s",
            "h2d_bytes_per_step": int(nbytes), "d2h_bytes_per_step": int(nbytes),
            "steps": steps, "ms_per_step": ms / steps, "wall_ms_per_step": wall * 1e3 / steps,
            "copy_GBps": {"h2d": rates["h2d"], "d2h": rates["d2h"]},
            "copy_ms_per_step": copy_ms,
            "note": f"headline workload: {NSETS} host FP64 spinors uploaded, {APPS_PER_STEP} "
                    f"applications in {APPS_PER_STEP // NSETS} batched launches, {NSETS} outputs "
                    "downloaded per step (CUDA events on the context stream); copy_GBps: plain "
                    "pinned copies of the same bytes, the bound of the step's transfers"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shapes (no autotuner)")
    ap.add_argument("--save-tune", metavar="PATH", help="save the autotuner's table (JSON) after the run")
    ap.add_argument("--load-tune", metavar="PATH",
                    help="launch shapes from a saved table instead of tuning (profiling the tuned launches)")
    ap.add_argument("--no-variants", action="store_true", help="skip the one-application-per-launch timings")
    ap.add_argument("--dslash-only", action="store_true", help="skip the solver, multi-RHS, multi-lattice and serving sections")
    ap.add_argument("--section", choices=["heatbath", "hmc", "dslash32", "solve", "mrhs", "cpu"],
                    help="run one section alone and print its JSON (profiling); no contract line")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.section:
        return run_one_section(args, world, rank, local)
    return run_ours(args, world, rank, local)


def run_cpu_plan():
    """The oracle's CPU baseline in full (no GPU): the bounded figures of the bench line, and
    the plain FP64 solves of the small (4^4) and the 32^3x64 kappa 0.155 workloads to 1e-10
    on all host cores, with the oracle's own even-odd CG."""
    import oracle
    from paper_1112_5280_gb300 import synth
    U = synth.random_links(SOLVE_DIMS, SOLVE_EPS, seed=synth.SEED_LINKS)
    b = synth.gaussian_spinor(SOLVE_DIMS, seed=synth.SEED_SOURCE)
    out = cpu_baseline_oracle((U, b))
    t0 = time.perf_counter()
    _, st, it, res = oracle.solve(SOLVE_DIMS, U, SOLVE_KAPPA, b, tol=1e-10, method=oracle.METHOD_CG_EO)
    dt = time.perf_counter() - t0
    out["plan"]["solve_32x64_cg_eo"] = {"ms": dt * 1e3, "solves_per_s": 1.0 / dt, "iters": it,
                                        "true_resid": res, "converged": st == 0,
                                        "threads": oracle.get_threads()}
    return out


def run_one_section(args, world, rank, local):
    global TUNE
    TUNE = not args.no_autotune
    if args.section == "cpu":
        if rank == 0:
            print(json.dumps({"section": "cpu", **run_cpu_plan()}))
        return 0
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
