#!/usr/bin/env python3
"""Benchmark: IHT iterations/s on the single-solve panel (n=5000, p=500000, k=50).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--config 1|2|3|4] [--grad-impl 0|1|2] [--no-cpu-baseline]
                    [--requests R]

One step = one full IHT least-squares solve (beta = 0 to convergence, every
step of the hot path: standardised gradient, top-k projection, step size,
backtracking, sparse residual update) on synthetic PLINK-packed genotypes
with the shapes of the paper's GWAS panels.  ``value`` = IHT iterations per
second over the K timed solves, inputs resident in HBM, device-timed with CUDA
events; ``e2e`` = the same metric through the host-buffer C-ABI call (y copied
in, beta/support copied out inside the timed region).  The packed genotype
matrix (625 MB) is larger than L2, so no flush is needed between steps.

Under torchrun (N > 1) every rank runs an independent replica of the same
solve on its own GPU (the single-solve path has no exchange step), value =
iterations of all ranks / max elapsed.

``--impl reference`` times the FP64 CPU oracle on the host cores (bounded
sample of the same workload); on rank 0 only.

``--config 3`` measures the batched cross-validation workload instead (n=6000,
p=1000000, 5 folds x k = 1..20 = 100 solves in one iht_fit_batch call):
one step = the whole batch to convergence, value = solves/s, beside the same
100 solves run one at a time through iht_fit on the same GPU.

``--config 4`` measures the serving stream (n=10000, p=1000000; requests with
a random subject subset of 2000-10000 rows, k in 5..200, fresh phenotype):
value = solves/s of the continuous-batching server with every request queued
at once (one step = R requests), beside Poisson arrivals at 0.5x and 1.2x
the one-at-a-time GPU rate with p50/p99 latency, and that one-at-a-time rate
itself (iht_fit per request, host inputs).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

FALLBACK_HBM_GBS = 6400.0

# DRAM bytes (read + write) of one single-column gradient launch on the
# n = 5000, p = 500 000 panel, from one ncu capture of this kernel version
# at the tuned stage count (dram__bytes_read.sum + dram__bytes_write.sum;
# summary in profiles/).
K1_TRAFFIC_BYTES = 646192384 + 3213568
# The same for the first multi-column launch of the cross-validation batch
# (44 residual columns of the 100 solves, the widest pass).
K2_TRAFFIC_FIRST_LAUNCH_BYTES = 1538364416 + 167354112


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# The paper's own timings (Sec. 3, Tables 1 and 2): context for the lines below,
# not a baseline -- another machine, FP64 OpenCL, no iteration counts or rates.
PAPER_CONTEXT = {
    "hardware": "1 six-core 2.67 GHz Xeon + 1 NVIDIA Tesla C2050 (Fermi, OpenCL), FP64",
    "path_time_packed_multicore_gpu_s": 65.48,
    "path_time_packed_multicore_s": 141.28,
    "path_time_float_single_core_s": 8.27,
    "path_workload": "NFBC1966 chromosome 1: 23,695 SNPs, n about 5.1k, k = 5..100 in steps of 5",
    "cv5_k1to50_with_refit_hours": {"BMI": 1.12, "HDL": 1.28, "LDL": 1.32, "TG": 1.49},
    "cv_workload": "NFBC1966 n about 4.7-5.1k, p about 333.7k, 5-fold CV over k = 1..50 and a refit",
    "note": "the paper reports no iteration counts, per-iteration times or GB/s",
}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), ws


def gather_rows(vals, world):
    """Every rank's row of per-rank figures, stacked [world, len] in rank order.

    With world > 1 this is an all-gather over the initialised process group
    (NCCL on the GPUs, gloo on the host); every rank gets the same array.
    """
    row = np.asarray(vals, dtype=np.float64)
    if world <= 1:
        return row[None, :]
    import torch
    import torch.distributed as dist
    dev = (torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl"
           else torch.device("cpu"))
    t = torch.tensor(row, device=dev)
    out = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(out, t)
    return torch.stack(out).cpu().numpy()


def weak_rate(rows, units, seconds):
    """Whole-job throughput of replicas: units summed over ranks / the slowest rank's time."""
    return float(rows[:, units].sum()) / float(rows[:, seconds].max())


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def warm_up(step, warmup: int, min_s: float = 0.5) -> int:
    """Untimed warm-up steps right before a timed region: at least `warmup` of
    them, continued until `min_s` seconds of steps have run.  The clock sampler
    starts just before, and a GPU that has idled runs its first few hundred
    milliseconds of work measurably slower (up to 8 % on the single-solve
    workload), so the timed steps start on a GPU already under load.  Returns
    the number of steps run (reported as warmup_steps_run)."""
    n, t0 = 0, time.perf_counter()
    while n < max(warmup, 0) or time.perf_counter() - t0 < min_s:
        step()
        n += 1
    return n


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                if self.uuid and self.uuid not in parts[0] and parts[0] not in self.uuid:
                    continue
                rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def gpu_uuid(torch, dev):
    try:
        u = torch.cuda.get_device_properties(dev).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        return None


def run_oracle_sample(cfg: int, max_iter: int, pn=None, bed=None, y=None):
    """FP64 oracle, as it stands, on the host cores: (iterations, seconds, threads)."""
    import oracle
    c = synth.CONFIGS[cfg]
    if pn is None:
        pn = synth.config_panel(cfg)
        bed = pn.bed()
        y, _, _ = synth.config_phenotype(cfg, pn)
    G = oracle.Geno.from_bed(bed, pn.n, pn.p)
    t0 = time.perf_counter()
    f = oracle.iht(G, y, c["k"], max_iter=max_iter, tol=c["tol"], trace=False)
    dt = time.perf_counter() - t0
    return f.iterations, dt, oracle.max_threads()


def oracle_parity(fo, beta, support, iterations, status, gtol=1e-5):
    """The GPU solve against the oracle's solve of the same problem: iterations
    the oracle certifies (the k-th and (k+1)-th |w| further apart than the FP32
    gradient error can move them, no backtracking decision within 1e-3 of its
    threshold) before its first tie-ambiguous one, the tie-ambiguous exclusion
    rate, and the final support and beta."""
    tr = fo.trace
    lead = fo.iterations
    for t in range(fo.iterations):
        if not (tr["gap"][t] > 10 * gtol * tr["wscale"][t] and not (tr["margin"][t] < 1e-3)):
            lead = t
            break
    beta = np.asarray(beta)
    rel = float(np.max(np.abs(beta - fo.beta)) / max(np.max(np.abs(fo.beta)), 1e-300))
    return {"oracle_iterations": int(fo.iterations), "certified_iterations": int(lead),
            "tie_ambiguous_exclusion_rate": 1.0 - lead / max(fo.iterations, 1),
            "same_iterations": int(iterations) == int(fo.iterations),
            "same_status": int(status) == int(fo.status),
            "support_equal": bool(np.array_equal(np.sort(np.asarray(support)), fo.support)),
            "beta_max_rel_err": rel, "beta_tolerance": 1e-4}


def reference_arm(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    cfg = args.config
    c = synth.CONFIGS[cfg]
    pn = synth.config_panel(cfg)
    bed = pn.bed()
    y, _, _ = synth.config_phenotype(cfg, pn)
    # iterations per step: the bounded sample shrinks with the step count so any
    # --steps finishes in about a minute of host time
    cap = max(1, min(args.oracle_iters, 50 // max(args.steps, 1)))
    for _ in range(args.warmup):
        run_oracle_sample(cfg, 1, pn, bed, y)         # the oracle has no warm state
    its, secs = 0, 0.0
    threads = 1
    for _ in range(args.steps):
        i, dt, threads = run_oracle_sample(cfg, cap, pn, bed, y)
        its += i
        secs += dt
    value = its / secs
    sample = (f"FP64 oracle IHT on {c['name']} capped at {cap} iterations per step "
              f"(setup + {cap} gradient passes, projections, step sizes)")
    out = {"impl": "reference", "metric": "IHT iterations/sec", "value": value, "unit": "iter/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": c["name"], "n": c["n"], "p": c["p"], "k": c["k"]},
           "cpu_baseline": {"value": value, "unit": "iter/s", "cores": threads, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": "iter/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def ours_arm(args):
    import torch
    import paper_1608_01398_b300 as iht

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local_rank}"))
    torch.cuda.set_device(local_rank)
    dev = local_rank
    cfg = args.config
    c = synth.CONFIGS[cfg]
    n, p, k = c["n"], c["p"], c["k"]

    t0 = time.perf_counter()
    pn = synth.config_panel(cfg)
    bed = pn.bed()
    y, causal, _ = synth.config_phenotype(cfg, pn, which=rank)    # replicas: own phenotype
    log(f"[bench] rank {rank}: generated {bed.nbytes / 1e6:.0f} MB panel in "
        f"{time.perf_counter() - t0:.1f}s")

    stream = torch.cuda.current_stream(dev)
    ctx = iht.Context(dev, stream)
    ds = iht.Dataset(ctx, bed, n, p)
    y_dev = torch.from_numpy(y).to(f"cuda:{dev}")
    fit_kw = dict(out_device=True, grad_impl=args.grad_impl, tol=c["tol"], max_iter=c["max_iter"])

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    clocks = ClockSampler(gpu_uuid(torch, dev))
    clocks.start()
    warm_steps = warm_up(lambda: iht.iht_fit(ds, y_dev, k, **fit_kw), args.warmup)
    torch.cuda.synchronize(dev)

    # ---- device-timed region: inputs resident in HBM -------------------------
    barrier()
    torch.cuda.synchronize(dev)
    l0 = iht.iht_kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    its, grad_ms, grad_n, replays = 0, 0.0, 0, 0
    statuses = []
    for _ in range(args.steps):
        r = iht.iht_fit(ds, y_dev, k, **fit_kw)
        its += r.iterations
        replays += r.graph_replays
        statuses.append(r.status)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    launches = iht.iht_kernel_launches() - l0
    clk = clocks.stop()
    elapsed = ev0.elapsed_time(ev1) / 1e3

    # ---- gradient-pass duration: CUDA events around every gradient launch of
    # the same solves run profiled (their iterations replay the per-iteration
    # graph with event nodes, which a conditional loop cannot hold; the pass
    # is the same kernel in the same launch shape)
    prof_steps = min(args.steps, 10)
    for _ in range(prof_steps):
        rp = iht.iht_fit(ds, y_dev, k, profile=1, **fit_kw)
        grad_ms += rp.grad_ms
        grad_n += rp.grad_launches
    torch.cuda.synchronize(dev)

    # ---- end to end through the host-buffer call ------------------------------
    y_pin = torch.empty(n, dtype=torch.float64).pin_memory()
    y_pin.numpy()[:] = y
    y_host = y_pin.numpy()
    warm_up(lambda: iht.iht_fit(ds, y_host, k, grad_impl=args.grad_impl, tol=c["tol"], max_iter=c["max_iter"]),
            args.warmup)                                     # untimed, as for the device-timed steps
    barrier()
    torch.cuda.synchronize(dev)
    w0 = time.perf_counter()
    e2e_its = 0
    for _ in range(args.steps):
        r = iht.iht_fit(ds, y_host, k, grad_impl=args.grad_impl, tol=c["tol"],
                        max_iter=c["max_iter"])
        e2e_its += r.iterations
    torch.cuda.synchronize(dev)
    e2e_wall = time.perf_counter() - w0
    barrier()
    beta_host, supp_host = r.beta, r.support

    # ---- aggregate over ranks --------------------------------------------------
    allv = gather_rows([its, elapsed, e2e_its, e2e_wall, grad_ms, grad_n], world)
    if rank == 0:
        max_el = float(allv[:, 1].max())
        value = weak_rate(allv, 0, 1)
        e2e_value = weak_rate(allv, 2, 3)
        hbm_peak, peak_kind = measured_peaks()
        alg_bytes = p * ((n + 3) // 4) + 12 * p + 4 * n      # packed genotypes + u, v, g + r
        per_launch_ms = grad_ms / max(grad_n, 1)
        achieved = alg_bytes / (per_launch_ms / 1e3) / 1e9 if grad_n else None
        iters_mean = its / args.steps
        ctl = 4 + 2 * 120 + 4 * iters_mean                   # status words and done flags
        out = {
            "metric": "IHT iterations/sec", "value": value, "unit": "iter/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "warmup_steps_run": warm_steps,
            "ms_per_step": 1e3 * max_el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "paper_context": PAPER_CONTEXT,
            "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": c["name"], "n": n, "p": p, "k": k,
                       "packed_bytes": p * ((n + 3) // 4), "iterations_per_solve": iters_mean,
                       "grad_impl": args.grad_impl, "l2": "inputs larger than L2 (no flush)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "genotype_gbs": achieved, "pct_hbm_peak": (100.0 * achieved / hbm_peak) if achieved else None,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": (achieved / hbm_peak) if achieved else None,
                         "traffic": K1_TRAFFIC_BYTES if cfg == 2 else None,
                         "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum of one ncu "
                                           "capture of this kernel version (profiles/), not this run",
                         "kernel": "gradient pass g = Z^T r", "peak_source": peak_kind,
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "kernel_timing": f"CUDA events around each of the {grad_n} gradient launches "
                                          f"of {prof_steps} profiled solves after the timed region"},
            "e2e": {"value": e2e_value, "unit": "iter/s", "h2d_bytes_per_step": 8 * n + 120,
                    "d2h_bytes_per_step": int(12 * k + ctl)},
            "gpu_launches": int(launches), "clocks": clk,
            "statuses": sorted(set(int(s) for s in statuses)),
            "graph_replays_per_step": replays / max(args.steps, 1),
            "pass_shapes": iht.tuning_summary().strip().splitlines(),
        }
        if not args.no_cpu_baseline and world == 1:
            import oracle
            G = oracle.Geno.from_bed(bed, pn.n, pn.p)
            t0 = time.perf_counter()
            fo = oracle.iht(G, y, k, tol=c["tol"], max_iter=c["max_iter"], trace=True)
            secs = time.perf_counter() - t0
            threads = oracle.max_threads()
            out["cpu_baseline"] = {
                "value": fo.iterations / secs, "unit": "iter/s", "cores": threads, "kind": "oracle",
                "sample": f"FP64 oracle IHT on {c['name']}: one full solve from beta = 0 "
                          f"({fo.iterations} iterations incl. set-up), {secs:.1f}s"}
            out["parity"] = oracle_parity(fo, beta_host, supp_host, r.iterations, r.status)
            # the same oracle on one host thread (its column-parallel loops serial)
            import oracle
            oracle.set_threads(1)
            try:
                i1, s1, _ = run_oracle_sample(cfg, 1, pn, bed, y)
            finally:
                oracle.set_threads(threads)
            out["cpu_baseline"]["single_thread"] = {
                "value": i1 / s1, "unit": "iter/s", "cores": 1,
                "sample": f"first {i1} iteration (incl. setup), {s1:.1f}s"}
        if cfg == 2 and world == 1 and not args.no_extra:
            del ds, ctx
            torch.cuda.empty_cache()
            out["batched"] = sub_run(3, ["--steps", "3", "--warmup", "1"], BATCHED_KEYS)
            out["serving"] = sub_run(4, ["--steps", "1", "--warmup", "1"], SERVING_KEYS)
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


BATCHED_KEYS = ("metric", "value", "unit", "ms_per_step", "config", "plain", "speedup_vs_plain",
                "roofline", "e2e", "model_selection", "clocks", "graph_replays_per_step")
SERVING_KEYS = ("metric", "value", "unit", "ms_per_step", "config", "plain", "speedup_vs_plain",
                "poisson", "latency_ms_all_queued", "e2e", "server", "clocks")


def sub_run(config: int, extra: list, keys) -> dict:
    """The batched (config 3) or serving (config 4) workload in a child process of
    this bench (same GPU, run after the single-solve line's timed region); its
    JSON line, reduced to the given keys."""
    cmd = [sys.executable, os.path.abspath(__file__), "--config", str(config), "--no-cpu-baseline",
           *extra]
    t0 = time.perf_counter()
    r = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT)
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    if r.returncode != 0 or not lines:
        return {"error": f"exit {r.returncode}: {r.stderr.strip().splitlines()[-1:] }"}
    d = json.loads(lines[-1])
    sub = {k: d[k] for k in keys if k in d}
    sub["command"] = " ".join(["python bench.py", "--config", str(config), "--no-cpu-baseline", *extra])
    sub["wall_s"] = time.perf_counter() - t0
    return sub


MR_PEAK_KEY = "bf16_tflops_sustained"
FP8_OVER_BF16 = 2.0                         # nominal dense ratio, 4.5 / 2.25 PFLOP/s
FALLBACK_TFLOPS = 1400.0
MR_LIMBS = 5                                # E4M3 limbs of each residual column


def measured_tensor_peak():
    """FP8 dense peak: the measured sustained BF16 GEMM rate x the nominal FP8/BF16 ratio."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return (FP8_OVER_BF16 * float(json.load(f)[MR_PEAK_KEY]),
                    "measured bf16 sustained x 2 (nominal fp8/bf16 ratio)")
    except (OSError, KeyError, ValueError):
        return FP8_OVER_BF16 * FALLBACK_TFLOPS, "fallback bf16 sustained x 2"


def cv_setup(cfg, rank=0):
    """The panel, a phenotype and the folds; replicas (rank > 0) draw their own phenotype and folds."""
    c = synth.CONFIGS[cfg]
    pn = synth.config_panel(cfg)
    bed = pn.bed()
    y, _, _ = synth.config_phenotype(cfg, pn, which=rank)
    lab = synth.cv_folds(pn.n, c["folds"], synth.BASE_SEED + 1000 * cfg + 7 + 101 * rank)
    train = [np.flatnonzero(lab != f).astype(np.int32) for f in range(c["folds"])]
    return c, pn, bed, y, train, lab


def cv_reference(args, c, pn, bed, y, train, iters_per_solve=None):
    """Oracle on a bounded sample: one solve (fold 0, largest k) capped at a few iterations."""
    import oracle
    G = oracle.Geno.from_bed(bed, pn.n, pn.p)
    cap = max(1, min(args.oracle_iters, 3))
    t0 = time.perf_counter()
    f = oracle.iht(G, y[train[0]], c["ks"][-1], rows=train[0], max_iter=cap, tol=c["tol"],
                   trace=False)
    dt = time.perf_counter() - t0
    sec_per_iter = dt / max(f.iterations, 1)
    ips = iters_per_solve if iters_per_solve else 10.0
    return {"value": 1.0 / (sec_per_iter * ips), "unit": "solves/s", "cores": oracle.max_threads(),
            "kind": "oracle",
            "sample": f"FP64 oracle, fold 0 k={c['ks'][-1]} on {c['name']}, {f.iterations} iterations "
                      f"(incl. setup) in {dt:.1f}s; solves/s extrapolated at {ips:.1f} iterations "
                      f"per solve"}


def cv_reference_arm(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    c, pn, bed, y, train, _ = cv_setup(3)
    for _ in range(args.warmup):
        pass     # the oracle has no warm state: each step is a fresh bounded sample
    vals = [cv_reference(args, c, pn, bed, y, train) for _ in range(max(args.steps, 1))]
    value = statistics.median(v["value"] for v in vals)
    cb = dict(vals[0])
    cb["value"] = value
    out = {"impl": "reference", "metric": "batched IHT solves/sec", "value": value,
           "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": c["name"], "n": c["n"], "p": c["p"], "folds": c["folds"],
                      "ks": [c["ks"][0], c["ks"][-1]]},
           "cpu_baseline": cb,
           "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def cv_arm(args):
    import torch
    import paper_1608_01398_b300 as iht

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local_rank}"))
    torch.cuda.set_device(local_rank)
    dev = local_rank
    t0 = time.perf_counter()
    c, pn, bed, y, train, lab = cv_setup(3, rank)
    n, p = c["n"], c["p"]
    log(f"[bench] rank {rank}: generated {bed.nbytes / 1e6:.0f} MB panel in "
        f"{time.perf_counter() - t0:.1f}s")
    stream = torch.cuda.current_stream(dev)
    ctx = iht.Context(dev, stream)
    ds = iht.Dataset(ctx, bed, n, p)
    cuda = f"cuda:{dev}"
    tr_dev = [torch.from_numpy(t).to(cuda) for t in train]
    y_dev = [torch.from_numpy(np.ascontiguousarray(y[t])).to(cuda) for t in train]
    probs = [(y_dev[f], k, tr_dev[f]) for f in range(c["folds"]) for k in c["ks"]]
    b = len(probs)
    kw = dict(out_device=True, dense=False, grad_impl=args.grad_impl, tol=c["tol"],
              max_iter=c["max_iter"])
    def barrier():
        if world > 1:
            torch.distributed.barrier()

    clocks = ClockSampler(gpu_uuid(torch, dev))
    clocks.start()
    warm_steps = warm_up(lambda: iht.iht_fit_batch(ds, probs, **kw), args.warmup)
    torch.cuda.synchronize(dev)
    barrier()
    torch.cuda.synchronize(dev)
    l0 = iht.iht_kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    solves, its, cols, grad_ms, grad_n, statuses, replays = 0, 0, 0, 0.0, 0, [], 0
    for _ in range(args.steps):
        res = iht.iht_fit_batch(ds, probs, profile=1, **kw)
        solves += b
        its += sum(r.iterations for r in res)
        cols += sum(max(r.iterations, 1) for r in res)
        grad_ms += res[0].grad_ms
        grad_n += res[0].grad_launches
        replays += res[0].graph_replays
        statuses += [r.status for r in res]
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    launches = iht.iht_kernel_launches() - l0
    clk = clocks.stop()
    elapsed = ev0.elapsed_time(ev1) / 1e3

    # the same solves one at a time (plain single-solve GPU path), timed once
    iht.iht_fit(ds, y_dev[0], c["ks"][0], rows=tr_dev[0], out_device=True)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plain_its = 0
    for (yy, k, rr) in probs:
        plain_its += iht.iht_fit(ds, yy, k, rows=rr, out_device=True, grad_impl=args.grad_impl,
                                 tol=c["tol"], max_iter=c["max_iter"]).iterations
    e1.record(stream)
    torch.cuda.synchronize(dev)
    plain_s = e0.elapsed_time(e1) / 1e3

    # end to end through the host-buffer call: host y and rows in, supports and beta_S out
    y_host = [np.ascontiguousarray(y[t]) for t in train]
    probs_h = [(y_host[f], k, train[f]) for f in range(c["folds"]) for k in c["ks"]]
    torch.cuda.synchronize(dev)
    w0 = time.perf_counter()
    for _ in range(args.steps):
        iht.iht_fit_batch(ds, probs_h, dense=False, grad_impl=args.grad_impl, tol=c["tol"],
                          max_iter=c["max_iter"])
    torch.cuda.synchronize(dev)
    e2e_wall = time.perf_counter() - w0

    # the whole model selection through iht_cv (Sec. 2.4): the 5 x 20 fits,
    # out-of-fold MSE on the device, k_best, the refit on all rows; host in and out
    iht.iht_cv(ds, y, lab, c["ks"], tol=c["tol"], max_iter=c["max_iter"])      # warm (tuned, graphs)
    torch.cuda.synchronize(dev)
    w0 = time.perf_counter()
    sel = iht.iht_cv(ds, y, lab, c["ks"], tol=c["tol"], max_iter=c["max_iter"])
    torch.cuda.synchronize(dev)
    sel_s = time.perf_counter() - w0

    allv = gather_rows([solves, elapsed, args.steps * b, e2e_wall], world)
    if rank == 0:
        value = weak_rate(allv, 0, 1)
        e2e_value = weak_rate(allv, 2, 3)
        peak, peak_kind = measured_tensor_peak()
        n_k = 4 * ((((n + 3) // 4) + 15) // 16) * 16     # samples of the contraction (K-steps x 16)
        # the method's flops: 2 n p per residual column, x 2 for the two-part residual
        # the scope counts (the pass computes five E4M3 limb columns per residual column)
        method_flops = 2.0 * n * p * 2 * cols
        achieved = method_flops / (grad_ms / 1e3) / 1e12 if grad_ms > 0 else None
        limb_tflops = (2.0 * n * p * MR_LIMBS * cols) / (grad_ms / 1e3) / 1e12 if grad_ms > 0 else None
        ktot = sum(c["ks"]) * c["folds"]
        h2d = sum(8 * t.size * len(c["ks"]) + 4 * t.size for t in train)   # y per solve, rows per fold
        out = {
            "metric": "batched IHT solves/sec", "value": value, "unit": "solves/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "warmup_steps_run": warm_steps,
            "ms_per_step": 1e3 * float(allv[:, 1].max()) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "paper_context": PAPER_CONTEXT,
            "dtype": "e4m3 operands (exact dosage, residual in 5 limbs), f32 accumulate, f64 scalars",
            "data": "synthetic",
            "config": {"workload": c["name"], "n": n, "p": p, "folds": c["folds"],
                       "ks": [c["ks"][0], c["ks"][-1]], "solves_per_step": b,
                       "iterations_per_solve": its / max(solves, 1),
                       "grad_impl": args.grad_impl, "l2": "inputs larger than L2 (no flush)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "plain": {"value": b / plain_s, "unit": "solves/s",
                      "what": "the same 100 solves one at a time through iht_fit (single-column path)",
                      "iterations": plain_its},
            "model_selection": {"seconds": sel_s, "k_best": int(sel.k_best),
                                "mse_at_k_best": float(sel.mse[list(c["ks"]).index(sel.k_best)]),
                                "refit_iterations": int(sel.fit.iterations),
                                "what": "iht_cv wall time: 5 folds x k = 1..20 as one batch, "
                                        "out-of-fold MSE on the device, the refit at k_best; "
                                        "host inputs and outputs"},
            "speedup_vs_plain": value / (b / plain_s),
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": (achieved / peak) if achieved else None,
                         "traffic": None,
                         "traffic_first_launch": K2_TRAFFIC_FIRST_LAUNCH_BYTES,
                         "kernel": "multi-column gradient pass (k_grad_mrhs)",
                         "peak_source": peak_kind,
                         "algorithmic_flops": "2 n p x 2 per residual column and pass (the "
                                              "two-part residual); launch durations by CUDA events",
                         "limb_column_tflops": limb_tflops,
                         "limb_columns_note": "the pass runs five E4M3 limb columns per residual "
                                              "column; limb_column_tflops counts those",
                         "columns_total": cols, "launches": grad_n,
                         "ms_per_launch": grad_ms / max(grad_n, 1), "contraction_samples": n_k},
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(12 * ktot)},
            "gpu_launches": int(launches), "clocks": clk,
            "statuses": sorted(set(int(s) for s in statuses)),
            "graph_replays_per_step": replays / max(args.steps, 1),
            "pass_shapes": iht.tuning_summary().strip().splitlines(),
        }
        if not args.no_cpu_baseline and world == 1:
            out["cpu_baseline"] = cv_reference(args, c, pn, bed, y, train, its / max(solves, 1))
        print(json.dumps(out), flush=True)
    del ds, ctx
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def panel_arm(args):
    """Large panel (n = 20 000, p = 4 M, 20 GB packed): the phenotypes in one batch."""
    import torch
    import paper_1608_01398_b300 as iht

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local_rank}"))
    torch.cuda.set_device(local_rank)
    dev = local_rank
    cfg = 5
    c = synth.CONFIGS[cfg]
    t0 = time.perf_counter()
    pn = synth.config_panel(cfg)
    bed = pn.bed()
    ys = [synth.config_phenotype(cfg, pn, which=rank * c["phenotypes"] + i)[0]
          for i in range(c["phenotypes"])]
    n, p, k = pn.n, pn.p, c["k"]
    log(f"[bench] rank {rank}: generated {bed.nbytes / 1e9:.1f} GB panel in {time.perf_counter() - t0:.1f}s")
    stream = torch.cuda.current_stream(dev)
    ctx = iht.Context(dev, stream)
    ds = iht.Dataset(ctx, bed, n, p)
    cuda = f"cuda:{dev}"
    y_dev = [torch.from_numpy(y).to(cuda) for y in ys]
    probs = [(yy, k, None) for yy in y_dev]
    b = len(probs)
    kw = dict(out_device=True, dense=False, grad_impl=args.grad_impl, tol=c["tol"], max_iter=c["max_iter"])
    clocks = ClockSampler(gpu_uuid(torch, dev))
    clocks.start()
    warm_steps = warm_up(lambda: iht.iht_fit_batch(ds, probs, **kw), args.warmup)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    l0 = iht.iht_kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    solves, its, cols, grad_ms, grad_n, statuses, replays = 0, 0, 0, 0.0, 0, [], 0
    for _ in range(args.steps):
        res = iht.iht_fit_batch(ds, probs, profile=1, **kw)
        solves += b
        its += sum(r.iterations for r in res)
        cols += sum(max(r.iterations, 1) for r in res)
        grad_ms += res[0].grad_ms
        grad_n += res[0].grad_launches
        replays += res[0].graph_replays
        statuses += [r.status for r in res]
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    launches = iht.iht_kernel_launches() - l0
    clk = clocks.stop()
    elapsed = ev0.elapsed_time(ev1) / 1e3

    # the same solves one at a time through iht_fit (single-column path)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for (yy, kk, _) in probs:
        iht.iht_fit(ds, yy, kk, out_device=True, grad_impl=args.grad_impl, tol=c["tol"],
                    max_iter=c["max_iter"])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    plain_s = e0.elapsed_time(e1) / 1e3

    # end to end through host buffers
    w0 = time.perf_counter()
    for _ in range(args.steps):
        iht.iht_fit_batch(ds, [(y, k, None) for y in ys], dense=False, grad_impl=args.grad_impl,
                          tol=c["tol"], max_iter=c["max_iter"])
    torch.cuda.synchronize(dev)
    e2e_wall = time.perf_counter() - w0

    allv = gather_rows([solves, elapsed, args.steps * b, e2e_wall], world)
    if rank == 0:
        value = weak_rate(allv, 0, 1)
        peak, peak_kind = measured_tensor_peak()
        achieved = 2.0 * n * p * MR_LIMBS * cols / (grad_ms / 1e3) / 1e12 if grad_ms > 0 else None
        out = {
            "metric": "batched IHT solves/sec", "value": value, "unit": "solves/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "warmup_steps_run": warm_steps,
            "ms_per_step": 1e3 * float(allv[:, 1].max()) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "paper_context": PAPER_CONTEXT,
            "dtype": "e4m3 operands (exact dosage, residual in 5 limbs), f32 accumulate, f64 scalars",
            "data": "synthetic",
            "config": {"workload": c["name"], "n": n, "p": p, "k": k, "phenotypes": b,
                       "iterations_per_solve": its / max(solves, 1), "grad_impl": args.grad_impl,
                       "l2": "inputs larger than L2 (no flush)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "plain": {"value": b / plain_s, "unit": "solves/s",
                      "what": f"the same {b} solves one at a time through iht_fit"},
            "speedup_vs_plain": value / (b / plain_s),
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": None,
                         "kernel": "multi-column gradient pass (k_grad_mrhs)", "peak_source": peak_kind,
                         "algorithmic_flops": "2 n p per residual limb column, five E4M3 limb "
                                              "columns per solve column",
                         "columns_total": cols, "launches": grad_n,
                         "ms_per_launch": grad_ms / max(grad_n, 1)},
            "e2e": {"value": weak_rate(allv, 2, 3), "unit": "solves/s",
                    "h2d_bytes_per_step": 8 * n * b, "d2h_bytes_per_step": 12 * k * b},
            "gpu_launches": int(launches), "clocks": clk,
            "statuses": sorted(set(int(s) for s in statuses)),
            "graph_replays_per_step": replays / max(args.steps, 1),
            "pass_shapes": iht.tuning_summary().strip().splitlines(),
        }
        if not args.no_cpu_baseline and world == 1:
            import oracle
            G = oracle.Geno.from_bed(bed, n, p)
            t1 = time.perf_counter()
            f = oracle.iht(G, ys[0], k, max_iter=1, tol=c["tol"], trace=False)
            dt = time.perf_counter() - t1
            ips = its / max(solves, 1)
            out["cpu_baseline"] = {
                "value": 1.0 / (dt / max(f.iterations, 1) * ips), "unit": "solves/s",
                "cores": oracle.max_threads(), "kind": "oracle",
                "sample": f"FP64 oracle, phenotype 0 on {c['name']}, {f.iterations} iteration "
                          f"(incl. setup) in {dt:.1f}s; solves/s extrapolated at {ips:.1f} "
                          f"iterations per solve"}
        print(json.dumps(out), flush=True)
    del ds, ctx
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def serve_setup(args, rank=0):
    """The panel and the request stream (replicas draw their own requests)."""
    cfg = 4
    c = synth.CONFIGS[cfg]
    pn = synth.config_panel(cfg)
    bed = pn.bed()
    reqs = synth.serving_requests(pn, args.requests, synth.BASE_SEED + 1000 * cfg + 11 + 101 * rank,
                                  workers=min(16, os.cpu_count() or 1))
    return c, pn, bed, reqs


def serve_reference_arm(args):
    """Oracle on a bounded sample: the first request, a few iterations, extrapolated."""
    import oracle
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    c, pn, bed, reqs = serve_setup(args)
    G = oracle.Geno.from_bed(bed, pn.n, pn.p)
    cap = max(1, min(args.oracle_iters, 3))
    vals, secs = [], 0.0
    for s in range(max(args.steps, 1)):
        q = reqs[s % len(reqs)]
        t0 = time.perf_counter()
        f = oracle.iht(G, q["y"], q["k"], rows=q["rows"], max_iter=cap, tol=c["tol"], trace=False)
        dt = time.perf_counter() - t0
        secs += dt
        vals.append(1.0 / (dt / max(f.iterations, 1) * 20.0))
    value = statistics.median(vals)
    out = {"impl": "reference", "metric": "served IHT solves/sec", "value": value,
           "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * secs / max(args.steps, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": c["name"], "n": c["n"], "p": c["p"], "requests": args.requests},
           "cpu_baseline": {"value": value, "unit": "solves/s", "cores": oracle.max_threads(),
                            "kind": "oracle",
                            "sample": f"FP64 oracle, one request per step capped at {cap} iterations "
                                      f"(incl. its statistics pass); solves/s extrapolated at 20 "
                                      f"iterations per solve"},
           "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def _serve_run(iht, srv, reqs, arrivals):
    """Submits reqs at the given offsets (s, from now), collects every result."""
    t0 = time.perf_counter()
    tickets, res = [], {}
    i = 0
    while i < len(reqs) or len(res) < len(reqs):
        now = time.perf_counter() - t0
        while i < len(reqs) and arrivals[i] <= now:
            q = reqs[i]
            tickets.append(srv.submit(q["y"], q["k"], q["rows"]))
            i += 1
        for t in tickets:
            if t not in res:
                r = srv.poll(t)
                if r is not None:
                    res[t] = r
        if i < len(reqs):
            time.sleep(max(0.0, min(0.0005, arrivals[i] - (time.perf_counter() - t0))))
        else:
            time.sleep(0.0005)
    wall = time.perf_counter() - t0
    out = [res[t] for t in tickets]
    lat = np.array([r.latency_s for r in out])
    return wall, lat, out


def _mg1_latency(service, arrivals):
    """Latency of one-at-a-time service (measured service times, cycled) under the arrivals."""
    free, lat = 0.0, []
    for i, a in enumerate(arrivals):
        start = max(a, free)
        free = start + service[i % len(service)]
        lat.append(free - a)
    return np.array(lat)


def serve_arm(args):
    import torch
    import paper_1608_01398_b300 as iht

    rank, local_rank, world = dist_env()
    t0 = time.perf_counter()
    c, pn, bed, reqs = serve_setup(args, rank)    # before any CUDA work (spawned workers)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local_rank}"))
    torch.cuda.set_device(local_rank)
    dev = local_rank
    log(f"[bench] rank {rank}: generated {bed.nbytes / 1e6:.0f} MB panel and {len(reqs)} requests in "
        f"{time.perf_counter() - t0:.1f}s")
    stream = torch.cuda.current_stream(dev)
    ctx = iht.Context(dev, stream)
    ds = iht.Dataset(ctx, bed, pn.n, pn.p)
    solve = dict(tol=c["tol"], max_iter=c["max_iter"])

    # one request at a time through iht_fit (host inputs and outputs)
    nplain = min(len(reqs), args.plain_requests)
    for q in reqs[:2]:
        iht.iht_fit(ds, q["y"], q["k"], rows=q["rows"], **solve)
    service = []
    for q in reqs[:nplain]:
        w0 = time.perf_counter()
        iht.iht_fit(ds, q["y"], q["k"], rows=q["rows"], **solve)
        service.append(time.perf_counter() - w0)
    plain_rate = len(service) / sum(service)

    srv = iht.Server(ds, max_slots=args.slots, hbm_budget=int(args.hbm_gb * 2**30), **solve)
    clocks = ClockSampler(gpu_uuid(torch, dev))
    clocks.start()
    warm_steps = warm_up(lambda: _serve_run(iht, srv, reqs[:min(len(reqs), 2 * args.slots)],
                                            np.zeros(len(reqs))), 1)
    if world > 1:
        torch.distributed.barrier()
    l0 = iht.iht_kernel_launches()
    cap_walls, lat_all, iters = [], [], []
    for _ in range(args.steps):
        wall, lat, out = _serve_run(iht, srv, reqs, np.zeros(len(reqs)))
        cap_walls.append(wall)
        lat_all.append(lat)
        iters += [r.iterations for r in out]
    if world > 1:
        torch.distributed.barrier()
    launches = iht.iht_kernel_launches() - l0
    clk = clocks.stop()
    st = srv.stats()
    value = weak_rate(gather_rows([len(reqs) * args.steps, sum(cap_walls)], world), 0, 1)
    rng = np.random.Generator(np.random.PCG64(synth.BASE_SEED + 4099))
    poisson = {}
    for mult in (0.5, 1.2):
        lam = mult * plain_rate
        npo = min(len(reqs), args.poisson_requests)
        arr = np.cumsum(rng.exponential(1.0 / lam, size=npo))
        arr -= arr[0]
        wall, lat, _ = _serve_run(iht, srv, reqs[:npo], arr)
        plain_lat = _mg1_latency(service, arr)
        poisson[f"{mult}x_plain_rate"] = {
            "arrival_rate": lam, "requests": npo, "served_solves_per_s": npo / wall,
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "plain_p50_ms": 1e3 * float(np.percentile(plain_lat, 50)),
            "plain_p99_ms": 1e3 * float(np.percentile(plain_lat, 99)),
            "plain_latency": "one-at-a-time queue replayed with the measured iht_fit service times"}
    srv.close()
    if rank == 0:
        lat = np.concatenate(lat_all)
        h2d = sum(8 * q["y"].size + 4 * q["rows"].size for q in reqs)
        d2h = sum(12 * q["k"] + 48 for q in reqs)
        out = {
            "metric": "served IHT solves/sec", "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "warmup_steps_run": warm_steps,
            "ms_per_step": 1e3 * sum(cap_walls) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "paper_context": PAPER_CONTEXT,
            "dtype": "e4m3 operands (exact dosage, residual in 5 limbs), f32 accumulate, f64 scalars",
            "data": "synthetic",
            "config": {"workload": c["name"], "n": pn.n, "p": pn.p, "requests_per_step": len(reqs),
                       "max_slots": args.slots, "hbm_budget_gib": args.hbm_gb,
                       "iterations_per_solve": float(np.mean(iters)),
                       "l2": "inputs larger than L2 (no flush)",
                       "arrivals": "all queued at once (capacity)"},
            "latency_ms_all_queued": {"p50": 1e3 * float(np.percentile(lat, 50)),
                                      "p99": 1e3 * float(np.percentile(lat, 99))},
            "plain": {"value": plain_rate, "unit": "solves/s", "requests": len(service),
                      "what": "iht_fit one request at a time, host inputs"},
            "speedup_vs_plain": value / plain_rate,
            "poisson": poisson,
            "server": {k: int(v) for k, v in st.items()},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches), "clocks": clk,
        }
        print(json.dumps(out), flush=True)
    del ds, ctx
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def replay_metrics(support, causal, signal, y):
    """Sec. 3.1 diagnostics of one replicate: precision = |S n C| / |S| and recall
    = |S n C| / |C| of the refit's support S against the causal set C, and
    h^2 = sample variance of the noise-free signal X beta_true / sample variance
    of y (the paper's approximation of narrow-sense heritability)."""
    s = set(int(j) for j in np.asarray(support).ravel())
    c = set(int(j) for j in causal)
    hit = len(s & c)
    return hit / max(len(s), 1), hit / max(len(c), 1), float(np.var(signal) / np.var(y))


def sim_arm(args):
    """Replay of the Sec. 3.1 simulation (synthetic stand-in for its chromosome-1
    matrix): per replicate, a phenotype with k_true causal SNPs at one SNR, 5-fold
    cross-validation over 100 model sizes on 5000 subjects through iht_cv, the
    refit's precision and recall against the causal set and its MSE on the 289
    held-out subjects; one step = the whole replay."""
    import torch
    import paper_1608_01398_b300 as iht

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local_rank}"))
    torch.cuda.set_device(local_rank)
    dev = local_rank
    cfg = 6
    c = synth.CONFIGS[cfg]
    pn = synth.config_panel(cfg)
    n, p = pn.n, pn.p
    stream = torch.cuda.current_stream(dev)
    ctx = iht.Context(dev, stream)
    ds = iht.Dataset(ctx, pn.bed(), n, p)
    cuda = f"cuda:{dev}"
    reps = args.sim_reps if args.sim_reps is not None else c["replicates"]
    split = np.random.Generator(np.random.PCG64(synth.BASE_SEED + 1000 * cfg + 101 * rank))
    test = np.sort(split.choice(n, size=c["test"], replace=False)).astype(np.int32)
    train = np.setdiff1d(np.arange(n), test).astype(np.int32)
    lab = np.full(n, -1, np.int32)
    lab[train] = synth.cv_folds(train.size, c["folds"], synth.BASE_SEED + 1000 * cfg + 7 + 101 * rank)
    _, u_tr, v_tr = iht.iht_counts(ds, rows=train)
    u_d, v_d = torch.from_numpy(u_tr).to(cuda), torch.from_numpy(v_tr).to(cuda)
    test_d = torch.from_numpy(test).to(cuda)
    cells = [(kt, s) for kt in c["k_true"] for s in c["snr_s"]]
    jobs = []
    for ci, (kt, s) in enumerate(cells):
        for r in range(reps):
            seed = synth.BASE_SEED + 1000 * cfg + 100000 * rank + 1000 * ci + r
            y, causal, beta = synth.phenotype(pn, kt, c["effect_var"] / s, c["noise_var"], seed)
            sig = synth.signal(pn, causal, beta)
            jobs.append((ci, kt, s, y, causal, sig))
    kw = dict(tol=c["tol"], max_iter=c["max_iter"], grad_impl=args.grad_impl)
    clocks = ClockSampler(gpu_uuid(torch, dev))
    clocks.start()
    warm_steps = warm_up(lambda: iht.iht_cv(ds, jobs[0][3], lab, synth.sim_path(jobs[0][1], c["path"],
                                                                                c["path_step"]), **kw),
                         args.warmup)                         # tuning, graphs, allocations
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    l0 = iht.iht_kernel_launches()
    rows = []
    w0 = time.perf_counter()
    for _ in range(args.steps):
        rows = []
        for ci, kt, s, y, causal, sig in jobs:
            sel = iht.iht_cv(ds, y, lab, synth.sim_path(kt, c["path"], c["path_step"]), **kw)
            supp = np.asarray(sel.fit.support)
            sb = torch.from_numpy(np.ascontiguousarray(sel.fit.beta[supp])).to(cuda)
            pred = iht.iht_zmul(ds, torch.from_numpy(supp.astype(np.int32)).to(cuda), sb, rows=test_d,
                                u=u_d, v=v_d).cpu().numpy()
            prec, rec, h2 = replay_metrics(supp, causal, sig, y)
            rows.append((ci, sel.k_best, prec, rec, float(np.mean((y[test] - pred) ** 2)), h2))
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - w0
    launches = iht.iht_kernel_launches() - l0
    clk = clocks.stop()
    allv = gather_rows([args.steps * len(jobs), wall], world)
    if rank == 0:
        table = []
        for ci, (kt, s) in enumerate(cells):
            rr = np.array([x[1:] for x in rows if x[0] == ci])
            table.append({"k_true": kt, "snr_pct": round(100.0 / s, 1), "replicates": int(rr.shape[0]),
                          "k_best": float(rr[:, 0].mean()), "precision": float(rr[:, 1].mean()),
                          "recall": float(rr[:, 2].mean()), "test_mse": float(rr[:, 3].mean()),
                          "h2": float(rr[:, 4].mean())})
        value = weak_rate(allv, 0, 1)
        out = {
            "metric": "simulation replicates/sec", "value": value, "unit": "replicates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "warmup_steps_run": warm_steps,
            "ms_per_step": 1e3 * float(allv[:, 1].max()) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "paper_context": PAPER_CONTEXT,
            "dtype": "e4m3 operands (exact dosage, residual in 5 limbs), f32 accumulate, f64 scalars",
            "data": "synthetic stand-in for the Sec. 3.1 chromosome-1 matrix",
            "config": {"workload": c["name"], "n": n, "p": p, "test_subjects": int(test.size),
                       "folds": c["folds"], "path_sizes": c["path"], "path_step": c["path_step"],
                       "replicates_per_cell": reps, "cells": len(cells),
                       "parallelism": "replicas" if world > 1 else "single"},
            "e2e": {"value": value, "unit": "replicates/s", "h2d_bytes_per_step": int(len(jobs) * 12 * n),
                    "d2h_bytes_per_step": int(len(jobs) * 8 * (p + c["test"]))},
            "results": table, "gpu_launches": int(launches), "clocks": clk,
            "what": "one step = every replicate: iht_cv (5 folds x 100 sizes as one batch, "
                    "out-of-fold MSE, refit), precision / recall of the refit's support against "
                    "the causal SNPs, MSE on the held-out subjects; metrics are diagnostics "
                    "(parity of iht_cv is tested against the oracle)",
        }
        print(json.dumps(out), flush=True)
    del ds, ctx
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 50 single solves, 3 CV batches, 1 serving pass)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4, 5, 6])
    ap.add_argument("--sim-reps", type=int, default=None,
                    help="replicates per (k_true, SNR) cell of --config 6 (default 10)")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--plain-requests", type=int, default=40)
    ap.add_argument("--poisson-requests", type=int, default=300)
    ap.add_argument("--slots", type=int, default=64)
    ap.add_argument("--hbm-gb", type=float, default=64.0)
    ap.add_argument("--grad-impl", type=int, default=0, choices=[0, 1, 2])
    ap.add_argument("--oracle-iters", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="single-solve line only (no batched / serving sub-runs)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = {3: 3, 4: 1, 5: 1, 6: 1}.get(args.config, 50)
    if args.config == 3:
        return cv_reference_arm(args) if args.impl == "reference" else cv_arm(args)
    if args.config == 4:
        return serve_reference_arm(args) if args.impl == "reference" else serve_arm(args)
    if args.config == 5:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the large panel's oracle "
                              "reference is the cpu_baseline sample of the --config 5 line"}))
            return 0
        return panel_arm(args)
    if args.config == 6:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the simulation replay has no "
                              "oracle arm: each replicate is 500 cross-validation fits"}))
            return 0
        return sim_arm(args)
    if args.impl == "reference":
        return reference_arm(args)
    return ours_arm(args)


if __name__ == "__main__":
    sys.exit(main())
