#!/usr/bin/env python
"""Benchmark: time to a certified top-k Katz ranking (Algorithm 1) and the
walk-count SpMV throughput on one GB300, through the library's C ABI.

One step = one katz_rank_static call: every iteration of Algorithm 1
(walk-count SpMV fused with the bound update, selection of the k-th lower
bound, deactivation count, converged()) until the ranking is certified.
Inputs are resident in HBM when the timed region starts; L2 is flushed
between steps.  value = GTEPS = r * nnz / time (walk-recurrence arcs
traversed per second, summed over ranks).

The default workload is the largest one: a Chung-Lu graph with 2^27
vertices and about 2.13 G arcs (int64 row offsets), certified top-100.  The
headline is the FP64 path (the paper's precision); the FP32-certified path is
timed beside it on the same graph ("fp32cert", with the speedup and whether
both certified the same ranking), and the FP32-certified bounds' per-node
deviation from the FP64 oracle at the same r is reported against the
rounding widening ("fp32cert_deviation_vs_oracle").  "cpu_baseline" times
the CPU oracle on all host cores (complete rankings), with a single-threaded
sample of its first iterations ("single_thread") and the host's nproc and CPU
model ("host").

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--precision fp64|fp32cert] [--no-compare]

N > 1 runs N independent replicas (the method needs no exchange between
GPUs at these sizes), launched by torch.distributed.run.

Beside the static line the default run serves a stream of update batches on
R-MAT23 (Algorithm 2 through the serving loop) and reports it under
"serving" (FP64 levels) and "serving_fp32cert" (FP32-certified levels):
capacity, p50/p99 latency at 200 batches/s and at 70% of capacity, device
time per batch and the static recomputation it is compared with.
--serve-batches 0 skips them; --workload serve-rmat23 makes the serving run
the headline (p99 latency).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "rmat22": dict(graph="rmat22", k=1000, eps=1e-9, alpha=0.0, precision=0,
                   desc="undirected R-MAT scale 22 (4,194,304 vertices), edge factor 16, (a,b,c,d)=(.57,.19,.19,.05), "
                        "symmetrised and deduplicated, int32 CSR; alpha=1/(deg_max+1); certified top-1000; eps=1e-9"),
    "rmat21": dict(graph="rmat21", k=1000, eps=1e-9, alpha=0.0, precision=0,
                   desc="undirected R-MAT scale 21 (2,097,152 vertices), edge factor 16, (a,b,c,d)=(.57,.19,.19,.05), "
                        "symmetrised and deduplicated, int32 CSR; alpha=1/(deg_max+1); certified top-1000; eps=1e-9 "
                        "(profiling case: col array larger than L2, a few GB on the device)"),
    "rmat24": dict(graph="rmat24", k=1000, eps=1e-9, alpha=0.0, precision=0,
                   desc="undirected R-MAT scale 24 (16,777,216 vertices), edge factor 16, (a,b,c,d)=(.57,.19,.19,.05), "
                        "symmetrised and deduplicated, int32 CSR; alpha=1/(deg_max+1); certified top-1000; eps=1e-9"),
    "rmat24-halfalpha": dict(graph="rmat24", k=1000, eps=1e-9, alpha="half", precision=0,
                             desc="undirected R-MAT scale 24, edge factor 16; alpha=0.5/deg_max; certified top-1000; "
                                  "eps=1e-9"),
    "chunglu27": dict(graph="chunglu27", k=100, eps=1e-9, alpha=0.0, precision=0,
                      desc="undirected Chung-Lu graph, n=2^27 (134,217,728) vertices, expected degrees Pareto with "
                           "exponent 2.1 and mean 16 (about 2^30 endpoint pairs before symmetrising and "
                           "deduplicating), int64 rowptr / int32 col CSR; alpha=1/(deg_max+1); certified top-100; "
                           "eps=1e-9"),
    "chunglu25": dict(graph="chunglu25", k=100, eps=1e-9, alpha=0.0, precision=0,
                      desc="undirected Chung-Lu graph, n=2^25 vertices, expected degrees Pareto with exponent 2.1 "
                           "and mean 16, int32 CSR; alpha=1/(deg_max+1); certified top-100; eps=1e-9 (profiling case "
                           "of the n=2^27 workload: walk vector larger than L2, a few GB on the device)"),
    "er16k": dict(graph="er16k", k=100, eps=1e-9, alpha=0.0, precision=0,
                  desc="undirected Erdos-Renyi n=16384, m=131072, int32 CSR; alpha=1/(deg_max+1); certified top-100; "
                       "eps=1e-9"),
}

SERVING = dict(graph="rmat23", k=100, eps=1e-9, rate=200.0, min_size=1, max_size=10000, p_insert=0.5,
               desc="undirected R-MAT scale 23 base graph (8,388,608 vertices, edge factor 16); update batches of "
                    "log-uniform size in [1, 10^4], 50% inserts of uniform non-edges / 50% deletes of uniform existing "
                    "edges; Poisson arrivals at 200 batches/s; deg_bound = deg_max + 64, alpha = 1/(deg_bound+1); "
                    "certified top-100 after every batch; eps=1e-9")

HBM_PEAK_FALLBACK = 6800.0  # GB/s, used only if MEASURED_PEAKS.json is absent
METRIC = "certified top-k Katz: walk-recurrence GTEPS (time to certified ranking in ms_per_step)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["serve-rmat23"], default="chunglu27")
    ap.add_argument("--precision", choices=["fp64", "fp32cert"], default=None,
                    help="precision of the headline value (default: FP64, the paper's)")
    ap.add_argument("--no-compare", action="store_true",
                    help="time the headline precision only (default: the other one is timed beside it)")
    ap.add_argument("--serve-precision", choices=["fp64", "fp32cert", "both"], default="both",
                    help="walk levels of the served handle (FP32-certified: FP32 from the level the ranking picks); "
                         "both: the FP64 run in 'serving', the FP32-certified one in 'serving_fp32cert'")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-iters", type=int, default=3,
                    help="--impl reference on graphs above 2^30 arcs: oracle iterations per step")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="CPU work of the cpu_baseline sample")
    ap.add_argument("--serve-batches", type=int, default=None,
                    help="batches of the serving stream (default 2000; 0 skips it beside the static line)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_PEAK_FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
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
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash():
    h = hashlib.sha1()
    for fn in ("katz_spmv.cu", "katz_common.cuh"):
        with open(os.path.join(ROOT, "paper_1807_03847_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def ncu_traffic(workload: str, precision: str):
    """DRAM bytes per SpMV launch from the committed ncu summary, if it was
    taken on this workload, in this precision, on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "spmv_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(f"{workload}-{precision}")
        if e and e.get("source_hash") == kernel_source_hash():
            return e
    except Exception:
        pass
    return None


def spmv_algorithmic_bytes(n, nnz, fp32: bool, off64: bool):
    """Compulsory bytes of one walk-count SpMV launch: col (4/nnz), rowptr,
    s_{r-1} read once, s_r write, c_r read+write, active flag read."""
    vb = 4 if fp32 else 8
    return 4 * nnz + (8 if off64 else 4) * (n + 1) + 2 * vb * n + 16 * n + n


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x, world, op):
    """x reduced over the ranks (NCCL: on the GPU; gloo: on the host)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def allreduce_max(x, world):
    import torch.distributed as dist
    return _reduce(x, world, dist.ReduceOp.MAX if world > 1 else None)


def allreduce_sum(x, world):
    import torch.distributed as dist
    return _reduce(x, world, dist.ReduceOp.SUM if world > 1 else None)


def replica_throughput(units_local, seconds_local, world):
    """Whole-job value of N independent replicas: the units all ranks
    processed over the slowest rank's time (barrier-bracketed regions)."""
    return allreduce_sum(units_local, world) / allreduce_max(seconds_local, world)


def cpu_baseline(g, wl, seconds):
    """The CPU oracle as it stands (Algorithm 1, OpenMP rows, sequential
    partial sort) on a bounded sample: complete certified rankings of the
    full graph, repeated until `seconds` of CPU work have been done (at least
    one).  Returns the baseline and the oracle session, which holds the last
    ranking's bounds (the caller closes it)."""
    import oracle

    s = oracle.Session(g.rowptr, g.col, True)
    # the same oracle on one thread, on a bounded sample (the first
    # iterations of Algorithm 1), before the multi-threaded rankings so that
    # the session ends on a complete ranking
    threads = oracle.max_threads()
    oracle.set_threads(1)
    t1 = time.perf_counter()
    r1 = s.iterations(wl["alpha"], wl["k"], wl["eps"], SINGLE_THREAD_ITERS)
    dt1 = time.perf_counter() - t1
    oracle.set_threads(threads)
    single = {"value": r1 * g.nnz / dt1 / 1e9, "unit": "GTEPS", "threads": 1,
              "sample": f"the first {r1} iterations of Algorithm 1 on the full {wl['graph']} graph; {dt1:.1f} s"}
    runs, arcs = 0, 0
    t0 = time.perf_counter()
    while True:
        r = s.iterations(wl["alpha"], wl["k"], wl["eps"], 10000)
        runs += 1
        arcs += r * g.nnz
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": arcs / dt / 1e9, "unit": "GTEPS", "cores": threads, "kind": "oracle",
            "sample": f"{runs} complete certified ranking(s) (r = {r}) of the full {wl['graph']} graph; "
                      f"{dt:.1f} s", "single_thread": single, "host": host_cpu()}, s


def host_cpu():
    """nproc and the CPU model of the host the oracle ran on."""
    model = platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "model": model}


def run_serving(batches, workers=2, slots=8, precision="fp64"):
    """Open-loop serving runs on one R-MAT23 handle: the batches of the stream
    are submitted at their arrival times to a katz_server; latency is
    submit -> certified top-k on the host.  First at the specified rate
    (200 batches/s), then at 70% of the capacity that run measured (so the
    queue is stable), then the static recomputation of the final graph
    (katz_rank_static on the same handle) as the baseline.  The capacity is
    the throughput of the first run when it saturates (batches of one handle
    are pipelined: the prepare of a batch overlaps the repair of the one
    before it, and two queued batches share one two-state pass, so one
    request's service time is not the rate)."""
    import torch

    import graphgen as gg

    cfg = SERVING
    g = gg.workload(cfg["graph"])
    D = g.deg_max() + 64
    spec = serve_once(g, D, batches, cfg["rate"], workers, slots, torch, precision)
    saturated = spec["achieved_rate"] < 0.97 * spec["offered_rate"]
    capacity = spec["achieved_rate"] if saturated else spec["offered_rate"]
    stable = serve_once(g, D, batches, round(0.7 * capacity, 1), workers, slots, torch, precision)
    spec["capacity_batches_per_s"] = capacity
    spec["within_capacity"] = stable
    return spec


def serve_once(g, D, batches, rate, workers, slots, torch, precision="fp64"):
    import graphgen as gg
    import paper_1807_03847_gb300 as K

    cfg = SERVING
    st = gg.stream(g, batches, seed=gg.SEED_BASE + 230, min_size=cfg["min_size"], max_size=cfg["max_size"],
                   p_insert=cfg["p_insert"], rate=rate, deg_bound=D)
    prec = K.KATZ_FP32_CERT if precision == "fp32cert" else K.KATZ_FP64
    h = K.Katz(torch.from_numpy(g.rowptr).cuda(), torch.from_numpy(g.col).cuda(),
               K.katz_default_opts(keep_history=1, deg_bound=D, precision=prec))
    info0 = h.rank(0.0, cfg["k"], cfg["eps"])
    srv = K.Server(workers=workers, slots=slots, slot_updates=cfg["max_size"])
    srv.attach(h, cfg["k"])
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    tickets = []
    t0 = time.perf_counter()
    for j in range(len(st)):
        delay = t0 + st.arrival[j] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        tickets.append(srv.submit(h, *st.batch(j)))
    results = [srv.wait(t, timeout_ms=600000) for t in tickets]
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    srv.close()
    bad = [r[0] for r in results if r[0] != 0]
    lat = np.array([r[2].latency_ms for r in results])
    svc = np.array([r[2].service_ms for r in results])
    dev = np.array([r[2].info.time_ms for r in results])
    aff = np.array([r[2].info.affected for r in results], np.float64)
    full = np.array([r[2].info.full_levels for r in results], np.float64)
    launches = int(sum(r[2].info.launches for r in results))
    fp32_levels = [r[2].info.fp32_levels for r in results]
    paired = np.array([r[2].paired for r in results], np.float64)
    sizes = st.sizes()
    # full static recomputation of the final graph, same handle (graph resident)
    rec_dev, rec_wall = [], []
    for _ in range(3):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        inf = h.rank(0.0, cfg["k"], cfg["eps"])
        rec_wall.append(1e3 * (time.perf_counter() - t1))
        rec_dev.append(inf.time_ms)
    h.close()
    small = sizes <= 100
    return {
        "offered_rate": rate, "achieved_rate": len(st) / wall,
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "service_p50_ms": float(np.percentile(svc, 50)), "service_p99_ms": float(np.percentile(svc, 99)),
        "device_p50_ms": float(np.percentile(dev, 50)),
        "p50_ms_batches_le_100": float(np.percentile(lat[small], 50)) if small.any() else None,
        "recompute_ms": float(np.median(rec_wall)), "recompute_device_ms": float(np.median(rec_dev)),
        "batches": int(len(st)), "updates": int(sizes.sum()), "rejected": len(bad),
        "affected_mean_frac": float(aff.mean() / g.n), "full_levels_mean": float(full.mean()),
        "r_initial": int(info0.r), "gpu_launches": launches, "workers": workers, "slots": slots,
        "precision": precision, "fp32_levels_initial": int(info0.fp32_levels),
        "paired_frac": float(paired.mean()),
        "fp32_levels_median": float(np.median(fp32_levels)),
        "clocks": clocks, "n": g.n, "nnz": g.nnz, "deg_bound": D, "desc": cfg["desc"],
        "latency": "submit (at the batch's arrival time) -> certified top-100 copied to the host",
    }


# graphs above this many arcs are sampled by the reference arm: each step runs
# the first --cpu-iters iterations of Algorithm 1 instead of a whole ranking
REFERENCE_SAMPLE_ARCS = 1 << 30
# iterations of the single-threaded oracle sample beside the cpu_baseline
SINGLE_THREAD_ITERS = 2


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, timed on the host cores
    on the same workload, metric and unit.  Each step is one complete
    certified ranking, or on graphs above 2^30 arcs a bounded sample of it
    (the first --cpu-iters iterations: walk recurrence, bounds, converged())
    so that the run stays within minutes."""
    world, rank = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import graphgen as gg
    import oracle

    wl = dict(WORKLOADS[args.workload])
    g = gg.workload(wl["graph"])
    if wl["alpha"] == "half":
        wl["alpha"] = 0.5 / g.deg_max()
    sampled = g.nnz > REFERENCE_SAMPLE_ARCS
    iters = args.cpu_iters if sampled else 10000
    s = oracle.Session(g.rowptr, g.col, True)
    times, edges = [], []
    r = 0
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = s.iterations(wl["alpha"], wl["k"], wl["eps"], iters)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            edges.append(r * g.nnz)
    s.close()
    total = sum(times)
    value = sum(edges) / total / 1e9
    if sampled:
        sample = (f"each step: the first {r} iterations of Algorithm 1 (walk recurrence, bounds, converged()) on "
                  f"the full {wl['graph']} graph, a bounded sample of one certified ranking (oracle, FP64, "
                  f"OpenMP rows + sequential partial sort)")
    else:
        sample = (f"each step: one complete certified ranking (r = {r} iterations of Algorithm 1) of the full "
                  f"{wl['graph']} graph (oracle, FP64, OpenMP rows + sequential partial sort)")
    line = {"metric": METRIC, "value": value, "unit": "GTEPS",
            "impl": "reference", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}-top{wl['k']}-fp64", "graph": wl["desc"], "n": g.n,
                       "nnz": g.nnz, "k": wl["k"], "eps": wl["eps"]},
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": sample, "host": host_cpu()},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_static(K, torch, g, wl, precision, steps, warmup, stream, flush, world, rank):
    """W untimed warm-up rankings, then exactly `steps` certified rankings
    timed with CUDA events on the handle's stream, L2 flushed before each,
    barrier + synchronize on both sides; clocks sampled during the timed
    region.  Returns the handle (still open), the infos and the step times."""
    rowptr_d = torch.from_numpy(g.rowptr).cuda()
    col_d = torch.from_numpy(g.col).cuda()
    opts = K.katz_default_opts(precision=precision, profile=1, cuda_stream=stream.cuda_stream,
                               l2_fetch_bytes=wl.get("l2_fetch", 0))
    h = K.Katz(rowptr_d, col_d, opts)
    del rowptr_d, col_d  # the handle holds its own relabelled copy
    for _ in range(warmup):
        h.rank(wl["alpha"], wl["k"], wl["eps"])
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    barrier(world)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    infos = []
    for i in range(steps):
        flush.zero_()
        evs[i][0].record(stream)
        infos.append(h.rank(wl["alpha"], wl["k"], wl["eps"]))
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop() if sampler else None
    return h, infos, [a.elapsed_time(b) for a, b in evs], clocks


def spmv_roofline(infos, n, nnz, off64, fp32_run, hbm_peak, hbm_src, tr):
    """Roofline of the walk-count SpMV (levels 2..r) from the launch times the
    library measured with CUDA events on its stream.  Algorithmic bytes per
    launch: col, row offsets, s_{r-1} read once, s_r written, c read and
    written, the active flags; an FP32-certified ranking's levels before its
    switch move FP64 values, the ones after it FP32 values (averaged over the
    launches)."""
    spmv_ms = sum(inf.spmv_ms for inf in infos)
    launches = sum(inf.spmv_launches for inf in infos)
    total_bytes = 0
    for inf in infos:
        levels = list(range(2, inf.r + 1))[:inf.spmv_launches]
        f32_from = inf.r - inf.fp32_levels + 1 if (fp32_run and inf.fp32_levels) else 1 << 30
        total_bytes += sum(spmv_algorithmic_bytes(n, nnz, lv >= f32_from, off64) for lv in levels)
        total_bytes += spmv_algorithmic_bytes(n, nnz, fp32_run, off64) * max(0, inf.spmv_launches - len(levels))
    t_launch = spmv_ms / 1e3 / max(launches, 1)
    bytes_alg = total_bytes / max(launches, 1)
    ach = bytes_alg / t_launch / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
            "traffic": tr["bytes_per_launch"] if tr else None,
            "traffic_source": tr.get("command") if tr else None,
            "peak_source": f"{hbm_src} hbm_gbs (burst copy)",
            "algorithmic_bytes_per_launch": bytes_alg, "spmv_ms_per_launch": t_launch * 1e3,
            "gathers_per_s": nnz / t_launch, "launches": launches,
            "limiter": "random gathers of s_{r-1} (one L1 request per arc; beyond L2 one DRAM sector per "
                       "missed gather) and, for FP64 levels, the integer adds of the exact row sums"}


def deviation_stats(lo, up, err, l_ref, u_ref):
    """Per-node deviation of FP32-certified bounds from the FP64 oracle's at
    the same r, absolute and relative to the reported rounding widening."""
    dl = np.abs(lo - l_ref)
    du = np.abs(up - u_ref)
    w = np.where(err > 0, err, np.inf)
    out = {}
    for name, d in (("lower", dl), ("upper", du)):
        rel = d / w
        out[name] = {"max_abs": float(d.max()), "p99_abs": float(np.percentile(d, 99)),
                     "max_over_widening": float(rel[np.isfinite(rel)].max(initial=0.0)),
                     "p99_over_widening": float(np.percentile(rel[np.isfinite(rel)], 99)) if np.isfinite(rel).any()
                     else 0.0}
    out["widening_max"] = float(err.max())
    out["widening_p99"] = float(np.percentile(err, 99))
    # each certified bound lies within err of the exact bound at r; the
    # oracle's FP64 bounds carry their own rounding (1e-12 relative)
    out["within_widening"] = bool(np.all(dl <= err + 1e-12 * np.abs(l_ref) + 1e-300) and
                                  np.all(du <= err + 1e-12 * np.abs(u_ref) + 1e-300))
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    if args.workload == "serve-rmat23":
        rank = int(os.environ.get("RANK", "0"))
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        if args.serve_precision == "both":
            args.serve_precision = "fp64"
        sv = run_serving(args.serve_batches or 2000, precision=args.serve_precision)
        if rank == 0:
            print(json.dumps({
                "metric": "update-to-certified top-100 latency p99 (serving, dynamic R-MAT23)",
                "value": sv["p99_ms"], "unit": "ms", "n_gpus": 1, "steps": sv["batches"], "warmup": 0,
                "ms_per_step": sv["p50_ms"], "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.serve_precision == "fp32cert" else "f64", "data": "synthetic",
                "config": {"workload": f"serve-rmat23-top100-{args.serve_precision}", "graph": sv["desc"],
                           "l2": "not flushed: requests run back to back as they arrive"},
                "serving": sv, "gpu_launches": sv["gpu_launches"], "clocks": sv["clocks"],
                "e2e": {"value": sv["p99_ms"], "unit": "ms",
                        "h2d_bytes_per_step": int(9 * sv["updates"] / sv["batches"]),
                        "d2h_bytes_per_step": 400},
            }), flush=True)
        return

    import graphgen as gg
    import paper_1807_03847_gb300 as K

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    wl = dict(WORKLOADS[args.workload])
    # the headline precision, and the other one timed beside it (--precision
    # picks the headline; --no-compare times it alone)
    head_prec = args.precision or ("fp64" if wl["precision"] == 0 else "fp32cert")
    other_prec = None if args.no_compare else ("fp32cert" if head_prec == "fp64" else "fp64")
    g = gg.workload(wl["graph"])
    n, nnz = g.n, g.nnz
    if wl["alpha"] == "half":
        wl["alpha"] = 0.5 / g.deg_max()
    stream = torch.cuda.current_stream()
    # the serving runs first, on the context's defaults (a headline handle
    # created with katz_opts.l2_fetch_bytes would leave the limit explicitly set)
    serving = serving32 = None
    if args.serve_batches is None:
        args.serve_batches = 2000
    if args.serve_batches > 0:
        if args.serve_precision in ("fp64", "both"):
            serving = run_serving(args.serve_batches, precision="fp64")
        if args.serve_precision in ("fp32cert", "both"):
            serving32 = run_serving(args.serve_batches, precision="fp32cert")
        torch.cuda.empty_cache()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)
    hbm_peak, hbm_src = peaks()
    off64 = (n + nnz) >= 0x7fffffff

    arms = {}
    for prec in [head_prec] + ([other_prec] if other_prec else []):
        code = K.KATZ_FP32_CERT if prec == "fp32cert" else K.KATZ_FP64
        h, infos, step_ms, clocks = time_static(K, torch, g, wl, code, args.steps, args.warmup, stream, flush,
                                                world, rank)
        total_s = sum(step_ms) / 1e3
        edges_local = sum(inf.r * nnz for inf in infos)
        arm = {"precision": prec, "infos": infos, "clocks": clocks,
               "total_s_max": allreduce_max(total_s, world),
               "value": replica_throughput(edges_local, total_s, world) / 1e9,
               "ranking": [int(x) for x in h.ranking(wl["k"])],
               "roofline": spmv_roofline(infos, n, nnz, off64, prec == "fp32cert", hbm_peak, hbm_src,
                                         ncu_traffic(args.workload, prec))}
        if prec == "fp32cert" and rank == 0 and world == 1 and not args.no_cpu_baseline:
            arm["bounds"] = h.bounds()  # compared with the oracle's below
        h.close()
        arms[prec] = arm
    head = arms[head_prec]
    infos = head["infos"]
    r = infos[-1].r
    launches = sum(inf.launches for inf in infos)
    fp32_head = head_prec == "fp32cert"

    # end to end through the public API from pinned host buffers
    e2e = None
    if not args.no_e2e:
        rp_pin = torch.from_numpy(g.rowptr).pin_memory()
        col_pin = torch.from_numpy(g.col).pin_memory()
        out_pin = torch.empty(wl["k"], dtype=torch.int32).pin_memory()
        e2e_opts = K.katz_default_opts(precision=K.KATZ_FP32_CERT if fp32_head else K.KATZ_FP64,
                                       cuda_stream=stream.cuda_stream, l2_fetch_bytes=wl.get("l2_fetch", 0))
        e2e_times, e2e_edges = [], 0
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hh = K.Katz(rp_pin, col_pin, e2e_opts)
            inf = hh.rank(wl["alpha"], wl["k"], wl["eps"])
            K.katz_get_ranking(hh.h, wl["k"], out_pin)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            hh.close()
            if i > 0:  # first call pays one-time module loading
                e2e_times.append(dt)
                e2e_edges += inf.r * nnz
        e2e_t = allreduce_max(sum(e2e_times), world)
        e2e = {"value": allreduce_sum(e2e_edges, world) / e2e_t / 1e9, "unit": "GTEPS",
               "h2d_bytes_per_step": int(g.rowptr.nbytes + g.col.nbytes), "d2h_bytes_per_step": int(4 * wl["k"]),
               "ms_per_step": 1e3 * e2e_t / len(e2e_times),
               "api": "katz_create_csr(host pinned CSR) + katz_rank_static + katz_get_ranking(host) + katz_destroy"}
        del rp_pin, col_pin


    cpu = None
    deviation = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, sess = cpu_baseline(g, wl, args.cpu_seconds)
        if "fp32cert" in arms and "bounds" in arms["fp32cert"]:
            lo, up, err = arms["fp32cert"]["bounds"]
            r32 = arms["fp32cert"]["infos"][-1].r
            if sess.info()["r"] != r32:  # the oracle's bounds at the FP32-certified run's r
                sess.run_fixed(wl["alpha"], r32)
            _, l_ref, u_ref = sess.bounds()
            deviation = deviation_stats(lo, up, err, l_ref, u_ref)
            deviation["r"] = r32
        sess.close()

    def arm_summary(a):
        inf = a["infos"][-1]
        return {"value": a["value"], "unit": "GTEPS", "ms_per_step": 1e3 * a["total_s_max"] / args.steps,
                "r": inf.r, "fp32_levels": int(inf.fp32_levels), "roofline": a["roofline"],
                "spmv_gteps": nnz / (a["roofline"]["spmv_ms_per_launch"] / 1e3) / 1e9,
                "gpu_launches": int(sum(i.launches for i in a["infos"])), "clocks": a["clocks"],
                "ranking_head": a["ranking"][:5]}

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": head["value"], "unit": "GTEPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * head["total_s_max"] / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if fp32_head else "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}-top{wl['k']}-{head_prec}",
                       "graph": wl["desc"], "n": n, "nnz": nnz, "k": wl["k"], "eps": wl["eps"],
                       "alpha": infos[-1].alpha, "r": r, "parallelism": f"replicas{world}",
                       "offsets": "int64" if off64 else "int32",
                       "l2_fetch_bytes": wl.get("l2_fetch", 0),
                       "l2": "flushed between steps (256 MB write); col array alone is larger than L2"},
            "time_to_certified_ms": 1e3 * head["total_s_max"] / args.steps,
            "spmv_gteps": nnz / (head["roofline"]["spmv_ms_per_launch"] / 1e3) / 1e9,
            "fp32_levels": int(infos[-1].fp32_levels),
            "roofline": head["roofline"], "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": head["clocks"], "ranking_head": head["ranking"][:5],
        }
        if other_prec:
            other = arms[other_prec]
            line[other_prec] = arm_summary(other)
            t32 = arms["fp32cert"]["total_s_max"]
            t64 = arms["fp64"]["total_s_max"]
            line["fp32cert_speedup_over_fp64"] = t64 / t32
            line["same_ranking_fp32cert_fp64"] = arms["fp32cert"]["ranking"] == arms["fp64"]["ranking"]
        if deviation is not None:
            line["fp32cert_deviation_vs_oracle"] = deviation
        line["serving"] = serving
        line["serving_fp32cert"] = serving32
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
