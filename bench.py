"""Benchmark of block-based triangle counting on one GB300 (or N replicas).

One step = the whole path on one synthetic graph already resident in device
memory: canonical edge set, degree order and orientation (bbtc_graph_create),
then partition, blocks, tasks, estimate/order and the per-task counting
kernel with the reduction (bbtc_count), then bbtc_graph_destroy.

Metric: oriented edges counted per second (m / step time; m = simple
undirected edges = oriented edges), whole job over all ranks. `e2e` repeats
the step through the same public calls from pinned HOST buffers, so the
host-to-device copy of the input CSR and the device-to-host read of the count
are inside the timed region.

The default workload is the Friendster-shaped Chung-Lu graph (65.6 M vertices,
1.8 G edges) at p = 1; the line also carries a summary of R-MAT scale 23 at
p = 4 (`secondary`). Every printed triangle count is compared with the CPU
oracle's stored count (`golden_match`).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload chunglu-friendster|rmat-s23|rmat-s14|rmat-sNN|
                                   batch-4096|serve] [--p P] [--kernel auto|intersect|hashmap]
                       [--budget-gb B[,B...]] [--secondary rmat-s23|none]
Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(the graph's tasks need no exchange); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "oriented edges/s counted (excl./incl. H2D), % HBM roofline; p50/p99 req latency"
UNIT = "edges/s"

WORKLOADS = {
    "rmat-s23": "R-MAT scale 23 (8,388,608 vertices), edge factor 16, a/b/c/d = "
                ".57/.19/.19/.05, seed 2; symmetrised, self-loops and duplicates removed "
                "by the path itself",
    "rmat-s14": "R-MAT scale 14 (16,384 vertices), edge factor 16, a/b/c/d = "
                ".57/.19/.19/.05, seed 1",
    "chunglu-friendster": "Friendster-shaped Chung-Lu: 65,608,366 vertices, 1,806,067,135 "
                          "pairs, degree exponent 2.1, expected degree capped at 5,000, seed 3; "
                          "symmetrised, self-loops and duplicates removed by the path itself",
    "batch-4096": "4096 independent graphs (seeds 100-4195), pair counts log-uniform "
                  "in [1e3, 2e6]; even g: G(n,m) with average degree 8-64, odd g: "
                  "R-MAT a=.57 with edge factor 8-32",
}
DEFAULT_WORKLOAD = "chunglu-friendster"
DEFAULT_P = {"rmat-s23": 4, "rmat-s14": 2, "chunglu-friendster": 1}
# rows of tests/golden/config_counts.txt (written by tests/golden/make_golden.py
# from graphgen and the CPU oracle alone)
GOLDEN_ROWS = {"rmat-s23": "rmat_s23_ef16_seed2", "rmat-s14": "rmat_s14_ef16_seed1",
               "chunglu-friendster": "chunglu_friendster_seed3"}
GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")


def make_graph(name: str):
    import graphgen
    if name == "rmat-s23":
        return graphgen.rmat_s23()
    if name == "rmat-s14":
        return graphgen.rmat_s14()
    if name == "chunglu-friendster":
        return graphgen.chunglu_friendster()
    if name.startswith("chunglu-friendster/"):  # smaller stand-ins of the same recipe
        return graphgen.chunglu_friendster(scale_down=int(name.split("/")[1]))
    if name.startswith("rmat-s"):  # smaller/larger instances of the same recipe (profiling)
        return graphgen.rmat(int(name[6:]), 16, 2)
    raise SystemExit(f"unknown workload {name}")


def golden_triangles(workload: str):
    """The oracle's stored triangle count of the workload, or None."""
    row = GOLDEN_ROWS.get(workload)
    path = os.path.join(GOLDEN_DIR, "config_counts.txt")
    if row is None or not os.path.exists(path):
        return None
    with open(path) as f:
        for line in f:
            parts = line.split()
            if parts and parts[0] == row:
                return int(parts[3])
    return None


def step_stats(values):
    """[median, min, p90] of per-step times (the paper reports medians of 5 runs)."""
    v = sorted(values)
    return [statistics.median(v), v[0], v[min(len(v) - 1, int(math.ceil(0.9 * len(v))) - 1)]]


def reduce_max_ms(ms: float, dist, device) -> float:
    """Slowest rank's time: the job is done when every replica is."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: int, world: int, ms: float) -> float:
    """Whole-job rate of `world` independent replicas, each doing units_per_rank."""
    return world * units_per_rank / (ms / 1000.0)


def kernel_source_hash() -> str:
    """sha256 of the counting kernel's source (a changed kernel voids old counters)."""
    import hashlib
    path = os.path.join(ROOT, "paper_2009_12457_gb300", "csrc", "count.cu")
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def recorded_traffic(workload: str, p: int, kernel: str):
    """DRAM bytes per counting-kernel launch from the committed ncu record, when it
    was taken on this kernel source and this workload; else None."""
    path = os.path.join(ROOT, "profiles", "k_count_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    for r in rec.get("records", []):
        if (r.get("source_sha256") == kernel_source_hash() and r.get("workload") == workload
                and r.get("p") == p and r.get("kernel") == kernel):
            return r.get("dram_bytes_per_launch")
    return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples every 100 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix=f"bbtc_clocks_gpu{gpu_index}_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- CPU oracle
#
# The oracle (single-threaded C, tests-only otherwise) is timed here on a
# bounded sample of the bench workload's own recipe: a scaled-down instance of
# the Friendster-shaped Chung-Lu graph (same exponent and cap, n and the pair
# count divided by `scale_down`) or a smaller R-MAT scale. Estimated seconds
# per oracle pass on one Grace core, from measured runs (R-MAT scale 19: 5.8 s;
# Chung-Lu / 256: about 4 s), pick the sample that fits the time budget.

CHUNGLU_SAMPLE_S = {1024: 0.6, 512: 1.6, 256: 4.1, 128: 9.9, 64: 24.0}


def oracle_sample(workload: str, budget_s: float):
    """(label, generator) of the largest sample whose oracle pass fits budget_s."""
    import graphgen
    if workload.startswith("chunglu-friendster"):
        sd = 1024
        for cand in sorted(CHUNGLU_SAMPLE_S, reverse=True):
            if CHUNGLU_SAMPLE_S[cand] <= budget_s:
                sd = cand
        return (f"Friendster-shaped Chung-Lu recipe scaled down {sd}x (gamma 2.1, cap 5,000, "
                f"seed 3)", lambda: graphgen.chunglu_friendster(scale_down=sd))
    scale = 12
    for s in range(12, 21):
        if 6.0 * 2.3 ** (s - 19) <= budget_s:
            scale = s
    return (f"R-MAT scale {scale}, edge factor 16, seed 2",
            lambda: graphgen.rmat(scale, 16, 2))


def run_oracle_sample(gen, p: int):
    """Oracle pipeline (prepare + Alg. 5 per task) on one sample graph; `gen` is a
    generator callable or an already generated (n, rowptr, colidx)."""
    import oracle
    n, rp, ci = gen() if callable(gen) else gen
    t0 = time.perf_counter()
    r = oracle.bbtc(n, rp, ci, p=p)
    dt = time.perf_counter() - t0
    return r["m"], dt, r["total"]


def cpu_baseline(workload: str, p: int):
    label, gen = oracle_sample(workload, 12.0)
    m, dt, total = run_oracle_sample(gen, p)
    return {"value": m / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle pipeline (canonicalise, order, orient, partition p={p}, "
                      f"Alg. 5 per task) on {label} ({m} edges, {dt:.2f} s, {total} "
                      f"triangles); single-threaded C"}


def reference_arm(args, rank: int, world: int):
    if rank != 0:
        return
    workload = args.workload or DEFAULT_WORKLOAD
    steps_total = args.steps + args.warmup
    label, gen = oracle_sample(workload, 150.0 / max(steps_total, 1))
    p = int(str(args.p).split(",")[0]) or DEFAULT_P.get(workload, 4)
    graph = gen()  # generated once; each step times the oracle on it
    for _ in range(args.warmup):
        run_oracle_sample(graph, p)
    times, m = [], 0
    for _ in range(args.steps):
        m, dt, _ = run_oracle_sample(graph, p)
        times.append(dt)
    ms = 1000.0 * sum(times) / len(times)
    value = m / (ms / 1000.0)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS.get(workload, workload), "p": p,
                   "sample": f"{label} ({m} edges) per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{label} per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ batched form

def run_batch(args, world, rank, local_rank):
    """4096 graphs: one union prep + one counting launch per step, against one
    plain create/count/destroy per graph; plus the union's count captured in a
    CUDA graph and replayed. Choices (p, kernel threshold, work-item size) come
    from the autotuner run on the union."""
    import torch
    import graphgen
    import paper_2009_12457_gb300 as bb
    from paper_2009_12457_gb300.autotune import Autotuner

    torch.cuda.set_device(local_rank)
    ng = int(args.workload.split("-")[1])
    graphs = graphgen.batch_graphs(ng)
    voff, rowptr, colidx = bb.batch_csr(graphs)
    flags = bb.INPUT_SYMMETRIC
    stream = torch.cuda.Stream()
    d_rp = torch.from_numpy(rowptr).cuda()
    d_ci = torch.from_numpy(colidx).cuda()
    singles = []
    for g, (n, rp, ci) in enumerate(graphs):
        e0, e1 = int(rowptr[voff[g]]), int(rowptr[voff[g + 1]])
        singles.append((n, (d_rp[voff[g]:voff[g] + n + 1] - e0).contiguous(), d_ci[e0:e1]))
    torch.cuda.synchronize()

    # autotune once on the union (choices are cached per size class)
    h = bb.bbtc_graph_create_batch(voff, d_rp, d_ci, flags, stream)
    choice = Autotuner(cache_path=None, repeats=1).tune(h, p_choices=(1, 2, 4, 8))
    m_total = bb.bbtc_graph_get_info(h)["m"]
    bb.bbtc_graph_destroy(h)
    kw = dict(p=choice["p"], kernel=choice["kernel"], hash_threshold=choice["hash_threshold"],
              chunk=choice["chunk"], stream=stream)

    def batched_step():
        hh = bb.bbtc_graph_create_batch(voff, d_rp, d_ci, flags, stream)
        pg = np.zeros(ng, dtype=np.uint64)
        try:
            bb.bbtc_count(hh, bb.make_opts(per_graph_out=pg, **kw))
        finally:
            bb.bbtc_graph_destroy(hh)
        return pg

    for _ in range(args.warmup):
        ref = batched_step()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = bb.bbtc_kernel_launches()
    with ClockSampler(local_rank) as clocks:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            got = batched_step()
            assert np.array_equal(got, ref)
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = bb.bbtc_kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1) / args.steps

    # the union's count alone, captured in a CUDA graph and replayed
    hh = bb.bbtc_graph_create_batch(voff, d_rp, d_ci, flags, stream)
    pg_first = np.zeros(ng, dtype=np.uint64)
    bb.bbtc_count(hh, bb.make_opts(per_graph_out=pg_first, **kw))
    pg_dev = torch.zeros(ng, dtype=torch.int64, device="cuda")
    tot_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
    aopts = bb.make_opts(per_graph_out=pg_dev, **kw)
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=stream):
        bb.bbtc_count_async(hh, aopts, tot_dev)
    cg.replay()
    torch.cuda.synchronize()
    assert np.array_equal(pg_dev.cpu().numpy().astype(np.uint64), ref)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            cg.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    captured_ms = e0.elapsed_time(e1) / args.steps
    bb.bbtc_graph_destroy(hh)

    # one plain create + count + destroy per graph (same inputs, same choices)
    def plain_step():
        out = np.zeros(ng, dtype=np.uint64)
        for g, (n, rp_g, ci_g) in enumerate(singles):
            hg = bb.bbtc_graph_create_async(n, rp_g, ci_g, flags, stream)
            try:
                out[g] = bb.bbtc_count(hg, bb.make_opts(**kw))
            finally:
                bb.bbtc_graph_destroy(hg)
        return out

    plain_step()
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    plain = plain_step()
    p1.record(stream)
    torch.cuda.synchronize()
    plain_ms = p0.elapsed_time(p1)
    assert np.array_equal(plain, ref), "batched and plain per-graph counts differ"

    # end to end: host inputs, per-graph counts read back every step
    h_rp = torch.from_numpy(rowptr).pin_memory()
    h_ci = torch.from_numpy(colidx).pin_memory()
    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    q0.record(stream)
    for _ in range(args.steps):
        hh = bb.bbtc_graph_create_batch(voff, h_rp, h_ci, flags, stream)
        pg = np.zeros(ng, dtype=np.uint64)
        bb.bbtc_count(hh, bb.make_opts(per_graph_out=pg, **kw))
        bb.bbtc_graph_destroy(hh)
    q1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = q0.elapsed_time(q1) / args.steps

    # every graph's count against the oracle's stored value (the first ng of 4096)
    golden_path = os.path.join(GOLDEN_DIR, "batch4096_counts.txt")
    golden_match = None
    if os.path.exists(golden_path):
        want = {}
        with open(golden_path) as f:
            for row in f:
                if row.strip() and not row.startswith("#"):
                    g_, _, _, tri = (int(x) for x in row.split())
                    want[g_] = tri
        if all(g_ in want for g_ in range(ng)):
            golden_match = bool(all(int(ref[g_]) == want[g_] for g_ in range(ng)))
    peak, peak_kind = measured_peaks()
    line = {
        "metric": METRIC, "value": m_total / (ms / 1000.0), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS.get(args.workload,
                                             f"{ng} independent graphs (seeds 100-{99 + ng}), "
                                             "the first of the 4096-graph recipe"),
                   "graphs": ng, "m_total": m_total,
                   "triangles_total": int(ref.sum()), "golden_match": golden_match,
                   "autotuned": choice,
                   "l2": "inputs larger than L2 (%.2f GB)" % (colidx.nbytes / 1e9)},
        "batched_vs_plain": {"plain_ms_per_step": plain_ms, "batched_ms_per_step": ms,
                             "speedup": plain_ms / ms,
                             "plain_edges_per_s": m_total / (plain_ms / 1000.0)},
        "captured_count_ms": captured_ms,
        "e2e": {"value": m_total / (e2e_ms / 1000.0), "unit": UNIT,
                "h2d_bytes_per_step": rowptr.nbytes + colidx.nbytes + voff.nbytes,
                "d2h_bytes_per_step": 8 * ng},
        "clocks": clocks.summary(), "gpu_launches": launches,
        "peak_hbm_gbs": {"value": peak, "source": peak_kind},
    }
    print(json.dumps(line), flush=True)
    if golden_match is False:
        raise SystemExit("batched per-graph counts differ from the oracle's stored counts")


# ------------------------------------------------------------ serving form

def run_serve(args, world, rank, local_rank):
    """Open-loop Poisson arrivals of count requests on R-MAT graphs of mixed scale
    (10-22, edge factor 16; each request's graph seed is drawn from its id, from
    a pool of `--serve-seeds` per scale so the device-resident cache can hit).
    Reports p50/p99 latency and graphs/s at each arrival rate, against two serial
    baselines: plain per-request launches (create + count + destroy, no cache, no
    batching) and one count per request on resident handles (the cache without
    the batching). Admission is by free device memory; --serve-budget-gb caps the
    cache as well when nonzero."""
    import torch
    import graphgen
    from paper_2009_12457_gb300 import serve

    torch.cuda.set_device(local_rank)
    scales = list(range(10, 23))
    seeds = args.serve_seeds
    rates = [float(x) for x in args.serve_rates.split(",")]

    def key_of(rid):
        d = graphgen.draw(5, 11, rid)
        return (scales[d % len(scales)], (d >> 32) % seeds)

    keys_all = [key_of(i) for i in range(200000)]
    pool = {}
    t0 = time.perf_counter()
    for k in sorted(set(keys_all[:20000])):
        pool[k] = graphgen.rmat(k[0], 16, 1000 * k[0] + k[1])
    gen_s = time.perf_counter() - t0

    def source(k):
        if k not in pool:
            pool[k] = graphgen.rmat(k[0], 16, 1000 * k[0] + k[1])
        return pool[k]

    # serial baselines on the first requests
    nser = min(args.serve_serial, len(keys_all))
    serve_p = int(str(args.p).split(",")[0])
    ser_counts, serial_gps = serve.serial_baseline(source, keys_all[:nser], symmetric=True,
                                                   p=serve_p)
    cached_counts, serial_cached_gps = serve.serial_cached_baseline(
        source, keys_all[:nser], symmetric=True, p=serve_p)
    if ser_counts != cached_counts:
        raise SystemExit("serial baselines disagree")
    expect = dict(zip(keys_all[:nser], ser_counts))
    budget = int(args.serve_budget_gb * (1 << 30)) or None
    results = []
    offset = 0
    for lam in rates:
        arrivals = serve.poisson_trace(lam, args.serve_seconds, seed=5)
        keys = keys_all[offset:offset + len(arrivals)]
        offset += len(arrivals)
        srv = serve.Server(source, device_budget_bytes=budget, max_batch=256, workers=2,
                           p=serve_p, symmetric=True)
        try:
            reqs = serve.run_open_loop(srv, keys, arrivals)
        finally:
            srv.close()
        bad = [r for r in reqs if r.status != 0]
        mismatched = sum(1 for r in reqs if r.key in expect and r.count != expect[r.key])
        summ = serve.latency_summary(reqs)
        summ.update({"rate_hz": lam, "failed": len(bad), "cache_hits": srv.hits,
                     "cache_misses": srv.misses, "evictions": srv.evictions,
                     "admission_waits": srv.admission_waits,
                     "counts_checked_against_serial": sum(1 for r in reqs if r.key in expect),
                     "counts_mismatched": mismatched, "errors": srv.errors[:4]})
        results.append(summ)
    best = max(r["graphs_per_s"] for r in results)
    line = {
        "metric": METRIC, "impl": "serve", "unit": "graphs/s",
        "value": best, "n_gpus": 1,
        "higher_is_better": True, "data": "synthetic",
        "config": {"workload": "serving: Poisson arrivals, R-MAT scales 10-22, edge factor 16",
                   "seconds_per_rate": args.serve_seconds, "seed_pool_per_scale": seeds,
                   "admission": "free device memory (bbtc_device_memory) minus a 4 GiB reserve"
                                + (f", cache capped at {args.serve_budget_gb} GB" if budget else ""),
                   "p": serve_p, "host_generation_s": gen_s},
        "serial_plain_graphs_per_s": serial_gps,
        "serial_cached_graphs_per_s": serial_cached_gps,
        "served_vs_serial_plain": best / serial_gps,
        "served_vs_serial_cached": best / serial_cached_gps,
        "rates": results,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- GPU path

def measure(args, workload: str, p: int, budget_gb: float, env, with_cpu: bool):
    """Times one workload at one (p, budget): W warm-up steps, then K timed steps
    from device-resident input and K from pinned host input. Returns rank 0's line
    (None on the other ranks)."""
    import torch
    import paper_2009_12457_gb300 as bb
    from paper_2009_12457_gb300 import shard
    world, rank, local_rank, dist = env
    # --shard: the ranks share one graph's task list (strong scaling); else every
    # rank counts its own replica (weak scaling)
    shard_tasks = bool(args.shard) and world > 1

    def barrier():
        if dist is not None:
            dist.barrier()

    n, rp, ci = make_graph(workload)
    flags = bb.INPUT_SYMMETRIC  # the generator lists every pair under both endpoints
    stream = torch.cuda.Stream()
    h_rp = torch.from_numpy(rp).pin_memory()
    h_ci = torch.from_numpy(ci).pin_memory()
    d_rp = h_rp.cuda()
    d_ci = h_ci.cuda()
    torch.cuda.synchronize()
    del rp, ci
    budget = int(budget_gb * (1 << 30))

    def step(device_resident: bool, want_info: bool = False):
        if device_resident:
            h = bb.bbtc_graph_create_async(n, d_rp, d_ci, flags, stream)
        else:
            h = bb.bbtc_graph_create_async(n, h_rp, h_ci, flags, stream)
        try:
            if shard_tasks:  # this rank's share of the task list; one sum over ranks
                total = shard.shard_count(h, p, rank, world, dist, "cuda", kernel=args.kernel,
                                          stream=stream, device_budget_bytes=budget,
                                          partition=args.partition)
            else:
                total = bb.bbtc_count(h, bb.make_opts(p=p, kernel=args.kernel, stream=stream,
                                                      device_budget_bytes=budget,
                                                      partition=args.partition))
            # the graph's sizes and wedge sums (an extra pass over the CSR) are
            # read in the warm-up only, outside the timed steps
            info = bb.bbtc_graph_get_info(h) if want_info else None
            tim = bb.bbtc_graph_get_timings(h)
        finally:
            bb.bbtc_graph_destroy(h)
        return total, info, tim

    # warm-up (also validates that every step gives the same count)
    totals = set()
    info = None
    for _ in range(args.warmup):
        total, info, _ = step(True, want_info=True)
        totals.add(total)
    m = info["m"]

    # timed: device-resident inputs
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    count_ms, prep_ms, plan_ms, stream_info = [], [], [], []
    launches0 = bb.bbtc_kernel_launches()
    with ClockSampler(local_rank) as clocks:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            total, _, tim = step(True)
            totals.add(total)
            count_ms.append(tim["count_ms"])
            prep_ms.append(tim["prep_ms"])
            plan_ms.append(tim["plan_ms"])
            stream_info.append({k: tim[k] for k in ("stream_rounds", "stream_h2d_bytes",
                                                    "stream_copy_ms", "stream_block_bytes",
                                                    "stream_device_peak_bytes",
                                                    "stream_mode")})
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = bb.bbtc_kernel_launches() - launches0
    ms = reduce_max_ms(ev0.elapsed_time(ev1) / args.steps, dist, "cuda")

    # timed: host inputs through the same calls (H2D and count D2H inside),
    # after one untimed host-input step (the device pool grows once for the
    # input copy)
    totals.add(step(False)[0])
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2e_phase = {"prep": [], "plan": [], "count_kernel": []}
    w0 = time.perf_counter()
    e0.record(stream)
    for _ in range(args.steps):
        total, _, tim = step(False)
        totals.add(total)
        e2e_phase["prep"].append(tim["prep_ms"])
        e2e_phase["plan"].append(tim["plan_ms"])
        e2e_phase["count_kernel"].append(tim["count_ms"])
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_wall_ms = 1000.0 * (time.perf_counter() - w0) / args.steps
    e2e_ms = reduce_max_ms(e0.elapsed_time(e1) / args.steps, dist, "cuda")
    barrier()

    if len(totals) != 1:
        raise SystemExit(f"inconsistent triangle counts across steps: {sorted(totals)}")
    triangles = next(iter(totals))
    golden = golden_triangles(workload)

    # load imbalance of the partition (Sec. 4.4): lambda = m_max / m_avg over the
    # p(p+1)/2 blocks, from one more (untimed) plan
    h = bb.bbtc_graph_create_async(n, d_rp, d_ci, flags, stream)
    try:
        bb.bbtc_graph_plan(h, bb.make_opts(p=p, kernel=args.kernel, stream=stream,
                                           partition=args.partition))
        nnz = bb.bbtc_graph_get_plan(h, p)["block_nnz"]
        dev_bytes = bb.bbtc_graph_get_info(h)["device_bytes"]
    finally:
        bb.bbtc_graph_destroy(h)
    lam = float(nnz.max()) / (m / (p * (p + 1) / 2)) if m else 1.0

    # pinned host-to-device bandwidth right now (streamed counts depend on it,
    # and it varies from box to box)
    h2d_gbs = None
    if budget:
        k = min(int(h_ci.numel()), 1 << 28)
        tmp = torch.empty(k, dtype=torch.int32, device="cuda")
        with torch.cuda.stream(stream):
            tmp.copy_(h_ci[:k], non_blocking=True)
            b0 = torch.cuda.Event(enable_timing=True)
            b1 = torch.cuda.Event(enable_timing=True)
            b0.record(stream)
            for _ in range(3):
                tmp.copy_(h_ci[:k], non_blocking=True)
            b1.record(stream)
        torch.cuda.synchronize()
        h2d_gbs = 3 * 4 * k / (b0.elapsed_time(b1) / 1000.0) / 1e9
        del tmp
    input_entries = int(h_ci.numel())
    del d_rp, d_ci, h_rp, h_ci
    torch.cuda.empty_cache()
    if rank != 0:
        return None

    peak, peak_kind = measured_peaks()
    kms = sum(count_ms) / len(count_ms)
    # bytes the destination-grouped counting kernel reads: the 16-byte in-edge
    # records, each N(v) staged once (4 B per oriented edge), and the part of each
    # N(u) above v (sum over u of d+(u)(d+(u)-1)/2 elements, 4 B each)
    own = 4 * (5 * m + info["wedges_out"])
    achieved = own / (kms / 1000.0) / 1e9
    # W_min: every edge's N(v) read once per in-edge of v; this kernel
    # never makes those reads, so it is reported for context, not as its roofline
    wmin = 4 * (m + info["wedges_in"])
    # bytes a merge-based intersection of both full lists would read:
    # 4 * sum over (u,v) of (d+(u) + d+(v)), with sum_(u,v) d+(u) = sum_u d+(u)^2
    # = 2 * sum_u C(d+(u), 2) + m
    wmerge = 4 * (2 * info["wedges_out"] + m + info["wedges_in"])
    h2d = (n + 1) * 8 + input_entries * 4
    traffic = recorded_traffic(workload, p, args.kernel) if not budget else None
    line = {
        "metric": METRIC,
        "value": (m / (ms / 1000.0)) if shard_tasks else replica_throughput(m, world, ms),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "strong" if shard_tasks else "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic",
        "config": {
            "workload": WORKLOADS.get(workload, workload), "p": p,
            "kernel": args.kernel, "partition": args.partition,
            "lambda": lam, "max_block_nnz": int(nnz.max()),
            "n": n, "m": m, "triangles": triangles,
            "golden_triangles": golden, "golden_match": (None if golden is None
                                                         else triangles == golden),
            "input_entries": input_entries,
            "l2": "inputs larger than L2 (input CSR %.2f GB, oriented CSR %.2f GB)"
                  % (h2d / 1e9, (m * 8 + (n + 1) * 8) / 1e9),
            "parallelism": ("task list shared over ranks (LPT by ExecTime), one sum"
                            if shard_tasks else "replicas" if world > 1 else "single GPU"),
            "phase_ms": {"prep": statistics.mean(prep_ms), "plan": statistics.mean(plan_ms),
                         "count_kernel": kms},
            "phase_ms_median_min_p90": {k: step_stats(v) for k, v in
                                        (("prep", prep_ms), ("plan", plan_ms),
                                         ("count_kernel", count_ms))},
            "device_budget_gb": budget_gb,
            "handle_and_plan_device_bytes": dev_bytes,
            "streaming": dict(stream_info[-1], pinned_h2d_gbs=h2d_gbs,
                              h2d_over_block_bytes=(stream_info[-1]["stream_h2d_bytes"] /
                                                    max(stream_info[-1]["stream_block_bytes"], 1)),
                              budget_bytes=budget) if budget else None,
        },
        "e2e": {"value": (m / (e2e_ms / 1000.0)) if shard_tasks
                else replica_throughput(m, world, e2e_ms), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8,
                "ms_per_step": e2e_ms, "host_wall_ms_per_step": e2e_wall_ms,
                "phase_ms": {k: statistics.mean(v) for k, v in e2e_phase.items()}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": traffic,
                     "traffic_source": ("committed ncu record of this kernel source and "
                                        "workload (profiles/k_count_traffic.json), not "
                                        "measured in this run" if traffic is not None else
                                        "no ncu record for this kernel source and workload"),
                     "kernel": "k_count (per-task counting, a9)",
                     "algorithmic_bytes": own,
                     "bytes_formula": "4*(5m + sum over u of d+(u)(d+(u)-1)/2): 16-byte "
                                      "in-edge records, each N(v) staged once, the probed "
                                      "part of each N(u) above v",
                     "w_min_bytes": wmin,
                     "w_min_formula": "4*(m + sum over oriented edges (u,v) of d+(v)); reads "
                                      "N(v) once per in-edge, which this kernel does not do",
                     "w_min_over_time_per_peak": wmin / (kms / 1000.0) / 1e9 / peak,
                     "w_merge_bytes": wmerge,
                     "peak_source": f"{peak_kind} hbm_gbs"},
        "clocks": clocks.summary(),
        "gpu_launches": launches,
    }
    if with_cpu:
        line["cpu_baseline"] = cpu_baseline(workload, p)
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=None,
                    help="chunglu-friendster (default), rmat-s23, rmat-s14, rmat-sNN, "
                         "chunglu-friendster/D (scaled down D times), batch-4096, serve")
    ap.add_argument("--secondary", default="rmat-s23",
                    help="with the default workload: a second workload summarised in the "
                         "same line ('none' to skip)")
    ap.add_argument("--p", default="0", help="blocks per side; a comma list runs each")
    ap.add_argument("--kernel", default="auto", choices=["auto", "intersect", "hashmap"])
    ap.add_argument("--partition", default="edges", choices=["edges", "probe"],
                    help="edges: contiguous parts balanced on oriented edges; probe: "
                         "probe-based partition bounding the largest block")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shard", action="store_true",
                    help="under torchrun: the ranks share one graph's tasks (Alg. 7 / Alg. 9) "
                         "instead of each counting a replica")
    ap.add_argument("--budget-gb", default="0",
                    help="comma list of device budgets (GB) for the counting step's blocks, "
                         "streamed from pinned host memory; 0 = resident; one line each")
    ap.add_argument("--serve-rates", default="200,500,1000,2000,5000")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-seeds", type=int, default=4)
    ap.add_argument("--serve-budget-gb", type=float, default=0.0,
                    help="cap on the serving cache (GB); 0 = admission by free device memory")
    ap.add_argument("--serve-serial", type=int, default=300)
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be at least 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    default_run = args.workload is None
    workload = args.workload or DEFAULT_WORKLOAD
    if workload.startswith("batch-"):
        run_batch(args, world, rank, local_rank)
        return
    if workload == "serve":
        run_serve(args, world, rank, local_rank)
        return

    import torch
    import paper_2009_12457_gb300 as bb

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    env = (world, rank, local_rank, dist)

    p_list = [int(x) for x in str(args.p).split(",")]
    p_list = [q or DEFAULT_P.get(workload.split("/")[0], 4) for q in p_list]
    budgets = [float(x) for x in str(args.budget_gb).split(",")]
    first = True
    for p in p_list:
        for budget_gb in budgets:
            try:
                line = measure(args, workload, p, budget_gb, env,
                               with_cpu=first and world == 1 and not args.no_cpu_baseline)
            except bb.BbtcError as e:  # e.g. a budget too small for one task's blocks
                line = {"metric": METRIC, "error": str(e), "p": p,
                        "device_budget_gb": budget_gb, "workload": workload}
            first = False
            if default_run and args.secondary != "none":  # every rank measures it
                sec = measure(args, args.secondary, DEFAULT_P.get(args.secondary, 4), 0.0, env,
                              with_cpu=False)
                if sec is not None and line is not None:
                    line["secondary"] = {
                        "workload": sec["config"]["workload"], "p": sec["config"]["p"],
                        "value": sec["value"], "unit": UNIT, "ms_per_step": sec["ms_per_step"],
                        "e2e": sec["e2e"], "phase_ms": sec["config"]["phase_ms"],
                        "triangles": sec["config"]["triangles"],
                        "golden_match": sec["config"]["golden_match"],
                        "roofline_frac": sec["roofline"]["frac"],
                        "roofline_achieved_gbs": sec["roofline"]["achieved"],
                        "w_min_over_time_per_peak": sec["roofline"]["w_min_over_time_per_peak"],
                        "clocks": sec["clocks"], "gpu_launches": sec["gpu_launches"]}
            if line is not None:
                print(json.dumps(line), flush=True)
            if line is not None and line.get("config", {}).get("golden_match") is False:
                raise SystemExit(f"triangle count {line['config']['triangles']} differs from "
                                 f"the oracle's {line['config']['golden_triangles']}")

    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
