#!/usr/bin/env python3
"""Benchmark of the GPU multilevel partitioner; prints one JSON line.

A step is one pass of the whole hot path over the benchmark graph:
compression of the CSR graph into the gap+VarInt format, a full multilevel
partition of the compressed graph, and a full partition of the plain CSR
graph (the metric compares both paths). Inputs are resident in HBM when the
timed region starts and are larger than L2, so no flush is needed.

value = level-0 LP clustering throughput on the compressed graph in GTEPS:
(clustering rounds x 2m adjacency entries) / CUDA-event time of those rounds.

--impl reference times the CPU oracle (the reference arm of this repo) on
bounded samples of the same workload.

Multi-GPU (torchrun, one process per GPU): the path shards as independent
graphs, so every rank partitions its own replica of the workload with no
collective on the data path (weak scaling); only the barrier and the
max-over-ranks timing use the process group.
"""
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

METRIC = "LP clustering GTEPS + partition time, compressed vs CSR; % of HBM peak"
WORKLOADS = {
    "rgg24": dict(gen="rgg2d", n=1 << 24, deg=16.0, k=64, seed=1,
                  desc="2D random geometric graph n=2^24, expected degree 16, unit weights, "
                       "k=64, eps=0.03, seed 1; gap+VarInt compressed and int32 CSR"),
    "rgg23": dict(gen="rgg2d", n=1 << 23, deg=16.0, k=64, seed=1,
                  desc="2D random geometric graph n=2^23 (half-size profiling case), expected "
                       "degree 16, unit weights, k=64, eps=0.03, seed 1"),
    "gnm14": dict(gen="gnm", n=1 << 14, m=1 << 17, k=8, seed=1,
                  desc="G(n,m) n=2^14 m=2^17, unit weights, k=8, eps=0.03, seed 1"),
    "rmat26": dict(gen="rmat", scale=26, ef=16, k=256, seed=1,
                   desc="R-MAT scale 26 edge factor 16 (0.57,0.19,0.19,0.05), symmetrised, "
                        "deduplicated, k=256, eps=0.03, seed 1; compressed with chunking and CSR"),
    "rmat22": dict(gen="rmat", scale=22, ef=16, k=256, seed=1,
                   desc="R-MAT scale 22 (profiling case of the skewed tiers), edge factor 16 "
                        "(0.57,0.19,0.19,0.05), symmetrised, deduplicated, k=256, eps=0.03, "
                        "seed 1; compressed with chunking"),
    "serve": dict(gen="serve", count=64, seed=1, log2_lo=10.0, log2_hi=26.0, resident_log2=26,
                  resident_deg=32.0, budget=150e9, workers=16, load=0.7,
                  desc="serving: 64 requests, n log-uniform in [2^10, 2^26], G(n,m) deg 8 / "
                       "RGG-2D deg 12 / RHG deg 16 gamma 2.8 in turn, k log-uniform in [2, 1024], "
                       "every 8th request on a resident compressed RHG n=2^26 deg 32 gamma 2.8; "
                       "Poisson arrivals at 70% of the measured capacity; 150 GB budget; eps=0.03"),
    "serve22": dict(gen="serve", count=128, seed=1, log2_lo=10.0, log2_hi=22.0, resident_log2=23,
                    resident_deg=32.0, budget=150e9, workers=16, load=0.7,
                    desc="serving (small): 128 requests, n log-uniform in [2^10, 2^22], the same "
                         "generators and k, every 8th request on a resident compressed RHG n=2^23 "
                         "deg 32 gamma 2.8; Poisson arrivals at 70% of capacity; 150 GB budget"),
    "batch4096": dict(gen="batch", count=4096, seed=1,
                      desc="batched: 4096 independent graphs, n log-uniform in [2^8, 2^16], "
                           "G(n,m) deg 8 / RGG-2D deg 12 / RHG deg 16 gamma 2.8 in turn, k in "
                           "{2,4,8,16,32} per graph, eps=0.03, seed 1; int32 CSR"),
}
EPS = 0.03
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e data-sheet bandwidth, the second denominator
KERNEL_NAMES = {"rate_lane": "k_rate_lane", "rate_small": "k_rate_small",
                "rate_mid": "k_rate_list (shared tables)", "rate_big": "k_rate_list (global tables)",
                "rate_huge": "k_rate_huge_chunks + k_rate_huge_decide"}


def host_cpu():
    """CPU model and logical core count of the host that runs the oracle."""
    import platform

    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                key, _, val = ln.partition(":")
                fields.setdefault(key.strip(), val.strip())
    except OSError:
        pass
    model = fields.get("model name")
    if not model and fields.get("CPU part"):
        model = f"{platform.machine()} implementer {fields.get('CPU implementer', '?')} " \
                f"part {fields['CPU part']}"
    return {"model": model or platform.machine(), "nproc": os.cpu_count()}


def make_graph(w):
    import synth

    if w["gen"] == "rgg2d":
        return synth.rgg2d(w["n"], w["deg"], w["seed"])
    if w["gen"] == "gnm":
        return synth.gnm(w["n"], w["m"], w["seed"])
    return synth.rmat(w["scale"], w["ef"], seed=w["seed"])


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


KERNEL_SOURCES = {  # files that define each profiled kernel family
    "rate": ("lp.cu", "decode.cuh", "tp_internal.cuh"),
}


def kernel_source_hash(family="rate"):
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2410_19119_gb300", "csrc")
    for name in KERNEL_SOURCES[family]:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_tag, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernels (same source hash) and workload."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}_{workload}.txt")
    try:
        fields = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    fields[k.strip()] = v.strip()
        if fields.get("source_hash") != kernel_source_hash("rate"):
            return None
        return float(fields["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) < 9:
                        continue
                    try:
                        sm.append(float(parts[1]))
                        mx = float(parts[2])
                    except ValueError:
                        continue
                    for name, val in zip(names, parts[5:9]):
                        if val.lower().startswith("active"):
                            reasons.add(name)
            os.unlink(self.path)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum of a list of floats over all ranks (identity
    without a process group): the slowest rank sets every time."""
    if dist is None:
        return list(values)
    import torch

    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def shard(count, rank, ws):
    """Indices of independent work units (graphs, requests) owned by a rank:
    round robin, so every rank gets a similar size mix; no unit is shared and
    no collective touches the data path."""
    return list(range(rank, count, ws))


def bench_config(w, n, m2, ws):
    """The config object both arms print (the reference arm runs the same
    workload on the host)."""
    return {"workload": w["desc"], "n": n, "m2": m2, "k": w["k"], "eps": EPS,
            "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{ws}"}


E2E_UNIT = "GTEPS"
E2E_DEF = ("level-0 LP clustering edges (5 rounds x 2m) per second of one whole user call "
           "chain: host CSR in, graph creation, compression, partition, partition back to host")


def cpu_oracle_lp(xadj, adj, k, seed, max_rounds=5, budget_s=12.0):
    """Oracle level-0 clustering rounds (one thread) until the budget is spent."""
    import oracle

    g = oracle.Graph(xadj, adj)
    n = g.n
    U = oracle.cluster_cap(n, k, oracle.eps_to_ppm(EPS))
    label = np.arange(n, dtype=np.int32)
    lw = np.ones(n, np.int64)
    t0 = time.perf_counter()
    rounds = 0
    while rounds < max_rounds:
        oracle.lp_rounds(g, label, lw, n, U, None, seed, oracle.tag(oracle.TAG_CLUSTER), 0, rounds,
                         1, 8)
        rounds += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return rounds * len(adj) / dt / 1e9, rounds, dt


def run_reference(args, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle

    xadj, adj = make_graph(w)
    g = oracle.Graph(xadj, adj)
    n = g.n
    U = oracle.cluster_cap(n, w["k"], oracle.eps_to_ppm(EPS))
    label = np.arange(n, dtype=np.int32)
    lw = np.ones(n, np.int64)
    tag = oracle.tag(oracle.TAG_CLUSTER)
    r = 0

    def one_round():
        nonlocal r, label, lw
        if r == 5:  # a level has five rounds; start the level again
            label = np.arange(n, dtype=np.int32)
            lw = np.ones(n, np.int64)
            r = 0
        oracle.lp_rounds(g, label, lw, n, U, None, w["seed"], tag, 0, r, 1, 8)
        r += 1

    for _ in range(args.warmup):
        one_round()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one_round()
    dt = time.perf_counter() - t0
    value = args.steps * len(adj) / dt / 1e9
    sample = f"one level-0 LP clustering round (8 sub-rounds) of the full graph per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": bench_config(w, n, len(adj), ws),
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                             "sample": sample, "host": host_cpu()},
            "e2e": {"value": value, "unit": E2E_UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_lp_only(args, w):
    """Level-0 clustering of the compressed graph only (for profiler captures)."""
    import torch

    import paper_2410_19119_gb300 as tp

    xadj, adj = make_graph(w)
    g = tp.graph_from_csr(xadj, adj).compress()
    n = len(xadj) - 1
    U = max(1, (30000 * n) // (1000000 * w["k"]))
    tp.lp_cluster(g, U, tp.default_params(seed=w["seed"]), 0)
    torch.cuda.synchronize()
    print(json.dumps({"lp_only": w["desc"], "n": n, "m2": len(adj)}))


def run_batch(args, w):
    """Batched mode: the whole batch per step through tp_partition_batch with
    autotuned knobs (one union graph per level), against the plain
    single-graph path (the same graphs partitioned one after another on one
    stream)."""
    import torch

    import paper_2410_19119_gb300 as tp
    import synth
    from paper_2410_19119_gb300 import autotune

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    # weak scaling: count graphs per GPU, every rank its own shard of a
    # recipe of count * ws graphs (independent problems, no collective)
    recipe_all = synth.batch_recipe(w["count"] * ws, seed=w["seed"])
    recipe = [recipe_all[i] for i in shard(len(recipe_all), rank, ws)]
    t0 = time.perf_counter()
    csr = [synth.batch_graph(s) for s in recipe]
    gen_s = time.perf_counter() - t0
    graphs = [tp.graph_from_csr(x, a) for x, a in csr]
    ks = [s["k"] for s in recipe]
    total_n = sum(len(x) - 1 for x, _ in csr)
    total_m2 = sum(len(a) for _, a in csr)
    t0 = time.perf_counter()
    params, table = autotune.autotune(graphs, ks, EPS, seed=w["seed"])
    tune_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        tp.partition_batch(graphs, ks, EPS, params)
    torch.cuda.synchronize()
    l0 = tp.launch_count()
    times = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = tp.partition_batch(graphs, ks, EPS, params)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    launches = tp.launch_count() - l0
    batch_s = statistics.median(times)
    if dist:
        dist.barrier()
    # the plain single-graph path, default knobs, one stream
    p0 = tp.default_params(seed=w["seed"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = [tp.partition(g, k, EPS, p0) for g, k in zip(graphs, ks)]
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    same = all(bool(torch.equal(a[0], b[0])) for a, b in zip(out, plain))
    batch_s, plain_s, same_f = max_over_ranks([batch_s, plain_s, 0.0 if same else 1.0], dist,
                                              "cuda")
    same = same_f == 0.0
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    knobs = {f: getattr(params, f) for f, _ in autotune.KNOBS}
    line = {
        "metric": METRIC, "value": len(graphs) * ws / batch_s, "unit": "graphs/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": batch_s * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": w["desc"], "graphs": len(graphs), "total_n": total_n,
                   "total_m2": total_m2, "timing": "host clock around the blocking batch call"},
        "batch_ms": batch_s * 1e3, "plain_single_graph_ms": plain_s * 1e3,
        "speedup_vs_plain": plain_s / batch_s, "identical_to_plain": same,
        "lp_level0_edges_per_s": 5.0 * total_m2 / batch_s,
        "autotune": {"knobs": knobs, "seconds": tune_s,
                     "trials": len(table)},
        "generate_s": gen_s, "gpu_launches": launches // max(args.steps, 1),
        "sum_cut": sum(st["cut"] for _, st in out),
    }
    print(json.dumps(line), flush=True)


def run_batch_once(args, w):
    """One warm-up and one timed batched partition with default knobs (for
    profiler captures)."""
    import torch

    import paper_2410_19119_gb300 as tp
    import synth

    recipe = synth.batch_recipe(w["count"], seed=w["seed"])
    graphs = [tp.graph_from_csr(*synth.batch_graph(s)) for s in recipe]
    ks = [s["k"] for s in recipe]
    p = tp.default_params(seed=w["seed"])
    tp.partition_batch(graphs, ks, EPS, p)
    torch.cuda.synchronize()
    l0 = tp.launch_count()
    t0 = time.perf_counter()
    out = tp.partition_batch(graphs, ks, EPS, p)
    torch.cuda.synchronize()
    st = out[0][1]
    print(json.dumps({"batch_once": w["desc"], "ms": (time.perf_counter() - t0) * 1e3,
                      "launches": tp.launch_count() - l0, "ms_coarsen": st["ms_coarsen"],
                      "ms_initial": st["ms_initial"], "ms_uncoarsen": st["ms_uncoarsen"],
                      "peak_bytes": st["peak_bytes"]}), flush=True)


def serve_recipe(w):
    """Requests of the serving workload (input generation only)."""
    import synth

    out = []
    for i in range(w["count"]):
        u = (synth._sm64(w["seed"], 3 * i) >> 11) * (1.0 / 9007199254740992.0)
        v = (synth._sm64(w["seed"], 3 * i + 1) >> 11) * (1.0 / 9007199254740992.0)
        k = max(2, min(1024, int(round(2.0 ** (1.0 + 9.0 * v)))))
        if i % 8 == 7:
            out.append({"resident": True, "k": k})
            continue
        n = int(round(2.0 ** (w["log2_lo"] + (w["log2_hi"] - w["log2_lo"]) * u)))
        gen = synth.BATCH_GENERATORS[i % 3]
        out.append({"resident": False, "gen": gen, "n": n, "k": k, "seed": (w["seed"] << 32) + i,
                    "deg": {"gnm": 8.0, "rgg2d": 12.0, "rhg": 16.0}[gen], "compress": i % 2 == 1})
    return out


def run_serve(args, w):
    """Serving with continuous batching: capacity (all requests at once),
    the plain path (one request at a time), then Poisson arrivals at 70% of
    the capacity with p50/p99 latency."""
    import torch

    import paper_2410_19119_gb300 as tp
    import synth

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    reqs = serve_recipe(w)
    t0 = time.perf_counter()
    host = {i: synth.batch_graph(r) for i, r in enumerate(reqs) if not r["resident"]}
    xr, ar = synth.rhg(1 << w["resident_log2"], w["resident_deg"], 2.8, w["seed"])
    gen_s = time.perf_counter() - t0
    resident = tp.graph_from_csr(xr, ar).compress()
    res_n, res_m2 = len(xr) - 1, len(ar)
    del xr, ar
    params = tp.default_params(seed=w["seed"])

    def submit(sv, i):
        r = reqs[i]
        if r["resident"]:
            return sv.submit(r["k"], EPS, graph=resident)
        x, a = host[i]
        return sv.submit(r["k"], EPS, xadj=x, adj=a, compress=r["compress"])

    def closed_loop(workers):
        with tp.Server(w["budget"], workers=workers, params=params) as sv:
            t0 = time.perf_counter()
            ts = [submit(sv, i) for i in range(len(reqs))]
            res = [sv.wait(t) for t in ts]
            return time.perf_counter() - t0, res, sv.peak_in_use()

    with tp.Server(w["budget"], workers=4, params=params) as sv:  # warm-up
        for _ in range(args.warmup):
            sv.wait(submit(sv, 0))
            sv.wait(submit(sv, 7))
    cap_s, cap_res, cap_peak = closed_loop(w["workers"])
    plain_s, plain_res, _ = closed_loop(1)
    same = all(np.array_equal(a[0], b[0]) for a, b in zip(cap_res, plain_res))
    rate = w["load"] * len(reqs) / cap_s
    rng = np.random.default_rng(w["seed"])
    runs = []
    for _ in range(max(args.steps, 1)):
        arrivals = np.cumsum(rng.exponential(1.0 / rate, len(reqs)))
        with tp.Server(w["budget"], workers=w["workers"], params=params) as sv:
            t0 = time.perf_counter()
            ts = []
            for i, at in enumerate(arrivals):
                d = at - (time.perf_counter() - t0)
                if d > 0:
                    time.sleep(d)
                ts.append(submit(sv, i))
            infos = [sv.wait(t)[2] for t in ts]
            span = time.perf_counter() - t0
        lat = np.array([f["total_ms"] for f in infos])
        runs.append({"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "mean_ms": float(lat.mean()), "throughput_rps": len(reqs) / span,
                     "queued_p99_ms": float(np.percentile([f["queued_ms"] for f in infos], 99))})
    if rank != 0:
        return
    edges = sum(len(host[i][1]) for i in host) + res_m2 * sum(1 for r in reqs if r["resident"])
    best = min(runs, key=lambda r: r["p99_ms"])
    line = {
        "metric": METRIC, "value": len(reqs) * ws / cap_s, "unit": "requests/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": cap_s * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": w["desc"], "requests": len(reqs), "resident_n": res_n,
                   "resident_m2": res_m2, "workers": w["workers"], "budget_bytes": w["budget"],
                   "timing": "host clock; capacity = all requests submitted at once"},
        "capacity_rps": len(reqs) / cap_s, "plain_single_graph_rps": len(reqs) / plain_s,
        "speedup_vs_plain": plain_s / cap_s, "identical_to_plain": same,
        "edges_per_s_capacity": edges / cap_s, "peak_budget_in_use_bytes": cap_peak,
        "peak_request_bytes": max(r[2]["peak_bytes"] for r in cap_res),
        "reruns_alone": sum(r[2]["retries"] for r in cap_res),
        "largest_request_n": max(len(host[i][0]) - 1 for i in host),
        "poisson": {"rate_rps": rate, **best, "runs": len(runs)},
        "generate_s": gen_s,
    }
    print(json.dumps(line), flush=True)


def run_batch_reference(args, w):
    """The oracle on a bounded sample of the batch: every step partitions the
    next 16 graphs of the recipe on one host thread."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import synth

    recipe = synth.batch_recipe(w["count"], seed=w["seed"])
    per_step = 16
    need = (args.warmup + args.steps) * per_step
    csr = [synth.batch_graph(s) for s in recipe[:need]]
    pos = 0

    def one_step():
        nonlocal pos
        for j in range(per_step):
            xadj, adj = csr[pos + j]
            oracle.partition(oracle.Graph(xadj, adj), recipe[pos + j]["k"], EPS,
                             oracle.Params(seed=w["seed"]))
        pos += per_step

    for _ in range(args.warmup):
        one_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one_step()
    dt = time.perf_counter() - t0
    value = args.steps * per_step / dt
    sample = f"{per_step} graphs of the recipe (in recipe order) per step, one thread"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "graphs/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": w["desc"]},
            "cpu_baseline": {"value": value, "unit": "graphs/s", "cores": 1, "kind": "oracle",
                             "sample": sample, "host": host_cpu()},
            "e2e": {"value": value, "unit": "graphs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_partition_only(args, w):
    """One compressed partition of the workload (for profiler captures)."""
    import torch

    import paper_2410_19119_gb300 as tp

    xadj, adj = make_graph(w)
    z = tp.graph_from_csr(xadj, adj).compress()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, st = tp.partition(z, w["k"], EPS, tp.default_params(seed=w["seed"]))
    torch.cuda.synchronize()
    st["wall_ms"] = (time.perf_counter() - t0) * 1e3
    print(json.dumps({"partition_only": w["desc"], **st}))


def rmat_extra(args, hbm):
    """Config 3 (R-MAT scale 26, k = 256, compressed with chunking) beside the
    headline: level-0 LP GTEPS and partition time over a fixed small count of
    partitions (one warm-up, two timed), and the per-tier rating roofline
    from one more partition with per-launch events."""
    import torch

    import paper_2410_19119_gb300 as tp

    w = WORKLOADS["rmat26"]
    t0 = time.perf_counter()
    xadj, adj = make_graph(w)
    gen_s = time.perf_counter() - t0
    n, m2 = len(xadj) - 1, len(adj)
    g = tp.graph_from_csr(xadj, adj)
    del xadj, adj
    z = g.compress()
    del g
    params = tp.default_params(seed=w["seed"])
    tp.partition(z, w["k"], EPS, params)
    torch.cuda.synchronize()
    runs = []
    for _ in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, st = tp.partition(z, w["k"], EPS, params)
        e1.record()
        torch.cuda.synchronize()
        runs.append((e0.elapsed_time(e1), st))
    tp.profile_read()
    tp.profile_enable(True)
    tp.partition(z, w["k"], EPS, params)
    tp.profile_enable(False)
    prof = tp.profile_read()
    st = runs[-1][1]
    lp_ms = statistics.mean(r[1]["ms_lp_level0"] for r in runs)
    tiers = {}
    for fam, e in prof.items():
        if fam.startswith("rate_") and e["launches"]:
            ms = e["ms"] / e["launches"]
            gbs = e["bytes"] / e["launches"] / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
            tiers[fam] = {"kernel": KERNEL_NAMES[fam], "launches": e["launches"],
                          "ms_total": e["ms"], "ms_per_launch": ms, "achieved_gbs": gbs,
                          "frac": gbs / hbm}
    zi = z.info()
    return {"workload": w["desc"], "n": n, "m2": m2, "compressed_bytes": zi["bytes"],
            "lp_gteps_compressed": 5.0 * m2 / lp_ms / 1e6, "lp_ms_level0": lp_ms,
            "partition_ms_compressed": statistics.mean(r[0] for r in runs),
            "partitions_timed": len(runs), "cut": st["cut"], "imbalance": st["imbalance"],
            "levels": st["levels"], "level_n": st["level_n"], "level_m2": st["level_m2"],
            "peak_bytes": st["peak_bytes"],
            "phase_ms": {"coarsen": st["ms_coarsen"], "initial": st["ms_initial"],
                         "uncoarsen": st["ms_uncoarsen"]},
            "rating_tiers_level0": tiers, "generate_s": gen_s}


def run_native(args, w):
    import torch

    import paper_2410_19119_gb300 as tp

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    dev_index = vis.split(",")[local] if vis and len(vis.split(",")) > local else str(local)
    xadj, adj = make_graph(w)
    n, m2 = len(xadj) - 1, len(adj)
    k = w["k"]
    params = tp.default_params(seed=w["seed"])
    stream = torch.cuda.current_stream()
    g = tp.graph_from_csr(xadj, adj)

    def step():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        z = g.compress()
        ev[1].record(stream)
        _, stz = tp.partition(z, k, EPS, params)
        ev[2].record(stream)
        _, stc = tp.partition(g, k, EPS, params)
        ev[3].record(stream)
        torch.cuda.synchronize()
        zinfo = z.info()
        return {"step_ms": ev[0].elapsed_time(ev[3]), "compress_ms": ev[0].elapsed_time(ev[1]),
                "part_z_ms": ev[1].elapsed_time(ev[2]), "part_c_ms": ev[2].elapsed_time(ev[3]),
                "stz": stz, "stc": stc, "zbytes": zinfo["bytes"], "zstream": zinfo["stream_bytes"],
                "z": z}

    for _ in range(args.warmup):
        step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = tp.launch_count()
    prof = {}
    recs = []
    with ClockSampler(dev_index) as clk:
        # timed steps run exactly what a user call runs (no per-launch events)
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        z = None
        for _ in range(args.steps):
            r = step()
            z = r.pop("z")  # keep only the last compressed graph
            recs.append(r)
        t_end.record(stream)
        torch.cuda.synchronize()
        launches = tp.launch_count() - launches0
        # second timed loop: the same compressed partition with CUDA events
        # around every rating launch of the level-0 clustering rounds (on the
        # launching stream), for the per-kernel roofline
        tp.profile_read()
        for _ in range(args.steps):
            tp.profile_enable(True)
            tp.partition(z, k, EPS, params)
            tp.profile_enable(False)
            for fam, e in tp.profile_read().items():
                acc = prof.setdefault(fam, {"launches": 0, "ms": 0.0, "bytes": 0.0})
                for key in acc:
                    acc[key] += e[key]
    del z
    total_ms = t_start.elapsed_time(t_end)
    rounds = params.cluster_rounds
    lp_edges = rounds * m2 * args.steps
    lp_ms_z = sum(r["stz"]["ms_lp_level0"] for r in recs)
    lp_ms_c = sum(r["stc"]["ms_lp_level0"] for r in recs)
    total_ms, lp_ms_z, lp_ms_c = max_over_ranks([total_ms, lp_ms_z, lp_ms_c], dist, "cuda")
    value = ws * lp_edges / lp_ms_z / 1e6
    gteps_csr = ws * lp_edges / lp_ms_c / 1e6

    # end to end through the public API: host CSR in pinned memory -> device
    # graph -> compress -> partition -> partition read back to the host
    px = torch.from_numpy(xadj).pin_memory()
    pa = torch.from_numpy(adj).pin_memory()
    host_part = torch.empty(n, dtype=torch.int32).pin_memory()
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gh = tp.graph_from_csr(px, pa)
        zh = gh.compress()
        part, _ = tp.partition(zh, k, EPS, params)
        host_part.copy_(part, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        del gh, zh
        if i >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_step = sum(e2e_ms) / len(e2e_ms)
    (e2e_step,) = max_over_ranks([e2e_step], dist, "cuda")
    e2e_value = ws * rounds * m2 / e2e_step / 1e6

    if rank != 0:
        dist.barrier()
        dist.destroy_process_group()
        return
    hbm, peak_kind = peaks()
    r0 = recs[0]
    # dominant rating kernel of the level-0 clustering rounds (by device time)
    rating = {f: e for f, e in prof.items() if f.startswith("rate_") and e["launches"]}
    top = max(rating, key=lambda f: rating[f]["ms"]) if rating else None
    roofline = None
    if top:
        e = rating[top]
        per_launch_bytes = e["bytes"] / e["launches"]
        per_launch_ms = e["ms"] / e["launches"]
        achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
        roofline = {"kernel": KERNEL_NAMES[top] + " (level-0 LP rating, compressed graph)",
                    "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm, "peak_source": peak_kind,
                    "peak_nominal": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                    "traffic": ncu_traffic(top, args.workload),
                    "alg_bytes_per_launch": per_launch_bytes, "launch_ms": per_launch_ms,
                    "launches": e["launches"]}
        try:  # the same rate counted in CSR-equivalent (decoded) bytes
            comp_round = r0["zstream"] + 4.0 * (n + 1) + 4.0 * m2 + 12.0 * n
            csr_round = 8.0 * (n + 1) + 4.0 * m2 + 4.0 * m2 + 12.0 * n
            roofline["decoded_equivalent_gbs"] = achieved * csr_round / comp_round
        except Exception:
            pass
    line = {
        "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": bench_config(w, n, m2, ws),
        "lp_gteps_csr": gteps_csr,
        "lp_ms_level0_compressed": lp_ms_z / args.steps, "lp_ms_level0_csr": lp_ms_c / args.steps,
        "partition_ms_compressed": statistics.mean(r["part_z_ms"] for r in recs),
        "partition_ms_csr": statistics.mean(r["part_c_ms"] for r in recs),
        "partition_ms_compressed_incl_compress": statistics.mean(
            r["part_z_ms"] + r["compress_ms"] for r in recs),
        "compress_ms": statistics.mean(r["compress_ms"] for r in recs),
        "compressed_bytes": r0["zbytes"], "csr_bytes": 8 * (n + 1) + 4 * m2,
        "cut": r0["stz"]["cut"], "cut_csr_path": r0["stc"]["cut"],
        "imbalance": r0["stz"]["imbalance"], "levels": r0["stz"]["levels"],
        "phase_ms_compressed": {"coarsen": r0["stz"]["ms_coarsen"],
                                "initial": r0["stz"]["ms_initial"],
                                "uncoarsen": r0["stz"]["ms_uncoarsen"]},
        "kernel_profile": prof,
        "kernel_profile_timing": "a second loop of --steps compressed partitions with CUDA "
                                 "events around each rating launch of the level-0 clustering",
        "roofline": roofline,
        "clocks": clk.summary(),
        "e2e": {"value": e2e_value, "unit": E2E_UNIT, "definition": E2E_DEF,
                "ms_per_step": e2e_step, "h2d_bytes_per_step": 8 * (n + 1) + 4 * m2,
                "d2h_bytes_per_step": 4 * n},
        "gpu_launches": launches,
    }
    if ws == 1 and w is WORKLOADS["rgg24"] and not args.no_rmat:
        line["rmat26"] = rmat_extra(args, hbm)
    if ws == 1 and not args.no_cpu_baseline:
        v, rounds_done, dt = cpu_oracle_lp(xadj, adj, k, w["seed"])
        line["cpu_baseline"] = {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                                "sample": f"{rounds_done} level-0 LP clustering round(s) of the "
                                          f"full CSR graph in {dt:.1f} s, one thread",
                                "host": host_cpu()}
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="rgg24")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-rmat", action="store_true",
                    help="skip the R-MAT scale 26 keys of the default line")
    ap.add_argument("--lp-only", action="store_true",
                    help="run only the level-0 clustering once (profiler captures)")
    ap.add_argument("--partition-only", action="store_true",
                    help="compress and partition once, print the stats (profiler captures)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if w["gen"] == "serve":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the serving workload's reference arm would be the oracle on "
                              "requests of up to 2^26 vertices and a 2^26-vertex resident graph; "
                              "it is timed on the batch and single-graph workloads instead"}))
        else:
            run_serve(args, w)
    elif w["gen"] == "batch":
        if args.impl == "reference":
            run_batch_reference(args, w)
        elif args.partition_only:
            run_batch_once(args, w)
        else:
            run_batch(args, w)
    elif args.lp_only:
        run_lp_only(args, w)
    elif args.partition_only:
        run_partition_only(args, w)
    elif args.impl == "reference":
        run_reference(args, w)
    else:
        run_native(args, w)


if __name__ == "__main__":
    main()
