#!/usr/bin/env python3
"""Benchmark: node2vec second-order walk throughput on GB300.

Default workload: R-MAT scale 20 (2^20 nodes, 16,777,216 undirected edges, fp32
weights U[0.1, 1]), p = 0.5, q = 2, walk length 100, 10 walks per node
(10,485,760 walks), seed 7.  One step = one grape_walks launch over the whole
job (every row of the output).  The graph is 418 MB and the output 4.2 GB, both
larger than the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the CPU oracle on the host cores
  python bench.py --mode serve ...       # continuous-batching server latency run

With N > 1 (torchrun, one rank per GPU) every rank builds the same graph and
runs its own shard of a job N times as large (walk ids [r*W, (r+1)*W)).
There is no collective on the data path.  The only communication is a barrier
and a max over ranks of the elapsed time.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes
import dataclasses
import hashlib
import glob
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = ("walk steps/sec + HBM sector GB/s vs ~8 TB/s; batched/served vs per-request; "
          "p50/p99")
UNIT = "walk steps/s"
SECTOR = 32


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="rmat20w", choices=["er1k", "rmat20w", "rmat21", "rmat22", "rmat24", "rmat26"])
    ap.add_argument("--mode", choices=["walks", "serve"], default="walks")
    ap.add_argument("--walks-per-node", type=int, default=0,
                    help="override the workload's walks per node (a smaller case of the same "
                         "graph, for profiling); 0 keeps the workload's own")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-contexts", action="store_true")
    ap.add_argument("--no-cumsum", action="store_true",
                    help="skip the cumulative-sum sampler vs rejection comparison")
    ap.add_argument("--no-specialisations", action="store_true",
                    help="skip the timing of the eight p == 1 / q == 1 / weighted variants")
    ap.add_argument("--cumsum-walks", type=int, default=1 << 20,
                    help="starts (one walk each) of the cumulative-sum comparison")
    ap.add_argument("--ef-quanta", default="64,1024",
                    help="Elias-Fano store leg: index quanta to build and walk ('' to skip)")
    ap.add_argument("--suss-k", type=int, default=0,
                    help="also time the workload's approximated walks (SUSS sub-samples of k "
                         "neighbours at nodes of degree above k)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--serve-rates", default="50,200,1000")
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--serve-graph", default="rmat26")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (barrier + max of elapsed times only)
# ---------------------------------------------------------------------------
class Dist:
    def __init__(self, n_gpus):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        if self.world != max(1, n_gpus) and self.world > 1:
            raise SystemExit(f"WORLD_SIZE={self.world} but --gpus {n_gpus}")
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def shard(total_walks: int, world: int, rank: int):
    """Contiguous walk-id shard [begin, end) of rank `rank`."""
    per = -(-total_walks // world)
    b = min(total_walks, rank * per)
    return b, min(total_walks, b + per)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the sources that define the walk kernels' device code and the
    graph layout they read (a profile taken on other sources is stale)."""
    h = hashlib.sha256()
    for name in ("walk_device.cuh", "graph.cu"):
        with open(os.path.join(ROOT, "paper_2110_06196_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", f"walk_kernel_{workload}.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("src_hash") != kernel_source_hash():
        return None
    return d.get("dram_bytes_per_launch")


def count_steps(out: torch.Tensor) -> int:
    """Transitions taken: valid entries minus one start per row with a valid start
    (counted in slices of rows, so no temporary grows with the job)."""
    total = 0
    step = max(1, (1 << 28) // max(1, out.shape[1]))
    for b in range(0, out.shape[0], step):
        part = out[b:b + step]
        total += int((part >= 0).sum(dtype=torch.int64)) - int((part[:, 0] >= 0).sum(dtype=torch.int64))
    return total


def algorithmic_bytes(c: dict, rows: int, walk_len: int) -> int:
    """Sector-granular lower bound on the DRAM bytes of one launch: one 32-byte
    sector per proposal whose entry has to be read (the entry holds the
    candidate, its weight and the candidate's row offset and degree, so an
    accepted step needs nothing more; returns and certain rejections are decided
    without one), one per acceptance-deciding membership test (the least any
    search structure can read), one per walk start (the start's record), plus
    the 4-byte output entries."""
    return SECTOR * (c["gathers"] + c["searches"] + c["walks"]) + 4 * rows * walk_len


def random_sector_peak(dev, gib=16, reads=1 << 31):
    """Calibrated random-sector roofline: useful GB/s of independent random
    32-byte sector reads over a buffer much larger than L2 (grape_sector_probe)."""
    from paper_2110_06196_gb300 import walk as W
    buf = torch.empty(gib << 28, dtype=torch.int32, device=dev)   # gib GiB
    buf.fill_(1)
    W.sector_probe(buf, reads // 8, seed=1)                     # warm-up
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    n = W.sector_probe(buf, reads, seed=2)
    e1.record()
    torch.cuda.synchronize(dev)
    s = e0.elapsed_time(e1) / 1e3
    del buf
    torch.cuda.empty_cache()
    return n * SECTOR / s / 1e9


def workload_desc(name, job):
    from paper_2110_06196_gb300 import synth
    s = synth.WORKLOADS[name]
    if s["kind"] == "er":
        g = f"Erdos-Renyi n={s['n']} m={s['m']} undirected (seed {s['seed']})"
    else:
        g = (f"R-MAT(a=.57,b=.19,c=.19) scale {s['scale']}, {s['m']} undirected edges"
             f"{', fp32 weights U[0.1,1]' if s['weighted'] else ', unweighted'} (seed {s['seed']})")
    return (f"{name}: {g}; node2vec p={job.p} q={job.q} walk_len={job.walk_len} "
            f"walks_per_node={job.walks_per_node} seed={job.seed}")


# ---------------------------------------------------------------------------
# CPU oracle timing (reported baseline; test infrastructure)
# ---------------------------------------------------------------------------
def oracle_rate(csr_np, job, seconds, starts=None):
    import oracle
    og = oracle.Graph(*csr_np)
    threads = os.cpu_count() or 1
    n = og.num_nodes if starts is None else len(starts)
    total = n * job.walks_per_node
    rng = np.random.default_rng(123)
    # calibrate on a small sample, then size the main sample to ~`seconds`
    probe = 64 * threads
    b = int(rng.integers(0, max(1, total - probe)))
    t0 = time.perf_counter()
    rows = oracle.walks_parallel(og, starts, job.walk_len, job.walks_per_node, job.p, job.q,
                                 job.seed, walk_ids=(b, b + probe), threads=threads)
    dt = time.perf_counter() - t0
    per_walk = max(dt / probe, 1e-9)
    count = int(min(total - 1, max(probe, seconds / per_walk)))
    b = int(rng.integers(0, max(1, total - count)))
    t0 = time.perf_counter()
    rows = oracle.walks_parallel(og, starts, job.walk_len, job.walks_per_node, job.p, job.q,
                                 job.seed, walk_ids=(b, b + count), threads=threads)
    dt = time.perf_counter() - t0
    steps = int((rows >= 0).sum()) - int((rows[:, 0] >= 0).sum())
    return steps / dt, threads, f"walk ids [{b}, {b + count}) of {total} ({count} walks, {steps} steps, {dt:.1f} s)"


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, dist):
    from paper_2110_06196_gb300 import BatchPlan, Graph, synth, walks, walks_host
    from paper_2110_06196_gb300 import walk as W
    from paper_2110_06196_gb300 import _lib

    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    spec = synth.WORKLOADS[args.workload]
    job = spec["job"]
    if args.walks_per_node > 0:
        job = dataclasses.replace(job, walks_per_node=args.walks_per_node)
    csr = synth.workload_graph(args.workload, device=dev)
    g = Graph.from_csr(csr, validate=False, device=dev)
    lib = g._lib
    n = csr.num_nodes
    num_entries = csr.num_entries
    # the library holds its own copy of the graph: release the generator's
    # tensors (kept on the host only where the CPU baseline needs them)
    want_cpu = (not args.no_cpu_baseline and dist.rank == 0 and dist.world == 1)
    want_batched = (not args.no_batched and dist.rank == 0 and args.workload == "rmat20w")
    csr_host = csr.numpy() if want_cpu else None
    ef_stores = {}
    if args.ef_quanta and dist.world == 1:
        from paper_2110_06196_gb300 import EFGraph
        for qs in args.ef_quanta.split(","):
            t0 = time.perf_counter()
            ef_stores[int(qs)] = (EFGraph.from_csr(csr, quantum=int(qs), validate=False, device=dev),
                                  time.perf_counter() - t0)
    if not want_batched:
        del csr
        csr = None
    torch.cuda.empty_cache()
    per_rank = n * job.walks_per_node                    # weak scaling: fixed work per GPU
    total = per_rank * dist.world
    wpn_total = job.walks_per_node * dist.world
    b, e = shard(total, dist.world, dist.rank)
    rows = e - b
    out = torch.empty((rows, job.walk_len), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = ctypes.c_void_p(stream.cuda_stream)
    outp = ctypes.c_void_p(out.data_ptr())

    def launch():
        code = lib.grape_walks_range(g.handle, None, n, job.walk_len, wpn_total, job.p, job.q,
                                     job.seed, b, rows, outp, sp)
        _lib.check(code, "grape_walks_range")

    for _ in range(max(args.warmup, 3)):
        launch()
    torch.cuda.synchronize(dev)
    g.stream_status()
    steps_per_launch = count_steps(out)
    # work counters for the byte accounting (one extra, untimed launch)
    g.counters(enable=True)
    launch()
    torch.cuda.synchronize(dev)
    cnt = g.counters()
    g.counters(enable=False)

    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [x.strip() for x in vis.split(",") if x.strip()]
    clocks = Clocks(ids[dist.local] if dist.local < len(ids) else str(dist.local))
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    time.sleep(0.3)                          # let the sampler start
    evs[0].record(stream)
    for k in range(args.steps):
        launch()
        evs[k + 1].record(stream)
    torch.cuda.synchronize(dev)
    dist.barrier()
    clk = clocks.stop()
    ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    elapsed = sum(ms) / 1e3
    elapsed_max = dist.max(elapsed)
    value = steps_per_launch * args.steps * dist.world / elapsed_max
    launch_ms = sum(ms) / len(ms)

    ref_sig = row_signature(out) if ef_stores else None
    approx = None
    if args.suss_k > 0 and dist.world == 1:
        from paper_2110_06196_gb300 import walks_approx
        for _ in range(2):
            walks_approx(g, None, job.walk_len, job.walks_per_node, job.p, job.q, job.seed,
                         suss_k=args.suss_k, out=out)
        torch.cuda.synchronize(dev)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(3):
            walks_approx(g, None, job.walk_len, job.walks_per_node, job.p, job.q, job.seed,
                         suss_k=args.suss_k, out=out)
        a1.record(stream)
        torch.cuda.synchronize(dev)
        ams = a0.elapsed_time(a1) / 3
        asteps = count_steps(out)
        approx = {"suss_k": args.suss_k, "ms_per_launch": ams, "steps_per_s": asteps / ams * 1e3,
                  "exact_ms_per_launch": None}
    del out
    torch.cuda.empty_cache()
    # end to end through the host-buffer entry point: H2D starts, walks, D2H rows
    starts_h = torch.arange(n, dtype=torch.int32).pin_memory()
    shard_starts = None
    e2e_rows = n * job.walks_per_node
    out_h = torch.empty((e2e_rows, job.walk_len), dtype=torch.int32).pin_memory()
    st_ptr = ctypes.c_void_p(starts_h.data_ptr())
    oh_ptr = ctypes.c_void_p(out_h.data_ptr())

    def e2e_step():
        code = lib.grape_walks_host(g.handle, st_ptr, n, job.walk_len, job.walks_per_node, job.p,
                                    job.q, job.seed + dist.rank, oh_ptr, sp)
        _lib.check(code, "grape_walks_host")

    e2e_step()
    e2e_steps = count_steps(torch.from_numpy(out_h.numpy()))
    dist.barrier()
    t0 = time.perf_counter()
    k_e2e = max(1, min(args.steps, 5))
    for _ in range(k_e2e):
        e2e_step()
    e2e_dt = dist.max(time.perf_counter() - t0)
    e2e_value = e2e_steps * k_e2e * dist.world / e2e_dt
    del shard_starts, out_h, starts_h
    ef_res = [bench_ef(st, build_s, job, n, dev, ref_sig, rows, g.info()["device_bytes"])
              for st, build_s in ef_stores.values()]
    for st, _ in ef_stores.values():
        st.close()

    peak, peak_kind = measured_peaks()
    alg = algorithmic_bytes(cnt, rows, job.walk_len)
    achieved = alg / (launch_ms / 1e3) / 1e9
    traffic = profiled_traffic(args.workload)
    rs_peak = random_sector_peak(dev)
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": launch_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded R-MAT / Erdos-Renyi stand-ins for the paper's graphs)",
        "config": {"workload": workload_desc(args.workload, job), "walks_per_gpu": rows,
                   "walk_len": job.walk_len, "steps_per_launch": steps_per_launch,
                   "graph_entries": num_entries,
                   "l2": "inputs larger than L2 (graph arrays and output rows > 129 MB)",
                   "parallelism": f"shards{dist.world}"},
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 4 * e2e_rows * job.walk_len},
        "gpu_launches": args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": f"{peak_kind} copy bandwidth",
                     "algorithmic_bytes_per_launch": alg,
                     "random_sector_peak": rs_peak,
                     "frac_of_random_sector_peak": achieved / rs_peak},
        "counters": {"trials_per_step": cnt["trials"] / max(1, cnt["steps"]),
                     "gathers_per_step": cnt["gathers"] / max(1, cnt["steps"]),
                     "filtered_per_step": cnt["filtered"] / max(1, cnt["steps"]),
                     "searches_per_step": cnt["searches"] / max(1, cnt["steps"]),
                     "probes_per_search": cnt["probes"] / max(1, cnt["searches"]),
                     "fallbacks": cnt["fallbacks"]},
        "clocks": clk,
    }
    if ef_res:
        for r in ef_res:
            r["frac_of_random_sector_peak"] = r["achieved_gbs"] / rs_peak
        res["elias_fano"] = ef_res
    if want_batched:
        res["batched"] = bench_batched(g, csr, dev)
    if approx is not None:
        approx["exact_ms_per_launch"] = launch_ms
        res["approx"] = approx
    if want_batched and not args.no_contexts:
        res["contexts"] = bench_contexts(g, job, n, dev, peak)
    if want_batched and not args.no_specialisations:
        res["specialisations"] = bench_specialisations(g, csr, job, n, dev)
    if want_batched and not args.no_cumsum:
        res["cumsum_sampler"] = bench_cumsum(g, job, n, dev, walks_n=args.cumsum_walks)
    if want_cpu:
        rate, cores, sample = oracle_rate(csr_host, job, args.cpu_seconds)
        res["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": sample}
    return res


def row_signature(out: torch.Tensor) -> tuple:
    """A position-weighted sum of every entry of the rows (int64, wrapping), and
    the number of rows: equal rows give equal signatures."""
    L = out.shape[1]
    wts = (torch.arange(L, device=out.device, dtype=torch.int64) * 2654435761 + 97) % 4294967291
    step = max(1, (1 << 26) // max(1, L))
    acc = torch.zeros((), dtype=torch.int64, device=out.device)
    for b in range(0, out.shape[0], step):
        part = out[b:b + step].to(torch.int64)
        rw = (torch.arange(b, b + part.shape[0], device=out.device, dtype=torch.int64)
              * 40503 + 1)[:, None]
        acc += ((part + 2) * wts[None, :] * rw).sum()
    return int(acc), out.shape[0]


def bench_ef(store, build_s, job, n, dev, ref_sig, rows, csr_bytes, reps=3):
    """The same job walked over the Elias-Fano store (grape_ef_walks): launch
    time, steps/s, the store's size against the CSR engine's graph, sectors
    read per step (counting launch) and the rows checked against the CSR
    engine's rows of the timed run (their row_signature, `ref_sig`)."""
    from paper_2110_06196_gb300 import ef_walks
    info = store.info()
    out = torch.empty((rows, job.walk_len), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def launch():
        ef_walks(store, None, job.walk_len, job.walks_per_node, job.p, job.q, job.seed, out=out)

    launch()
    torch.cuda.synchronize(dev)
    store.stream_status()
    same = row_signature(out) == ref_sig
    steps = count_steps(out)
    store.counters(True)
    launch()
    c = store.counters()
    store.counters(False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        launch()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / reps
    m, u = info["num_entries"], info["universe"]
    ceil_log = 0
    while m and (m << ceil_log) < u:
        ceil_log += 1
    alg = 32 * c["sectors"] + 4 * out.numel()
    del out
    torch.cuda.empty_cache()
    return {"quantum": info["quantum"], "ms_per_launch": ms, "steps_per_s": steps / ms * 1e3,
            "rows_equal_csr_engine": same, "build_s": build_s,
            "low_bits": info["low_bits"], "code_bits": info["code_bits"],
            "structure_bytes": info["structure_bytes"], "device_bytes": info["device_bytes"],
            "csr_engine_graph_bytes": csr_bytes,
            "bits_per_entry": 8 * info["structure_bytes"] / max(1, m),
            "paper_bound_bits_per_entry": 2 + ceil_log,
            "sectors_per_step": c["sectors"] / max(1, c["steps"]),
            "membership_tests_per_step": c["membership_tests"] / max(1, c["steps"]),
            "trials_per_step": c["trials"] / max(1, c["steps"]),
            "algorithmic_bytes_per_launch": alg, "achieved_gbs": alg / ms / 1e6}


def bench_specialisations(g, csr, job, n, dev, walks_n=1 << 20, reps=3):
    """GRAPE's eight node2vec specialisations (p == 1 or not, q == 1 or not,
    weighted or not) on the first walks_n starts of this graph, one walk each of
    the job's length: the weighted graph as built, and the same rows without
    weights.  p = 0.5 and q = 2 stand for p != 1 and q != 1."""
    from paper_2110_06196_gb300 import Graph, walks
    ns = min(n, walks_n)
    gu = Graph(csr.offsets, csr.dsts, None, validate=False, device=dev)
    out = torch.empty((ns, job.walk_len), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    res = []
    for weighted, gg in ((False, gu), (True, g)):
        for (p, q) in [(1.0, 1.0), (0.5, 1.0), (1.0, 2.0), (0.5, 2.0)]:
            walks(gg, None, job.walk_len, 1, p, q, job.seed, num_starts=ns, out=out)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                walks(gg, None, job.walk_len, 1, p, q, job.seed, num_starts=ns, out=out)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / reps
            res.append({"weighted": weighted, "p": p, "q": q, "ms_per_launch": ms,
                        "steps_per_s": count_steps(out) / ms * 1e3})
    gu.close()
    del out
    torch.cuda.empty_cache()
    rates = [r["steps_per_s"] for r in res]
    return {"walks": ns, "variants": res, "fastest_over_slowest": max(rates) / min(rates)}


def bench_cumsum(g, job, n, dev, walks_n=1 << 20, reps=3):
    """The paper's cumulative-sum sampler at every step (grape_walks_cumsum)
    against rejection (grape_walks) on the first walks_n starts, one walk each:
    at the job's (p, q), and at an adversarial p = 1/16, q = 4 where rejection
    accepts few proposals (outward moves at 1/64 of the bound, times w/wmax).
    Each entry: launch ms, steps/s, and rejection's proposals per step."""
    from paper_2110_06196_gb300 import walks, walks_cumsum
    ns = min(n, walks_n)
    out = torch.empty((ns, job.walk_len), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    res = []
    for (p, q) in [(job.p, job.q), (1.0 / 16, 4.0)]:
        entry = {"p": p, "q": q, "walks": ns}
        for name, fn in (("rejection", walks), ("cumsum", walks_cumsum)):
            fn(g, None, job.walk_len, 1, p, q, job.seed, num_starts=ns, out=out)
            torch.cuda.synchronize(dev)
            if name == "rejection":
                g.counters(enable=True)
                fn(g, None, job.walk_len, 1, p, q, job.seed, num_starts=ns, out=out)
                torch.cuda.synchronize(dev)
                c = g.counters()
                g.counters(enable=False)
                entry["rejection_trials_per_step"] = c["trials"] / max(1, c["steps"])
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn(g, None, job.walk_len, 1, p, q, job.seed, num_starts=ns, out=out)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / reps
            steps = count_steps(out)
            entry[name] = {"ms_per_launch": ms, "steps_per_s": steps / ms * 1e3}
        res.append(entry)
    del out
    torch.cuda.empty_cache()
    return res


def bench_contexts(g, job, n, dev, peak, window=5, chunk=1 << 22):
    """The whole job's SkipGram/CBOW context windows (window 5 each side),
    streamed in chunks of walk ids through grape_walk_contexts into one reused
    device buffer (walk rows only in scratch), and the windows kernel alone
    (grape_contexts_from_rows) against the copy peak: it reads 4 B and writes
    8 * window B per walk entry."""
    from paper_2110_06196_gb300 import contexts, contexts_from_rows, walks
    total = n * job.walks_per_node
    L = job.walk_len
    out = torch.empty((chunk, L, 2 * window), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def run_job():
        for b in range(0, total, chunk):
            c = min(chunk, total - b)
            contexts(g, None, L, job.walks_per_node, job.p, job.q, job.seed, window=window,
                     walk_begin=b, walk_count=c, out=out[:c])

    run_job()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run_job()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    last = total - (total - 1) // chunk * chunk
    pairs_last = int((out[:last] >= 0).sum())
    # the windows kernel alone, on one chunk of materialised rows
    rows = walks(g, None, L, job.walks_per_node, job.p, job.q, job.seed, out=None)[:chunk].contiguous()
    contexts_from_rows(rows, window, out=out)
    torch.cuda.synchronize(dev)
    reps = 5
    e0.record(stream)
    for _ in range(reps):
        contexts_from_rows(rows, window, out=out)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    kms = e0.elapsed_time(e1) / reps
    kbytes = rows.numel() * 4 * (1 + 2 * window)
    del rows, out
    torch.cuda.empty_cache()
    entries = total * L * 2 * window
    return {"window": window, "walks": total, "chunk_walks": chunk, "ms": ms,
            "context_entries_per_s": entries / (ms / 1e3),
            "skipgram_pairs_in_last_chunk": pairs_last,
            "windows_kernel": {"ms": kms, "bytes": kbytes, "achieved_gbs": kbytes / kms / 1e6,
                               "peak_gbs": peak, "frac": kbytes / kms / 1e6 / peak}}


def bench_batched(g, csr, dev):
    """512 uneven requests (start counts log-uniform in [1, 1e5], lengths
    uniform in [10, 200], p, q in {0.25..4}, seeds 0..511) on this graph: one
    persistent launch from a CUDA graph vs one grape_walks launch per request."""
    from paper_2110_06196_gb300 import BatchPlan, autotune_batched, synth, walks
    mix = synth.request_mix(csr.num_nodes, 512, gen_seed=1234, max_starts=100_000, len_lo=10,
                            len_hi=200)
    reqs = [dict(starts=torch.from_numpy(r.starts).to(dev), walk_len=r.walk_len, walks_per_node=1,
                 p=r.p, q=r.q, seed=r.seed) for r in mix]
    sample = [reqs[j] for j in range(0, 512, 4)]
    best = autotune_batched(g, [dict(x) for x in sample])
    plan = BatchPlan(g, reqs)
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):
        plan.launch()
    torch.cuda.synchronize(dev)
    steps = sum(count_steps(o) for o in plan.outputs())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record(stream)
    for _ in range(reps):
        plan.launch()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_batch = e0.elapsed_time(e1) / reps / 1e3
    outs = [r["out"] for r in reqs]
    for r, o in zip(reqs, outs):                       # warm the per-call path
        walks(g, r["starts"], r["walk_len"], 1, r["p"], r["q"], r["seed"], out=o)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(reps):
        for r, o in zip(reqs, outs):
            walks(g, r["starts"], r["walk_len"], 1, r["p"], r["q"], r["seed"], out=o)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_seq = e0.elapsed_time(e1) / reps / 1e3
    plan.close()
    return {"value": steps / t_batch, "unit": UNIT, "sequential_value": steps / t_seq,
            "speedup_vs_per_request": t_seq / t_batch, "requests": 512, "steps": steps,
            "ms_batched": t_batch * 1e3, "ms_sequential": t_seq * 1e3,
            "tuning": {"chunk_walks": best["chunk_walks"],
                       "shorter_min": best["shorter_min"]}}


# ---------------------------------------------------------------------------
# serving run
# ---------------------------------------------------------------------------
def run_serve(args, dist):
    from paper_2110_06196_gb300 import Graph, Server, synth
    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    csr = synth.workload_graph(args.serve_graph, device=dev)
    g = Graph.from_csr(csr, validate=False, device=dev)
    del csr
    torch.cuda.empty_cache()
    n = g.num_nodes
    results = []
    for ri, rate in enumerate(float(x) for x in args.serve_rates.split(",")):
        mix = synth.request_mix(n, args.serve_requests, gen_seed=77 + ri, max_starts=1_000_000,
                                len_lo=20, len_hi=120, first_seed=10_000 * ri)
        arrivals = synth.poisson_arrivals(rate, len(mix), seed=5 + ri)
        srv = Server(g, output_cap_bytes=40 << 30, max_inflight=4096, chunk_walks=0,
                     max_chunks=1 << 24, idle_exit_us=2000)
        outs = [torch.empty((len(r.starts), r.walk_len), dtype=torch.int32).pin_memory()
                for r in mix]
        lat = []
        done_steps = 0
        import threading
        stop = threading.Event()

        def collect():
            nonlocal done_steps
            while len(lat) < len(mix):
                t, l, rows = srv.wait_any(timeout_ms=600_000)
                lat.append(l)
                r = rows
                done_steps += int((r >= 0).sum()) - int((r[:, 0] >= 0).sum())

        th = threading.Thread(target=collect)
        th.start()
        t0 = time.perf_counter()
        for j, r in enumerate(mix):
            delay = arrivals[j] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            srv.submit(r.starts, r.walk_len, r.p, r.q, r.seed, out=outs[j])
        th.join()
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        lat_ms = np.array(lat) * 1e3
        results.append({"rate_req_s": rate, "requests": len(mix), "steps_per_s": done_steps / wall,
                        "p50_ms": float(np.percentile(lat_ms, 50)),
                        "p99_ms": float(np.percentile(lat_ms, 99)),
                        "max_ms": float(lat_ms.max()), "wall_s": wall,
                        "kernel_launches": st["kernel_launches"]})
    # Saturation: every request of one mix at once, through the server, then
    # the same requests as one grape_walks_host launch each, one after another.
    from paper_2110_06196_gb300 import walks_host
    mix = synth.request_mix(n, args.serve_requests, gen_seed=99, max_starts=1_000_000,
                            len_lo=20, len_hi=120, first_seed=90_000)
    outs = [torch.empty((len(r.starts), r.walk_len), dtype=torch.int32).pin_memory() for r in mix]
    srv = Server(g, output_cap_bytes=40 << 30, max_inflight=4096, chunk_walks=0,
                 max_chunks=1 << 24, idle_exit_us=2000)
    t0 = time.perf_counter()
    tickets = [srv.submit(r.starts, r.walk_len, r.p, r.q, r.seed, out=o) for r, o in zip(mix, outs)]
    lat = []
    for _ in tickets:
        _, l, _ = srv.wait_any(timeout_ms=600_000)
        lat.append(l)
    t_srv = time.perf_counter() - t0
    srv.close()
    steps = sum(int((o >= 0).sum()) - int((o[:, 0] >= 0).sum()) for o in outs)
    seq_outs = [torch.empty_like(o).pin_memory() for o in outs]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for r, o in zip(mix, seq_outs):
        walks_host(g, r.starts, r.walk_len, 1, r.p, r.q, r.seed, out=o)
    t_seq = time.perf_counter() - t0
    same = all(torch.equal(a, b) for a, b in zip(outs, seq_outs))
    lat_ms = np.array(lat) * 1e3
    saturation = {"requests": len(mix), "steps": steps, "served_steps_per_s": steps / t_srv,
                  "sequential_steps_per_s": steps / t_seq,
                  "served_vs_one_launch_per_request": t_seq / t_srv,
                  "p50_ms": float(np.percentile(lat_ms, 50)),
                  "p99_ms": float(np.percentile(lat_ms, 99)),
                  "rows_identical_to_one_launch_per_request": bool(same)}
    best = max(max(r["steps_per_s"] for r in results), saturation["served_steps_per_s"])
    return {"metric": METRIC, "value": best, "unit": UNIT, "n_gpus": 1, "steps": len(results),
            "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"serving on {args.serve_graph}: Poisson arrivals, starts "
                                   "log-uniform [1,1e6], len U[20,120], p,q in {0.25..4}, "
                                   "admission under a 40 GB output cap"},
            "serving": results, "saturation": saturation}


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands, on the host cores
# ---------------------------------------------------------------------------
def run_reference(args, dist):
    if dist.rank != 0:
        return None
    from paper_2110_06196_gb300 import synth
    job = synth.WORKLOADS[args.workload]["job"]
    csr = synth.workload_graph(args.workload, device="cpu")
    csr_np = csr.numpy()
    seconds = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    rates, sample = [], None
    for k in range(args.warmup + args.steps):
        rate, cores, sample = oracle_rate(csr_np, job, seconds)
        if k >= args.warmup:
            rates.append(rate)
    value = statistics.median(rates)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": workload_desc(args.workload, job)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    dist = Dist(args.gpus)
    try:
        if args.impl == "reference":
            res = run_reference(args, dist)
        elif args.mode == "serve":
            res = run_serve(args, dist) if dist.rank == 0 else None
        else:
            res = run_ours(args, dist)
        if dist.rank == 0 and res is not None:
            print(json.dumps(res), flush=True)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
