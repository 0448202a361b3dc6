#!/usr/bin/env python3
"""Benchmark: node2vec second-order walk throughput on GB300.

Headline workload: R-MAT scale 24 (2^24 nodes, 268,435,456 undirected edges,
unweighted, max degree ~1e5), p = 1, q = 0.25, walk length 80, 10 walks per
node (167,772,160 walks, 7.06 G steps), seed 11.  One step = one grape_walks
launch over the whole job (every row of the output).  The graph (19.6 GB) and
the output (53.7 GB) are both far larger than the 129 MB L2, so no flush is
needed between steps.

Beside the headline, rank 0 of a one-GPU run also reports: the random-sector
ceiling (a sweep of the gather probe), the CPU oracle on the host cores (all
cores and one thread), the weighted R-MAT scale-20 job (per call, batched 512
requests, context windows, the eight specialisations, the paper's cumulative
-sum sampler, the Elias-Fano store), and continuous-batching serving on the
R-MAT scale-26 graph (2^30 undirected edges) under Poisson arrivals.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the CPU oracle on the host cores

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

T0 = time.perf_counter()


def log(msg):
    """Progress on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.perf_counter() - T0:7.1f} s] {msg}", file=sys.stderr, flush=True)


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
    ap.add_argument("--workload", default="rmat24", choices=["er1k", "rmat20w", "rmat21", "rmat22", "rmat24", "rmat26"])
    ap.add_argument("--extras-workload", default="rmat20w",
                    help="graph of the batched / contexts / specialisations / cumulative-sum / "
                         "Elias-Fano legs ('' to skip them)")
    ap.add_argument("--walks-per-node", type=int, default=0,
                    help="override the workload's walks per node (a smaller case of the same "
                         "graph, for profiling); 0 keeps the workload's own")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-hub-ab", action="store_true",
                    help="skip the membership-search schedule comparison")
    ap.add_argument("--probe-buffer-sweep", action="store_true",
                    help="run only the random-sector probe over buffers of 32 MB to 64 GB "
                         "and print its table")
    ap.add_argument("--no-probe-sweep", action="store_true",
                    help="time only the probe's default shape instead of sweeping it")
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
    ap.add_argument("--cpu-single-seconds", type=float, default=8.0)
    ap.add_argument("--serve-rates", default="50,200,1000")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-max-s", type=float, default=120.0,
                    help="a rate's arrivals stop after this many seconds")
    ap.add_argument("--serve-saturation", type=int, default=400,
                    help="requests submitted at once for the served-vs-per-request ratio")
    ap.add_argument("--serve-graph", default="rmat26")
    ap.add_argument("--serve-warm-requests", type=int, default=500,
                    help="requests of the lowest rate served again with the kernel kept warm")
    ap.add_argument("--serve-host-gib", type=int, default=16,
                    help="pinned host arena for served rows (GiB)")
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


def sector_minimal_bytes(c: dict, rows: int, walk_len: int) -> int:
    """Sector-granular lower bound on the DRAM bytes of one launch of this
    engine: one 32-byte sector per proposal whose entry has to be read (the
    entry holds the candidate, its weight and the candidate's row offset and
    degree, so an accepted step needs nothing more; returns and certain
    rejections are decided without one), one per acceptance-deciding membership
    test (the least any search structure can read), one per walk start (the
    start's record), plus the 4-byte output entries."""
    return SECTOR * (c["gathers"] + c["searches"] + c["walks"]) + 4 * rows * walk_len


def model_bytes(c: dict, weighted: bool) -> int:
    """The per-step byte model of the method: every transition reads the
    32-byte sector of the next node's offsets and writes its 4-byte output
    entry (36 B); every proposal reads its 32-byte candidate sector, plus a
    32-byte weight sector on a weighted graph; every membership-search probe
    reads one 32-byte sector.  36 + E (32 + 32 [weighted]) + 32 S per step,
    with E proposals and S probes per step taken from the counting launch."""
    return 36 * c["steps"] + SECTOR * (2 if weighted else 1) * c["trials"] + SECTOR * c["probes"]


def random_sectors(c: dict) -> int:
    """Independent random 32-byte sectors one launch reads: the proposal
    entries read, the membership probes and the walk starts' records."""
    return c["gathers"] + c["probes"] + c["walks"]


PROBE_SHAPES = [(w, l) for w, ls in ((4, (8, 16, 32, 64)), (16, (8, 16, 32)), (32, (4, 8, 16)))
                for l in ls]


def random_sector_peak(dev, gib=16, reads=1 << 29, sweep=True):
    """The random-sector ceiling: independent random 32-byte sector reads over
    a buffer far larger than L2 (grape_sector_probe), timed with CUDA events
    over a sweep of load width, loads in flight per thread, resident blocks
    per SM and cache path.  Returns (best sectors/s, best shape, the sweep)."""
    from paper_2110_06196_gb300 import walk as W
    buf = torch.empty(gib << 28, dtype=torch.int32, device=dev)   # gib GiB
    buf.fill_(1)
    stream = torch.cuda.current_stream(dev)
    shapes = []
    if sweep:
        for mode in (0, 1, 2):
            for (w, l) in PROBE_SHAPES:
                for bps in (2, 4, 8):
                    shapes.append((mode, w, l, bps))
    else:
        shapes = [(0, 32, 8, 0)]
    W.sector_probe(buf, reads // 4, seed=1)                         # warm-up
    rows = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for (mode, w, l, bps) in shapes:
        torch.cuda.synchronize(dev)
        e0.record(stream)
        n, res = W.sector_probe(buf, reads, seed=2, mode=mode, load_bytes=w, loads_in_flight=l,
                                blocks_per_sm=bps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        rows.append({"mode": ["nc", "cg", "cs"][mode], "load_bytes": w, "loads_in_flight": l,
                     "blocks_per_sm": res, "threads_per_sm": 256 * res,
                     "sectors_per_s": n / ms * 1e3, "gbs": n * SECTOR / ms / 1e6})
    del buf
    torch.cuda.empty_cache()
    best = max(rows, key=lambda r: r["sectors_per_s"])
    return best["sectors_per_s"], best, rows


def probe_buffer_sweep(dev, reads=1 << 29):
    """The random-sector probe (grape_sector_probe) over buffers from 32 MB to
    64 GB, for three shapes: 32-byte loads 8 in flight (.nc), 4-byte loads 32
    in flight (.cs), and both sectors of a random 64-byte block 4 in flight
    (.nc; counted as two sectors).  Where the rate stops falling with the
    buffer size is where L2 stops helping.  Returns sectors/s per size and shape."""
    from paper_2110_06196_gb300 import walk as W
    shapes = (("32B x8 nc", 0, 32, 8), ("4B x32 cs", 2, 4, 32), ("64B block x4 nc", 0, 64, 4))
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows = []
    for mb in (32, 96, 256, 1024, 4096, 16384, 65536):
        buf = torch.empty(mb << 18, dtype=torch.int32, device=dev)     # mb MiB
        buf.fill_(1)
        row = {"buffer_mib": mb}
        for name, mode, w, l in shapes:
            W.sector_probe(buf, reads // 8, seed=1, mode=mode, load_bytes=w, loads_in_flight=l)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            n, _ = W.sector_probe(buf, reads, seed=2, mode=mode, load_bytes=w, loads_in_flight=l)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            row[name] = n / e0.elapsed_time(e1) * 1e3
        rows.append(row)
        del buf
        torch.cuda.empty_cache()
    return {"probe_buffer_sweep": rows, "unit": "32-byte sectors/s", "reads_per_shape": reads}


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
def oracle_rate(csr_np, job, seconds, starts=None, threads=None):
    """The oracle as it stands (walks_parallel, one contiguous walk-id range per
    thread; threads=1 is the plain single-threaded walker) on a random sample of
    the job's walk ids sized to about `seconds` of work."""
    import oracle
    og = oracle.Graph(*csr_np)
    threads = threads or os.cpu_count() or 1
    n = og.num_nodes if starts is None else len(starts)
    total = n * job.walks_per_node
    rng = np.random.default_rng(123)
    # calibrate on a small sample, then size the main sample to ~`seconds`
    probe = 64 * threads if threads > 1 else 256
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
def job_steps(degrees: torch.Tensor, job) -> int:
    """Transitions of a whole-graph job on an undirected graph: a walk leaves
    its start unless the start is isolated, and then never meets a dead end
    (every node it reaches has the edge it came by), so each walk from a
    non-isolated start takes walk_len - 1 transitions."""
    return int((degrees > 0).sum()) * job.walks_per_node * (job.walk_len - 1)


def time_launches(g, job, n, b, rows, wpn_total, dev, steps, warmup, dist=None, clocks=None):
    """grape_walks_range over walk ids [b, b + rows) of the job: `warmup`
    untimed launches, one counting launch (work counters), then `steps` timed
    launches with a CUDA event after each on the launching stream, bracketed by
    a barrier and a device synchronisation.  Returns the per-launch times, the
    steps of one launch, the counters and the clock record."""
    from paper_2110_06196_gb300 import _lib
    lib = g._lib
    out = torch.empty((rows, job.walk_len), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = ctypes.c_void_p(stream.cuda_stream)
    outp = ctypes.c_void_p(out.data_ptr())

    def launch():
        code = lib.grape_walks_range(g.handle, None, n, job.walk_len, wpn_total, job.p, job.q,
                                     job.seed, b, rows, outp, sp)
        _lib.check(code, "grape_walks_range")

    for _ in range(warmup):
        launch()
    torch.cuda.synchronize(dev)
    g.stream_status()
    steps_per_launch = count_steps(out)
    g.counters(enable=True)
    launch()
    torch.cuda.synchronize(dev)
    cnt = g.counters()
    g.counters(enable=False)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    if clocks:
        clocks.start()
        time.sleep(0.3)                      # let the sampler start
    evs[0].record(stream)
    for k in range(steps):
        launch()
        evs[k + 1].record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]
    return ms, steps_per_launch, cnt, clk, out


def e2e_buffers(n, job):
    """Pinned host starts (0..n-1) and rows for the end-to-end calls,
    allocated before the device timing, as a user allocates them once and
    reuses them."""
    rows = n * job.walks_per_node
    starts_h = host_rows(n)
    starts_h.copy_(torch.arange(n, dtype=torch.int32))
    return starts_h, host_rows(rows * job.walk_len).view(rows, job.walk_len)


def e2e_rate(g, job, n, steps_per_job, dist, k, bufs=None):
    """The same job end to end through grape_walks_host, the call a user with
    host buffers makes: the starts go in from pinned host memory and the rows
    come back into pinned host memory inside every timed call.  Two untimed calls, then k timed ones.  Returns
    (steps/s, H2D bytes, D2H bytes per call)."""
    from paper_2110_06196_gb300 import _lib
    lib = g._lib
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    rows = n * job.walks_per_node
    starts_h, out_h = bufs if bufs is not None else e2e_buffers(n, job)
    st_ptr = ctypes.c_void_p(starts_h.data_ptr())
    oh_ptr = ctypes.c_void_p(out_h.data_ptr())

    def call():
        code = lib.grape_walks_host(g.handle, st_ptr, n, job.walk_len, job.walks_per_node, job.p,
                                    job.q, job.seed + dist.rank, oh_ptr, sp)
        _lib.check(code, "grape_walks_host")

    call()
    call()
    dist.barrier()
    t0 = time.perf_counter()
    for _ in range(k):
        call()
    dt = dist.max(time.perf_counter() - t0)
    h2d, d2h = 4 * n, 4 * rows * job.walk_len
    del starts_h, out_h, bufs
    from paper_2110_06196_gb300 import walk as W
    W.trim_scratch(0)                        # the call's pooled device scratch goes back
    return steps_per_job * k * dist.world / dt, h2d, d2h


def roofline(cnt, rows, walk_len, weighted, launch_ms, peak, peak_kind, traffic, rs):
    """The dominant kernel against the measured copy peak, under the method's
    per-step byte model and under this engine's sector-granular minimum, and
    its random sectors against the measured random-sector ceiling `rs`
    (sectors/s, or None)."""
    s = launch_ms / 1e3
    mb = model_bytes(cnt, weighted)
    sm = sector_minimal_bytes(cnt, rows, walk_len)
    rsec = random_sectors(cnt)
    steps = max(1, cnt["steps"])
    r = {"bound": "hbm", "achieved": mb / s / 1e9, "peak": peak, "unit": "GB/s",
         "frac": mb / s / 1e9 / peak, "traffic": traffic,
         "peak_kind": f"{peak_kind} copy bandwidth",
         "bytes_model": "per step 36 B (offsets sector + output entry) + per proposal 32 B "
                        "(+32 B weights) + 32 B per search probe",
         "algorithmic_bytes_per_launch": mb, "bytes_per_step": mb / steps,
         "sector_minimal": {"bytes_per_launch": sm, "bytes_per_step": sm / steps,
                            "achieved": sm / s / 1e9, "frac": sm / s / 1e9 / peak},
         "random_sectors_per_launch": rsec, "random_sectors_per_step": rsec / steps,
         "random_sectors_per_s": rsec / s}
    if rs:
        r["random_sector_peak_sectors_per_s"] = rs
        r["random_sector_peak_gbs"] = rs * SECTOR / 1e9
        r["frac_of_random_sector_peak"] = rsec / s / rs
    if traffic:
        r["traffic_over_model_bytes"] = traffic / mb
    return r


def counters_view(cnt):
    st = max(1, cnt["steps"])
    return {"trials_per_step": cnt["trials"] / st, "gathers_per_step": cnt["gathers"] / st,
            "filtered_per_step": cnt["filtered"] / st,
            "searches_per_step": cnt["searches"] / st,
            "probes_per_search": cnt["probes"] / max(1, cnt["searches"]),
            "probes_per_step": cnt["probes"] / st,
            "hash_probes_per_step": cnt.get("hash_probes", 0) / st, "fallbacks": cnt["fallbacks"]}


def run_ours(args, dist):
    from paper_2110_06196_gb300 import Graph, synth

    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    solo = dist.rank == 0 and dist.world == 1
    spec = synth.WORKLOADS[args.workload]
    job = spec["job"]
    if args.walks_per_node > 0:
        job = dataclasses.replace(job, walks_per_node=args.walks_per_node)
    log(f"building {args.workload}")
    csr = synth.workload_graph(args.workload, device=dev)
    g = Graph.from_csr(csr, validate=False, device=dev)
    n = csr.num_nodes
    num_entries = csr.num_entries
    degrees = csr.degrees()
    log("graph resident; timing walks")
    e2e_bufs = e2e_buffers(n, job)
    want_cpu = not args.no_cpu_baseline and solo
    csr_host = csr.numpy() if want_cpu else None
    # the library holds its own copy of the graph
    del csr
    torch.cuda.empty_cache()
    per_rank = n * job.walks_per_node                    # weak scaling: fixed work per GPU
    total = per_rank * dist.world
    wpn_total = job.walks_per_node * dist.world
    b, e = shard(total, dist.world, dist.rank)
    rows = e - b
    warm = max(args.warmup, 3)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [x.strip() for x in vis.split(",") if x.strip()]
    clocks = Clocks(ids[dist.local] if dist.local < len(ids) else str(dist.local))
    ms, steps_per_launch, cnt, clk, out = time_launches(g, job, n, b, rows, wpn_total, dev,
                                                        args.steps, warm, dist, clocks)
    elapsed_max = dist.max(sum(ms) / 1e3)
    value = steps_per_launch * args.steps * dist.world / elapsed_max
    launch_ms = sum(ms) / len(ms)
    ref_sig = row_signature(out) if (args.ef_quanta and solo) else None
    hub = None
    if solo and not args.no_hub_ab:
        log("membership-search schedules")
        hub = bench_hub_schedules(g, job, n, rows, out, dev, launch_ms)
    approx = None
    if args.suss_k > 0 and solo:
        approx = bench_approx(g, job, out, dev, args.suss_k, launch_ms)
    del out
    torch.cuda.empty_cache()
    if spec["kind"] != "er" and dist.world == 1:
        assert steps_per_launch == job_steps(degrees, job), "rows do not have the job's steps"
    log(f"walks {launch_ms:.1f} ms per launch; end to end")
    e2e_value, h2d, d2h = e2e_rate(g, job, n, steps_per_launch, dist, max(1, min(args.steps, 5)),
                                   e2e_bufs)
    del e2e_bufs
    log(f"end to end {e2e_value / 1e9:.2f} G steps/s; random-sector probe")
    peak, peak_kind = measured_peaks()
    rs, rs_best, rs_sweep = (None, None, None)
    if dist.rank == 0:
        rs, rs_best, rs_sweep = random_sector_peak(dev, sweep=not args.no_probe_sweep)
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world,
        "steps": args.steps, "warmup": warm, "ms_per_step": launch_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded R-MAT / Erdos-Renyi stand-ins for the paper's graphs)",
        "config": config_of(args.workload, job, rows, steps_per_launch, num_entries, dist.world),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "call": "grape_walks_host (pinned host starts and rows)",
                "frac_of_device_value": e2e_value / value},
        "gpu_launches": args.steps,
        "roofline": roofline(cnt, rows, job.walk_len, spec.get("weighted", False), launch_ms,
                             peak, peak_kind, profiled_traffic(args.workload), rs),
        "counters": counters_view(cnt),
        "clocks": clk,
    }
    if rs_sweep:
        res["random_sector_probe"] = {"best": rs_best, "sweep": rs_sweep,
                                      "buffer": "16 GiB, 2^29 reads per shape"}
    if approx is not None:
        res["approx"] = approx
    if hub is not None:
        res["hub_schedule"] = hub
    if ref_sig is not None and args.ef_quanta:
        log("Elias-Fano stores")
        res["elias_fano"] = bench_ef_stores(args, g, job, n, dev, ref_sig, rows, rs)
    if want_cpu:
        log("CPU oracle")
        rate, cores, sample = oracle_rate(csr_host, job, args.cpu_seconds)
        rate1, _, sample1 = oracle_rate(csr_host, job, args.cpu_single_seconds, threads=1)
        res["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": sample,
                               "single_thread": {"value": rate1, "cores": 1, "sample": sample1}}
        del csr_host
    g.close()
    del g
    torch.cuda.empty_cache()
    if solo and args.extras_workload:
        log(f"{args.extras_workload} legs")
        res[args.extras_workload] = extras(args, dev, peak, peak_kind, rs)
    if solo and not args.no_serve:
        log("serving")
        res["served"] = bench_serve(args, dev)
    log("done")
    return res


def config_of(workload, job, rows, steps_per_launch, num_entries, world):
    return {"workload": workload_desc(workload, job), "walks_per_gpu": rows,
            "walk_len": job.walk_len, "steps_per_launch": steps_per_launch,
            "graph_entries": num_entries,
            "l2": "inputs larger than L2 (graph arrays and output rows > 129 MB)",
            "parallelism": f"shards{world}"}


def bench_hub_schedules(g, job, n, rows, out, dev, plain_ms, reps=3):
    """The headline job under each membership-search schedule (the graph's
    tuning knobs): the edge hash (default); the sorted-row search alone; with
    sector pivots from a list length on, with an L2 persisting window over the
    pivots, and with warp-cooperative narrowing of long lists.  Launch time
    (CUDA events), probes per step (counting launch), and the rows' signature
    against the default schedule's."""
    INT = 0x7fffffff
    base = g.get_tuning().as_dict()
    stream = torch.cuda.current_stream(dev)
    ref = row_signature(out)
    res = [{"schedule": "edge hash, one bucket per membership test (default)",
            "ms_per_launch": plain_ms}]
    variants = [("sorted-row search, per-lane interpolation", dict(edge_hash=0)),
                ("sorted rows + sector pivots, lists >= 512", dict(edge_hash=0, pivot_min=512)),
                ("sorted rows + sector pivots >= 128 + 96 MB L2 persisting window on them",
                 dict(edge_hash=0, pivot_min=128, l2_persist_mb=96)),
                ("sorted rows + warp-cooperative narrowing, lists > 8192",
                 dict(edge_hash=0, warp_search_min=8192)),
                ("sorted rows + warp-cooperative narrowing, lists > 1024",
                 dict(edge_hash=0, warp_search_min=1024))]
    for name, kw in variants:
        t = dict(base)
        t.update(kw)
        g.set_tuning(**t)
        walks_into(g, job, n, rows, out)
        torch.cuda.synchronize(dev)
        same = row_signature(out) == ref
        g.counters(enable=True)
        walks_into(g, job, n, rows, out)
        torch.cuda.synchronize(dev)
        c = g.counters()
        g.counters(enable=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            walks_into(g, job, n, rows, out)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        st = max(1, c["steps"])
        res.append({"schedule": name, "tuning": kw, "ms_per_launch": e0.elapsed_time(e1) / reps,
                    "rows_equal_default": same, "probes_per_step": c["probes"] / st,
                    "pivot_probes_per_step": c["pivot_probes"] / st,
                    "hash_probes_per_step": c["hash_probes"] / st})
    base.update(l2_persist_mb=0)
    g.set_tuning(**base)
    return res


def walks_into(g, job, n, rows, out):
    from paper_2110_06196_gb300 import _lib
    code = g._lib.grape_walks_range(g.handle, None, n, job.walk_len, job.walks_per_node, job.p,
                                    job.q, job.seed, 0, rows, ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check(code, "grape_walks_range")


def bench_approx(g, job, out, dev, suss_k, exact_ms):
    """The workload's approximated walks (SUSS sub-samples of k neighbours)."""
    from paper_2110_06196_gb300 import walks_approx
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):
        walks_approx(g, None, job.walk_len, job.walks_per_node, job.p, job.q, job.seed,
                     suss_k=suss_k, out=out)
    torch.cuda.synchronize(dev)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(3):
        walks_approx(g, None, job.walk_len, job.walks_per_node, job.p, job.q, job.seed,
                     suss_k=suss_k, out=out)
    a1.record(stream)
    torch.cuda.synchronize(dev)
    ams = a0.elapsed_time(a1) / 3
    return {"suss_k": suss_k, "ms_per_launch": ams, "steps_per_s": count_steps(out) / ams * 1e3,
            "exact_ms_per_launch": exact_ms}


def bench_ef_stores(args, g, job, n, dev, ref_sig, rows, rs):
    """The headline job over the Elias-Fano store at each index quantum."""
    from paper_2110_06196_gb300 import EFGraph, synth
    csr = synth.workload_graph(args.workload, device=dev)
    res = []
    for qs in args.ef_quanta.split(","):
        t0 = time.perf_counter()
        st = EFGraph.from_csr(csr, quantum=int(qs), validate=False, device=dev)
        build_s = time.perf_counter() - t0
        r = bench_ef(st, build_s, job, n, dev, ref_sig, rows, g.info()["device_bytes"])
        if rs:
            r["frac_of_random_sector_peak"] = r["sectors_per_s"] / rs
        st.close()
        res.append(r)
    del csr
    torch.cuda.empty_cache()
    return res


def extras(args, dev, peak, peak_kind, rs):
    """The weighted R-MAT scale-20 job (per call and end to end) and the legs
    that run on its graph: batched requests, context windows, the eight
    specialisations, the paper's cumulative-sum sampler."""
    from paper_2110_06196_gb300 import Graph, synth

    class _Solo:
        world, rank = 1, 0

        def barrier(self):
            pass

        def max(self, x):
            return x

    wl = args.extras_workload
    spec = synth.WORKLOADS[wl]
    job = spec["job"]
    csr = synth.workload_graph(wl, device=dev)
    g = Graph.from_csr(csr, validate=False, device=dev)
    n = csr.num_nodes
    rows = n * job.walks_per_node
    ms, steps, cnt, _, out = time_launches(g, job, n, 0, rows, job.walks_per_node, dev, 10, 3)
    launch_ms = sum(ms) / len(ms)
    del out
    torch.cuda.empty_cache()
    e2e_value, _, _ = e2e_rate(g, job, n, steps, _Solo(), 3)
    res = {"workload": workload_desc(wl, job), "value": steps / (launch_ms / 1e3),
           "ms_per_launch": launch_ms, "steps_per_launch": steps,
           "e2e": {"value": e2e_value, "unit": UNIT},
           "roofline": roofline(cnt, rows, job.walk_len, spec.get("weighted", False), launch_ms,
                                peak, peak_kind, profiled_traffic(wl), rs),
           "counters": counters_view(cnt)}
    log("batched")
    if not args.no_batched:
        res["batched"] = bench_batched(g, csr, dev)
    log("contexts, specialisations, cumulative sums")
    if not args.no_contexts:
        res["contexts"] = bench_contexts(g, job, n, dev, peak)
    if not args.no_specialisations:
        res["specialisations"] = bench_specialisations(g, csr, job, n, dev)
    if not args.no_cumsum:
        res["cumsum_sampler"] = bench_cumsum(g, job, n, dev, walks_n=args.cumsum_walks)
    g.close()
    del g, csr
    torch.cuda.empty_cache()
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
            "algorithmic_bytes_per_launch": alg, "achieved_gbs": alg / ms / 1e6,
            "sectors_per_s": c["sectors"] / ms * 1e3}


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
# serving
# ---------------------------------------------------------------------------
def host_rows(elems, pin=True):
    """int32 host buffer: page-locked (pinned) when pin, so that the copy
    engines write it directly; pageable otherwise."""
    return torch.empty(elems, dtype=torch.int32, pin_memory=pin)


class PinnedArena:
    """Served rows land in one page-locked host arena allocated before the
    arrivals start (page-locking during the run can stall the device), carved
    first-fit into per-request slices and given back once a request's rows
    are counted.  Should the arena be full, a request gets a buffer of its own."""

    def __init__(self, elems, pin=True):
        self.pin = pin
        self.buf = host_rows(elems, pin)
        self.free = [(0, elems)]                 # sorted (offset, length)
        self.extra = 0

    def take(self, elems):
        elems = (elems + 63) // 64 * 64
        for i, (o, n) in enumerate(self.free):
            if n >= elems:
                self.free[i:i + 1] = [(o + elems, n - elems)] if n > elems else []
                return ("arena", o, elems), self.buf[o:o + elems]
        self.extra += 1
        return ("own", 0, elems), host_rows(elems, self.pin)

    def give(self, key):
        kind, o, n = key
        if kind != "arena":
            return
        self.free.append((o, n))
        self.free.sort()
        merged = []
        for a, m in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + m)
            else:
                merged.append((a, m))
        self.free = merged


def bench_serve(args, dev):
    """Continuous batching on the resident R-MAT scale-26 graph: Poisson
    arrivals at each rate (args.serve_requests requests, or args.serve_max_s
    seconds of arrivals), latency from submit to rows in host memory, and the
    server's device-counted transitions per second of wall time.  Then a
    saturation run: args.serve_saturation requests submitted at once against
    the same requests as one grape_walks_host launch each, rows compared."""
    import threading
    from paper_2110_06196_gb300 import Graph, Server, synth, walks_host
    # host buffers first: page-locked once, reused by every run
    pool = PinnedArena(args.serve_host_gib << 28)   # GiB of int32
    csr = synth.workload_graph(args.serve_graph, device=dev)
    g = Graph.from_csr(csr, validate=False, device=dev)
    n = g.num_nodes
    deg = csr.degrees().cpu().numpy()
    del csr
    torch.cuda.empty_cache()
    sat_mix = synth.request_mix(n, args.serve_saturation, gen_seed=99, max_starts=1_000_000,
                                len_lo=20, len_hi=120, first_seed=90_000)
    sizes = [len(r.starts) * r.walk_len for r in sat_mix]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    sat_buf = host_rows(int(offs[-1]))
    seq_buf = host_rows(int(offs[-1]))
    results = []
    rates = [float(x) for x in args.serve_rates.split(",")]
    # (rate index, idle exit): every rate with the default 2 ms idle exit, and
    # the lowest rate again with the resident kernel kept warm between requests
    runs = [(ri, 2000, args.serve_requests) for ri in range(len(rates))]
    if args.serve_warm_requests > 0:
        runs.append((0, 200_000, args.serve_warm_requests))
    for ri, idle_us, nreq in runs:
        rate = rates[ri]
        count = int(min(nreq, max(1, rate * args.serve_max_s)))
        mix = synth.request_mix(n, count, gen_seed=77 + ri, max_starts=1_000_000, len_lo=20,
                                len_hi=120, first_seed=10_000 * ri)
        arrivals = synth.poisson_arrivals(rate, len(mix), seed=5 + ri)
        log(f"serving {len(mix)} requests at {rate:g}/s, idle exit {idle_us} us")
        srv = Server(g, output_cap_bytes=40 << 30, max_inflight=4096, chunk_walks=0,
                     max_chunks=1 << 24, idle_exit_us=idle_us)
        bufs = {}
        lat = []
        mu = threading.Lock()
        checked = [0, 0]                        # requests checked, of which wrong

        def collect():
            while len(lat) < len(mix):
                t, l, rows = srv.wait_any(timeout_ms=600_000)
                with mu:
                    j, key = bufs.pop(t)
                lat.append(l)
                if j % 50 == 0:                 # rows follow the job's step count
                    r = mix[j]
                    want = int((deg[r.starts] > 0).sum()) * (r.walk_len - 1)
                    got = int((rows >= 0).sum()) - int((rows[:, 0] >= 0).sum())
                    checked[0] += 1
                    checked[1] += int(got != want)
                with mu:
                    pool.give(key)

        th = threading.Thread(target=collect)
        th.start()
        st0 = 0
        t0 = time.perf_counter()
        for j, r in enumerate(mix):
            delay = arrivals[j] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            elems = len(r.starts) * r.walk_len
            with mu:
                key, buf = pool.take(elems)
            out = buf[:elems].view(len(r.starts), r.walk_len)
            t = srv.submit(r.starts, r.walk_len, r.p, r.q, r.seed, out=out)
            with mu:
                bufs[t] = (j, key)
        th.join()
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        lat_ms = np.array(lat) * 1e3
        offered = sum(int((deg[r.starts] > 0).sum()) * (r.walk_len - 1) for r in mix)
        results.append({"rate_req_s": rate, "idle_exit_us": idle_us, "requests": len(mix),
                        "wall_s": wall,
                        "steps_per_s": (st["steps"] - st0) / wall,
                        "offered_steps_per_s": offered / arrivals[-1],
                        "p50_ms": float(np.percentile(lat_ms, 50)),
                        "p99_ms": float(np.percentile(lat_ms, 99)),
                        "max_ms": float(lat_ms.max()),
                        "kernel_launches": st["kernel_launches"],
                        "kernel_timeouts": st["kernel_timeouts"],
                        "host_buffers_outside_arena": pool.extra,
                        "requests_step_checked": checked[0],
                        "requests_step_mismatch": checked[1]})
    # Saturation: every request of one mix at once through the server, then the
    # same requests as one grape_walks_host launch each, one after another.
    mix = sat_mix
    outs = [sat_buf[int(offs[j]):int(offs[j + 1])].view(len(r.starts), r.walk_len)
            for j, r in enumerate(mix)]
    # five runs through fresh servers: the median run is reported, and all five
    runs = []
    for _ in range(5):
        srv = Server(g, output_cap_bytes=40 << 30, max_inflight=4096, chunk_walks=0,
                     max_chunks=1 << 24, idle_exit_us=2000)
        t0 = time.perf_counter()
        tickets = [srv.submit(r.starts, r.walk_len, r.p, r.q, r.seed, out=o)
                   for r, o in zip(mix, outs)]
        lat = []
        for _ in tickets:
            _, l, _ = srv.wait_any(timeout_ms=600_000)
            lat.append(l)
        runs.append((time.perf_counter() - t0, lat))
        steps = srv.stats()["steps"]
        srv.close()
    runs.sort(key=lambda r: r[0])
    t_srv, lat = runs[len(runs) // 2]
    seq_outs = [seq_buf[int(offs[j]):int(offs[j + 1])].view(len(r.starts), r.walk_len)
                for j, r in enumerate(mix)]
    seq_runs = []
    for _ in range(3):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for r, o in zip(mix, seq_outs):
            walks_host(g, r.starts, r.walk_len, 1, r.p, r.q, r.seed, out=o)
        seq_runs.append(time.perf_counter() - t0)
    t_seq = statistics.median(seq_runs)
    same = all(torch.equal(a, b) for a, b in zip(outs, seq_outs))
    lat_ms = np.array(lat) * 1e3
    g.close()
    del g, outs, seq_outs, pool, sat_buf, seq_buf
    torch.cuda.empty_cache()
    return {"graph": f"{args.serve_graph}: " + workload_graph_desc(args.serve_graph),
            "mix": "starts log-uniform [1, 1e6] (uniform ids), len U[20, 120], p, q in "
                   "{0.25, 0.5, 1, 2, 4}; 40 GB output cap; latency = submit to rows in host memory",
            "rates": results,
            "saturation": {"requests": len(mix), "steps": steps,
                           "served_steps_per_s": steps / t_srv,
                           "served_s_of_five_runs": [r[0] for r in runs],
                           "sequential_s_of_three_runs": seq_runs,
                           "sequential_steps_per_s": steps / t_seq,
                           "served_vs_one_launch_per_request": t_seq / t_srv,
                           "p50_ms": float(np.percentile(lat_ms, 50)),
                           "p99_ms": float(np.percentile(lat_ms, 99)),
                           "rows_identical_to_one_launch_per_request": bool(same)}}


def workload_graph_desc(name):
    from paper_2110_06196_gb300 import synth
    s = synth.WORKLOADS[name]
    return (f"R-MAT(a=.57,b=.19,c=.19) scale {s['scale']}, {s['m']} undirected edges"
            f"{', fp32 weights U[0.1,1]' if s['weighted'] else ', unweighted'} (seed {s['seed']})")


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands, on the host cores
# ---------------------------------------------------------------------------
def run_reference(args, dist):
    """The oracle as it stands on the host cores, on the headline job: each
    step times a bounded random sample of the job's walk ids.  Its `config` is
    the GPU arm's (same workload, rows, steps per launch, graph), so the two
    lines describe the same job; the sample is stated in `sample`."""
    if dist.rank != 0:
        return None
    from paper_2110_06196_gb300 import synth
    job = synth.WORKLOADS[args.workload]["job"]
    if args.walks_per_node > 0:
        job = dataclasses.replace(job, walks_per_node=args.walks_per_node)
    # input synthesis only (no walk arithmetic): on the GPU when there is one,
    # bit-identical to the CPU construction
    gen_dev = "cuda" if torch.cuda.is_available() else "cpu"
    csr = synth.workload_graph(args.workload, device=gen_dev)
    degrees = csr.degrees()
    csr_np = csr.numpy()
    n = csr.num_nodes
    num_entries = csr.num_entries
    del csr
    if gen_dev == "cuda":
        torch.cuda.empty_cache()
    rows = n * job.walks_per_node
    seconds = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    rates, sample, cores = [], None, os.cpu_count()
    for k in range(args.warmup + args.steps):
        rate, cores, sample = oracle_rate(csr_np, job, seconds)
        if k >= args.warmup:
            rates.append(rate)
    value = statistics.median(rates)
    steps = job_steps(degrees, job)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (seeded R-MAT / Erdos-Renyi stand-ins for the paper's graphs)",
            "config": config_of(args.workload, job, rows, steps, num_entries, dist.world),
            "sample": f"each step: {sample} on {cores} host threads",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    dist = Dist(args.gpus)
    try:
        if args.probe_buffer_sweep:
            torch.cuda.set_device(dist.local)
            res = probe_buffer_sweep(torch.device("cuda", dist.local)) if dist.rank == 0 else None
        elif args.impl == "reference":
            res = run_reference(args, dist)
        else:
            res = run_ours(args, dist)
        if dist.rank == 0 and res is not None:
            print(json.dumps(res), flush=True)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
