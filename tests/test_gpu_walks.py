"""GPU parity of the per-call path (grape_walks through the C ABI) against the
CPU oracle: bit-exact int32 rows.

Coverage: the eight p == 1 / q == 1 / weighted specialisations over a (p, q)
grid; membership searched in N(t) only, in the shorter of N(t) and N(x), or
mixed by degree; the exact fallback
(trial caps 0 and 2); tiny and structured graphs (house with a self-loop,
directed with a dead end, star, path, K_n); ragged walk counts and lengths,
unaligned output, explicit start lists, out-of-range starts, shards of a job,
host-buffer calls; the 1,000-node ER workload in full; the R-MAT scale-20
weighted workload at full size in full (10.5 M walks); and the scale-24
hub-heavy workload at full size on 2^20 walk ids in blocks plus every walk that
starts at one of the top 100 hubs (and both on sampled ids with top-64 hubs).
"""
import numpy as np
import pytest
import torch

import oracle
import _law
from paper_2110_06196_gb300 import Graph, GrapeError, synth, walks, walks_host
from paper_2110_06196_gb300 import walk as W

pytestmark = pytest.mark.gpu

PQ5 = (0.25, 0.5, 1.0, 2.0, 4.0)


def csr_from_np(off, dst, w=None, n=None):
    return synth.CSRGraph(torch.from_numpy(off), torch.from_numpy(dst),
                          None if w is None else torch.from_numpy(w), len(off) - 1)


def small_graphs():
    out = {}
    n, e = _law.graph_house()
    out["house"] = (csr_from_np(*_law.csr_from_edges(n, e, None, True)), True)
    wts = [0.1 + 0.9 * ((7 * k + 3) % 11) / 10 for k in range(len(e))]
    out["house_w"] = (csr_from_np(*_law.csr_from_edges(n, e, wts, True)), True)
    n, e = _law.graph_directed()
    out["directed"] = (csr_from_np(*_law.csr_from_edges(n, e, None, False)), False)
    wd = [0.2 + 0.15 * (k % 6) for k in range(len(e))]
    out["directed_w"] = (csr_from_np(*_law.csr_from_edges(n, e, wd, False)), False)
    out["star"] = (csr_from_np(*_law.csr_from_edges(9, [(0, i) for i in range(1, 9)])), True)
    out["path"] = (csr_from_np(*_law.csr_from_edges(12, [(i, i + 1) for i in range(11)])), True)
    kn = [(i, j) for i in range(8) for j in range(i + 1, 8)]
    out["k8"] = (csr_from_np(*_law.csr_from_edges(8, kn)), True)
    return out


_RMAT12 = {}


def rmat12(weighted):
    if weighted not in _RMAT12:
        _RMAT12[weighted] = synth.rmat(12, 40000, seed=21, weighted=weighted)
    return _RMAT12[weighted]


def check_parity(csr, starts, walk_len, wpn, p, q, seed, undirected=True, tuning=None,
                 graph=None, out=None):
    g = graph or Graph.from_csr(csr, undirected=undirected)
    if tuning:
        g.set_tuning(**tuning)
    got = walks(g, starts, walk_len, wpn, p, q, seed, out=out)
    torch.cuda.synchronize()
    g.stream_status()
    got = got.cpu().numpy()
    og = oracle.Graph(*csr.numpy())
    cap = g.get_tuning().trial_cap
    want, rc = oracle.walks(og, None if starts is None else np.asarray(starts), walk_len, wpn,
                            p, q, seed, trial_cap=cap)
    assert rc == 0
    if not np.array_equal(got, want):
        bad = np.argwhere((got != want).any(axis=1))[:, 0]
        raise AssertionError(f"{len(bad)} rows differ, first {bad[:5].tolist()}:\n"
                             f"gpu    {got[bad[0]].tolist()}\noracle {want[bad[0]].tolist()}")
    return got


def test_device_philox_matches_published_vectors_and_oracle():
    import os
    kat = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [[int(x, 16) for x in l.split()] for l in open(kat)
            if l.strip() and not l.startswith("#")]
    rng = np.random.default_rng(5)
    rnd = rng.integers(0, 2**32, size=(4096, 6), dtype=np.uint64)
    ck = np.concatenate([np.array([r[:6] for r in rows], np.uint64), rnd]).astype(np.uint32)
    got = W.philox4x32_10(torch.from_numpy(ck.view(np.int32)).cuda()).cpu().numpy().view(np.uint32)
    for j, r in enumerate(rows):
        assert got[j].tolist() == r[6:10]
    for j in range(len(rows), len(ck)):
        assert got[j].tolist() == oracle.philox4x32_10(ck[j, :4], ck[j, 4:6]).tolist()


@pytest.mark.parametrize("name", sorted(small_graphs()))
def test_small_graphs_all_pq(name):
    csr, und = small_graphs()[name]
    g = Graph.from_csr(csr, undirected=und)
    for p in PQ5:
        for q in PQ5:
            check_parity(csr, None, 17, 9, p, q, seed=int(p * 100 + q * 10), undirected=und,
                         graph=g)


@pytest.mark.parametrize("weighted", [False, True], ids=["unweighted", "weighted"])
@pytest.mark.parametrize("shorter_min", [0, 16, 0x7fffffff], ids=["shorter", "mixed", "n_t"])
def test_rmat12_specialisations_and_search_paths(weighted, shorter_min):
    csr = rmat12(weighted)
    g = Graph.from_csr(csr)
    g.set_tuning(shorter_min=shorter_min)
    for (p, q) in [(1.0, 1.0), (2.0, 1.0), (1.0, 0.5), (0.5, 2.0), (4.0, 0.25), (0.25, 4.0)]:
        check_parity(csr, None, 24, 2, p, q, seed=99, graph=g)


HUB_SCHEDULES = [dict(edge_hash=0, pivot_min=1), dict(edge_hash=0, pivot_min=32),
                 dict(edge_hash=0, pivot_min=0x7fffffff),
                 dict(edge_hash=0, warp_search_min=0), dict(edge_hash=0, warp_search_min=32),
                 dict(edge_hash=0, pivot_min=32, warp_search_min=300),
                 dict(edge_hash=0, pivot_min=1, l2_persist_mb=16),
                 dict(edge_hash=1), dict(edge_hash=1, pivot_min=1)]


@pytest.mark.parametrize("weighted", [False, True], ids=["unweighted", "weighted"])
@pytest.mark.parametrize("schedule", HUB_SCHEDULES,
                         ids=lambda d: "-".join(f"{k}{v}" for k, v in d.items()))
@pytest.mark.parametrize("shorter_min", [0, 0x7fffffff], ids=["shorter", "n_t"])
def test_rmat12_hub_search_schedules(weighted, schedule, shorter_min):
    """The degree-aware search schedules (sector pivots from a list length on,
    warp-cooperative narrowing above a list length, the L2 window on the
    pivots) change no row: R-MAT 12 (degrees up to ~1,000) against the oracle."""
    csr = rmat12(weighted)
    g = Graph.from_csr(csr)
    g.set_tuning(shorter_min=shorter_min, **schedule)
    g.counters(enable=True)
    for (p, q) in [(1.0, 0.5), (0.5, 2.0), (4.0, 0.25), (0.25, 4.0)]:
        check_parity(csr, None, 24, 2, p, q, seed=98, graph=g)
    c = g.counters()
    g.counters(enable=False)
    if schedule.get("edge_hash", 1):
        # every membership test reads its pair's bucket first
        assert c["hash_probes"] == c["searches"] > 0
    elif schedule.get("pivot_min", 0x7fffffff) < 0x7fffffff:
        assert c["pivot_probes"] > 0 and c["hash_probes"] == 0
    else:
        assert c["pivot_probes"] == 0 and c["hash_probes"] == 0
    assert c["pivot_probes"] + c["hash_probes"] <= c["probes"]


def _chunk_straddling_graph(weighted):
    """Undirected graph for the common-neighbour filter build, which cuts the
    entry array into chunks of 512 entries: ten hubs of about 700 neighbours
    (rows that straddle chunk boundaries), runs of isolated nodes between
    non-empty rows, self-loops on hubs and leaves, a 61-node clique (pairs with
    many common neighbours) and random edges (triangles)."""
    rng = np.random.default_rng(2024)
    n = 2400
    live = np.array([v for v in range(n) if v % 7 != 3 and not 1500 <= v < 1540])
    edges = set()
    for h in range(10):
        for x in rng.choice(live[live >= 10], size=700, replace=False):
            edges.add((h, int(x)))
        for h2 in range(h + 1, 10):
            edges.add((h, h2))
    for a in range(100, 161):
        for b in range(a + 1, 161):
            if a % 7 != 3 and b % 7 != 3:
                edges.add((a, b))
    for _ in range(5000):
        a, b = (int(v) for v in rng.choice(live, size=2, replace=False))
        edges.add((min(a, b), max(a, b)))
    for v in (0, 1, 17, 250, 2399):
        edges.add((v, v))
    edges = sorted(edges)
    wts = rng.uniform(0.1, 1.0, size=len(edges)).astype(np.float32) if weighted else None
    return csr_from_np(*_law.csr_from_edges(n, edges, wts, True))


@pytest.mark.parametrize("weighted", [False, True], ids=["unweighted", "weighted"])
def test_filters_built_over_chunks_straddling_rows(weighted):
    """Rows equal the oracle's on a graph whose hub rows cross the filter
    build's chunk boundaries, with isolated runs and self-loops, for (p, q)
    where membership decides acceptance."""
    csr = _chunk_straddling_graph(weighted)
    assert csr.num_entries > 20 * 512
    g = Graph.from_csr(csr)
    for p, q in ((1.0, 0.25), (0.5, 4.0), (2.0, 0.5)):
        check_parity(csr, None, 40, 3, p, q, seed=int(p * 100 + q * 10), graph=g)


def test_hub_search_schedules_on_a_hub_graph():
    """A hub of degree 6,000 joined to a ring: every search meets long lists,
    pivot and warp schedules both run many rounds; rows equal the oracle's."""
    hub = 6000
    edges = [(0, i) for i in range(1, hub + 1)] + [(i, i + 1) for i in range(1, hub)] + \
            [(i, i + 7) for i in range(1, hub - 7, 3)]
    csr = csr_from_np(*_law.csr_from_edges(hub + 1, edges))
    for sched in ({}, dict(edge_hash=0), dict(edge_hash=0, pivot_min=1),
                  dict(edge_hash=0, warp_search_min=0),
                  dict(edge_hash=0, pivot_min=64, warp_search_min=1000)):
        g = Graph.from_csr(csr)
        g.set_tuning(shorter_min=0x7fffffff, **sched)
        for (p, q) in [(1.0, 0.25), (2.0, 0.5)]:
            check_parity(csr, None, 30, 3, p, q, seed=11, graph=g)


def _edge_hash_bucket(a, b, n, pairs):
    """The bucket the library's edge hash gives the pair {a, b} (the table's
    layout rule, restated for the test: k bits per id, about 3.5 pairs per
    8-slot bucket, the mixing bijection of 2k-bit keys)."""
    k = 1
    while k < 31 and (1 << k) < n:
        k += 1
    K = 2 * k
    bb = 0
    while bb < K and (1 << bb) * 3.5 < pairs:
        bb += 1
    bb = max(bb, K - 31)
    mask = (1 << K) - 1
    x = ((min(a, b) << k) | max(a, b)) & mask
    x ^= x >> (K // 2 + 1)
    x = (x * 0x9E3779B97F4A7C15) & mask
    x ^= x >> (K // 3 + 1)
    x = (x * 0xD6E8FEB86659FD93) & mask
    x ^= x >> (K // 2 + 1)
    return x >> (K - bb)


def test_edge_hash_overflowed_bucket_falls_back_to_the_rows():
    """14 pairs that share one 8-slot bucket of the edge hash, among 180 other
    pairs: tests on pairs the bucket could not hold read the sorted rows, and
    every row equals the oracle's."""
    n, total = 64, 190
    from itertools import combinations
    allp = [(a, b) for a, b in combinations(range(n), 2)]
    by = {}
    for a, b in allp:
        by.setdefault(_edge_hash_bucket(a, b, n, total), []).append((a, b))
    crowd = max(by.values(), key=len)[:14]
    assert len(crowd) == 14
    rng = np.random.default_rng(3)
    rest = [allp[i] for i in rng.permutation(len(allp))]
    edges = list(crowd)
    for pr in rest:
        if len(edges) == total:
            break
        if pr not in crowd:
            edges.append(pr)
    csr = csr_from_np(*_law.csr_from_edges(n, edges))
    g = Graph.from_csr(csr)
    assert g.info()["edge_hash_bytes"] > 0
    g.counters(enable=True)
    for (p, q) in [(1.0, 0.25), (0.5, 2.0), (4.0, 0.25)]:
        check_parity(csr, None, 40, 20, p, q, seed=17, graph=g)
    c = g.counters()
    g.counters(enable=False)
    assert c["hash_probes"] == c["searches"] > 0
    assert c["probes"] > c["hash_probes"]          # some tests went on to the rows


@pytest.mark.parametrize("cap", [0, 2])
def test_exact_fallback_paths(cap):
    for weighted in (False, True):
        csr = rmat12(weighted)
        g = Graph.from_csr(csr)
        g.set_tuning(trial_cap=cap)
        for (p, q) in [(0.25, 4.0), (2.0, 0.5), (1.0, 1.0)]:
            check_parity(csr, None, 12, 1, p, q, seed=3, graph=g)
    n, e = _law.graph_directed()
    csr = csr_from_np(*_law.csr_from_edges(n, e, [0.3 + 0.1 * k for k in range(len(e))], False))
    g = Graph.from_csr(csr, undirected=False)
    g.set_tuning(trial_cap=cap)
    check_parity(csr, None, 15, 20, 0.5, 2.0, seed=4, undirected=False, graph=g)


@pytest.mark.parametrize("weighted", [False, True], ids=["unweighted", "weighted"])
def test_work_counters_match_the_oracle(weighted):
    """Transitions, proposals drawn and fallback steps are the oracle's counts
    exactly (the kernel takes the same decisions); proposals whose entry was
    read are a subset of those drawn, and strictly fewer once returns or the
    larger non-return threshold let the kernel decide without a read; the
    neighbour filters settle some membership tests."""
    csr = rmat12(weighted)
    g = Graph.from_csr(csr)
    og = oracle.Graph(*csr.numpy())
    cap = g.get_tuning().trial_cap
    g.counters(enable=True)
    try:
        for (p, q) in [(1.0, 1.0), (0.5, 2.0), (0.25, 1.0), (4.0, 0.25)]:
            walks(g, None, 20, 2, p, q, 17)
            c = g.counters()
            st = oracle.OracleStats()
            _, rc = oracle.walks(og, None, 20, 2, p, q, 17, trial_cap=cap, stats=st)
            assert rc == 0
            assert (c["steps"], c["trials"], c["fallbacks"]) == (st.steps, st.trials, st.fallbacks)
            assert c["walks"] == 2 * csr.num_nodes
            assert c["gathers"] <= c["trials"]
            if p < min(1.0, q):
                # half or more of the non-return proposals fail 1/(p amax)
                assert c["gathers"] < 0.75 * c["trials"]
            if q != 1.0:
                # the pair filters (common neighbours; 96 bits unweighted, 32
                # weighted) settle part of the membership tests
                assert c["filtered"] > 0
            else:
                assert c["filtered"] == 0
    finally:
        g.counters(enable=False)


@pytest.mark.parametrize("walk_len", [1, 2, 3, 5, 33])
@pytest.mark.parametrize("wpn", [1, 3])
def test_ragged_lengths_and_counts(walk_len, wpn):
    csr = rmat12(True)
    starts = np.random.default_rng(walk_len).integers(0, csr.num_nodes, 1000 + walk_len)
    check_parity(csr, starts.astype(np.int32), walk_len, wpn, 0.5, 2.0, seed=walk_len)


def test_unaligned_output_buffer():
    csr = rmat12(False)
    g = Graph.from_csr(csr)
    rows, L = 777, 13
    buf = torch.empty(rows * L + 1, dtype=torch.int32, device="cuda")
    out = buf[1:].view(rows, L)
    assert out.data_ptr() % 16 != 0
    starts = np.arange(rows, dtype=np.int32) % csr.num_nodes
    check_parity(csr, starts, L, 1, 2.0, 0.5, seed=8, graph=g, out=out)


def test_out_of_range_starts_set_status_and_fill_minus_one():
    csr = rmat12(False)
    g = Graph.from_csr(csr)
    starts = torch.tensor([0, -1, 5, csr.num_nodes, 7], dtype=torch.int32, device="cuda")
    out = walks(g, starts, 6, 1, 1.0, 1.0, seed=1)
    with pytest.raises(GrapeError) as ei:
        g.stream_status()
    assert ei.value.name == "GRAPE_ERR_DEVICE"
    o = out.cpu().numpy()
    assert (o[1] == -1).all() and (o[3] == -1).all()
    assert o[0, 0] == 0 and o[2, 0] == 5 and o[4, 0] == 7
    g.stream_status()          # cleared


def test_argument_errors():
    csr = rmat12(False)
    g = Graph.from_csr(csr)
    for bad in [dict(p=0.0), dict(q=-1.0), dict(p=float("nan")), dict(walk_len=0),
                dict(walks_per_node=0)]:
        kw = dict(walk_len=4, walks_per_node=1, p=1.0, q=1.0)
        kw.update(bad)
        with pytest.raises(GrapeError) as ei:
            walks(g, None, kw["walk_len"], kw["walks_per_node"], kw["p"], kw["q"], 0,
                  out=torch.empty((csr.num_nodes, 4), dtype=torch.int32, device="cuda"))
        assert ei.value.name == "GRAPE_ERR_INVALID_ARG"


def test_invalid_graphs_are_rejected():
    off = torch.tensor([0, 2, 3, 4], dtype=torch.int64)
    cases = {
        "unsorted": (off, torch.tensor([2, 1, 0, 0], dtype=torch.int32), None),
        "id_range": (off, torch.tensor([1, 7, 0, 0], dtype=torch.int32), None),
        "offsets": (torch.tensor([0, 3, 2, 4]), torch.tensor([1, 2, 0, 0], dtype=torch.int32), None),
        "weights": (off, torch.tensor([1, 2, 0, 0], dtype=torch.int32),
                    torch.tensor([1.0, -1.0, 1.0, 1.0])),
        "asymmetric": (off, torch.tensor([1, 2, 0, 1], dtype=torch.int32), None),
    }
    for name, (o, d, w) in cases.items():
        with pytest.raises(GrapeError) as ei:
            Graph(o, d, w, undirected=True, validate=True)
        assert ei.value.name == "GRAPE_ERR_INVALID_GRAPH", name


def test_shards_reassemble_the_job():
    csr = rmat12(True)
    g = Graph.from_csr(csr)
    full = walks(g, None, 20, 3, 0.5, 2.0, seed=17).cpu().numpy()
    lib = g._lib
    total = csr.num_nodes * 3
    bounds = [0, 1, 4097, 9000, total]
    for b, e in zip(bounds[:-1], bounds[1:]):
        out = torch.empty((e - b, 20), dtype=torch.int32, device="cuda")
        import ctypes
        code = lib.grape_walks_range(g.handle, None, csr.num_nodes, 20, 3, 0.5, 2.0, 17, b, e - b,
                                     ctypes.c_void_p(out.data_ptr()), W._stream_ptr())
        assert code == 0
        assert np.array_equal(out.cpu().numpy(), full[b:e])


def test_host_buffer_entry_point_matches_device_path():
    csr = rmat12(True)
    g = Graph.from_csr(csr)
    starts = np.random.default_rng(1).integers(0, csr.num_nodes, 3001).astype(np.int32)
    dev = walks(g, torch.from_numpy(starts).cuda(), 31, 2, 2.0, 0.5, seed=5).cpu().numpy()
    host = walks_host(g, starts, 31, 2, 2.0, 0.5, seed=5)
    assert np.array_equal(dev, host)


@pytest.mark.parametrize("pinned", [False, True], ids=["pageable", "pinned"])
def test_host_buffer_entry_point_in_slices(pinned):
    """Outputs above the slice size leave in several slices whose copies
    overlap the walks of later slices; rows equal the device path's."""
    csr = rmat12(False)
    g = Graph.from_csr(csr)
    wpn, L = 1300, 9                      # 5.3 M rows of 36 bytes (191 MB): 2 slices
    dev = walks(g, None, L, wpn, 0.5, 2.0, seed=8).cpu().numpy()
    out = torch.empty(dev.shape, dtype=torch.int32)
    if pinned:
        out = out.pin_memory()
    host = walks_host(g, None, L, wpn, 0.5, 2.0, seed=8, out=out)
    assert np.array_equal(dev, host.numpy())


def test_er1k_workload_full_parity():
    csr = synth.workload_graph("er1k")
    job = synth.WORKLOADS["er1k"]["job"]
    check_parity(csr, None, job.walk_len, job.walks_per_node, job.p, job.q, job.seed)


def _sampled_parity(name, n_sample, hubs=64, threads=None):
    spec = synth.WORKLOADS[name]
    job = spec["job"]
    csr = synth.workload_graph(name, device="cuda")
    g = Graph.from_csr(csr, validate=False)
    out = walks(g, None, job.walk_len, job.walks_per_node, job.p, job.q, job.seed)
    torch.cuda.synchronize()
    g.stream_status()
    n = csr.num_nodes
    total = n * job.walks_per_node
    rng = np.random.default_rng(2024)
    ids = rng.choice(total, size=n_sample, replace=False)
    deg = csr.degrees()
    top = torch.topk(deg, hubs).indices.cpu().numpy()
    hub_ids = (top[None, :] + n * np.arange(job.walks_per_node)[:, None]).ravel()
    ids = np.unique(np.concatenate([ids, hub_ids, [0, total - 1]]))
    ids_t = torch.from_numpy(ids).cuda()
    got = out[ids_t].cpu().numpy()
    # every step follows an edge: checked on the device for a block of rows
    blk = out[: min(total, 200_000)].to(torch.int64)
    a, b = blk[:, :-1], blk[:, 1:]
    valid = b >= 0
    keys = csr.offsets.new_zeros(0)
    row_off = csr.offsets
    lo = row_off[a.clamp(min=0)]
    hi = row_off[a.clamp(min=0) + 1]
    # membership of b in row a by searchsorted over the global (row, dst) key space
    gkeys = torch.repeat_interleave(torch.arange(n, device="cuda"), (row_off[1:] - row_off[:-1])) * n \
        + csr.dsts.to(torch.int64)
    q = a.clamp(min=0) * n + b.clamp(min=0)
    pos = torch.searchsorted(gkeys, q[valid])
    ok = gkeys[pos.clamp(max=gkeys.numel() - 1)] == q[valid]
    assert bool(ok.all()), "a GPU step left the edge set"
    del gkeys, keys, lo, hi, blk, a, b, q, pos, ok
    del out
    torch.cuda.empty_cache()
    og = oracle.Graph(*csr.numpy())
    want = np.empty_like(got)
    import os
    from concurrent.futures import ThreadPoolExecutor
    parts = np.array_split(np.arange(len(ids)), threads or os.cpu_count() or 4)

    def run(part):
        want[part] = oracle.walk_rows(og, None, job.walk_len, job.walks_per_node, job.p, job.q,
                                      job.seed, ids[part])

    with ThreadPoolExecutor(len(parts)) as ex:
        list(ex.map(run, parts))
    bad = np.argwhere((got != want).any(axis=1))[:, 0]
    assert len(bad) == 0, f"{len(bad)} of {len(ids)} sampled rows differ, first id {ids[bad[0]]}"
    return len(ids)


def test_rmat20_weighted_workload_sampled_parity():
    assert _sampled_parity("rmat20w", 20000) > 20000


@pytest.mark.slow
def test_rmat24_workload_sampled_parity():
    assert _sampled_parity("rmat24", 20000) > 20000


@pytest.mark.slow
def test_rmat20w_workload_full_parity():
    # the whole job (10,485,760 walks x 100 entries, 1.05 G steps) against the
    # oracle, its walk ids split over the host cores in blocks of 2^20
    spec = synth.WORKLOADS["rmat20w"]
    job = spec["job"]
    csr = synth.workload_graph("rmat20w", device="cuda")
    g = Graph.from_csr(csr, validate=False)
    out = walks(g, None, job.walk_len, job.walks_per_node, job.p, job.q, job.seed)
    torch.cuda.synchronize()
    g.stream_status()
    total = out.shape[0]
    og = oracle.Graph(*csr.to("cpu").numpy())
    block = 1 << 20
    for lo in range(0, total, block):
        hi = min(total, lo + block)
        want = oracle.walks_parallel(og, None, job.walk_len, job.walks_per_node, job.p, job.q,
                                     job.seed, walk_ids=(lo, hi))
        got = out[lo:hi].cpu().numpy()
        bad = np.argwhere((got != want).any(axis=1))[:, 0]
        assert len(bad) == 0, f"walk {lo + bad[0]} differs ({len(bad)} rows in [{lo}, {hi}))"


@pytest.mark.slow
def test_rmat24_workload_million_walks_and_hub_starts():
    # 2^20 walk ids in 8 blocks at seeded offsets, plus every walk from the top
    # 100 hubs, of the full 167.8 M-walk job
    spec = synth.WORKLOADS["rmat24"]
    job = spec["job"]
    csr = synth.workload_graph("rmat24", device="cuda")
    g = Graph.from_csr(csr, validate=False)
    out = walks(g, None, job.walk_len, job.walks_per_node, job.p, job.q, job.seed)
    torch.cuda.synchronize()
    g.stream_status()
    n = csr.num_nodes
    total = out.shape[0]
    top = torch.topk(csr.degrees(), 100).indices.cpu().numpy()
    og = oracle.Graph(*csr.to("cpu").numpy())
    del csr
    block = 1 << 17
    rng = np.random.default_rng(24)
    starts = np.sort(rng.choice(total // block, size=8, replace=False)) * block
    checked = 0
    for lo in starts:
        hi = lo + block
        want = oracle.walks_parallel(og, None, job.walk_len, job.walks_per_node, job.p, job.q,
                                     job.seed, walk_ids=(int(lo), int(hi)))
        got = out[int(lo):int(hi)].cpu().numpy()
        bad = np.argwhere((got != want).any(axis=1))[:, 0]
        assert len(bad) == 0, f"walk {lo + bad[0]} differs"
        checked += block
    hub_ids = (top[None, :] + n * np.arange(job.walks_per_node)[:, None]).ravel()
    want = oracle.walk_rows(og, None, job.walk_len, job.walks_per_node, job.p, job.q, job.seed,
                            hub_ids)
    got = out[torch.from_numpy(hub_ids).cuda()].cpu().numpy()
    assert np.array_equal(got, want)
    assert checked + len(hub_ids) >= (1 << 20)
