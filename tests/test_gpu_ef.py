"""GPU parity of the Elias-Fano graph store (grape_ef_* through the C ABI)
against the CPU oracles, bit for bit:

* the store itself: the low and high words and both indexes equal the Elias-Fano
  oracle's arrays for graphs with and without isolated nodes, directed, with a
  self-loop, |V| = 1, |V| a power of two, fewer entries than nodes (l > k), no
  entries at all, and quanta 1 to 1024; hub rows get bucket directories;
* select and rank on every index and on random and boundary values (bucket
  edges, row edges, values at and beyond u) equal the oracle's;
* walks over the store equal the walk oracle's rows on tiny structured graphs
  over a (p, q) grid, on R-MAT scale 12 weighted and unweighted, with trial caps
  0 and 2, ragged lengths, explicit and out-of-range starts; and equal the CSR
  engine's rows (itself oracle-checked) on the whole R-MAT scale-20 weighted job,
  with sampled rows checked against the oracle;
* work counters: steps, proposals and fallbacks equal the oracle's counts, and
  codes are read for every proposal except those decided without a read;
* invalid CSRs are rejected.
"""
import numpy as np
import pytest
import torch

import oracle
import _law
from oracle import elias_fano as OEF
from paper_2110_06196_gb300 import EFGraph, Graph, GrapeError, ef_walks, synth, walks

pytestmark = pytest.mark.gpu

PQ5 = (0.25, 0.5, 1.0, 2.0, 4.0)


def csr_np(off, dst, w=None):
    return synth.CSRGraph(torch.from_numpy(np.asarray(off, np.int64)),
                          torch.from_numpy(np.asarray(dst, np.int32)),
                          None if w is None else torch.from_numpy(np.asarray(w, np.float32)),
                          len(off) - 1)


def store_graphs():
    g = {}
    n, e = _law.graph_house()
    g["house"] = csr_np(*_law.csr_from_edges(n, e, None, True))
    n, e = _law.graph_directed()
    g["directed"] = csr_np(*_law.csr_from_edges(n, e, None, False))
    g["one_node"] = csr_np([0, 1], [0])
    g["one_node_empty"] = csr_np([0, 0], [])
    g["no_entries"] = csr_np([0] * 9, [])
    g["pow2_nodes"] = synth.erdos_renyi(256, 700, seed=8)
    g["er300"] = synth.erdos_renyi(300, 1200, seed=3)
    g["sparse_l_gt_k"] = synth.erdos_renyi(1000, 200, seed=9)   # 400 entries < 1000 nodes
    g["rmat10"] = synth.rmat(10, 6000, seed=4)
    return g


DIRECTED = {"directed", "directed_w"}


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("name", sorted(store_graphs()))
@pytest.mark.parametrize("quantum", [1, 8, 64, 1024])
def test_store_words_equal_oracle(name, quantum):
    csr = store_graphs()[name]
    off, dst, _ = csr.numpy()
    want = OEF.EFGraph(off, dst, csr.num_nodes, quantum=quantum)
    g = EFGraph.from_csr(csr, quantum=quantum, undirected=name not in DIRECTED)
    info = g.info()
    assert info["code_bits"] == want.k and info["low_bits"] == want.ef.l
    assert info["universe"] == want.ef.u and info["num_zeros"] == want.ef.num_zeros
    assert info["high_bits"] == want.ef.high_len
    got = g.export()
    torch.cuda.synchronize()
    assert np.array_equal(_u64(got["low"]), want.ef.low_words)
    assert np.array_equal(_u64(got["high"]), want.ef.high_words)
    assert np.array_equal(got["ones_index"].cpu().numpy(), want.ef.ones_index)
    assert np.array_equal(got["zeros_index"].cpu().numpy(), want.ef.zeros_index)
    assert info["max_degree"] == (int(np.diff(off).max()) if len(off) > 1 else 0)


@pytest.mark.parametrize("name", ["house", "directed", "one_node", "sparse_l_gt_k", "rmat10",
                                  "no_entries", "pow2_nodes"])
@pytest.mark.parametrize("quantum", [1, 16, 1024])
def test_select_rank_equal_oracle(name, quantum):
    csr = store_graphs()[name]
    off, dst, _ = csr.numpy()
    want = OEF.EFGraph(off, dst, csr.num_nodes, quantum=quantum).ef
    g = EFGraph.from_csr(csr, quantum=quantum, undirected=name not in DIRECTED)
    rng = np.random.default_rng(quantum)
    m, u, l = want.n, want.u, want.l
    idx = np.arange(m) if m <= 3000 else rng.integers(0, m, 3000)
    if m:
        got = g.select(torch.from_numpy(idx.astype(np.int64))).cpu().numpy()
        assert got.tolist() == [want.select(int(i)) for i in idx]
    # values: random, bucket edges, codes and their neighbours, row edges, beyond u
    vals = set(rng.integers(-3, u + 5, 1500).tolist())
    for h in range(0, min((u >> l) + 2, 400)):
        vals.update({(h << l) - 1, h << l, (h << l) + 1})
    codes = want.values() if m <= 3000 else np.array([want.select(int(i)) for i in idx[:300]])
    for c in codes[:1000]:
        vals.update({int(c) - 1, int(c), int(c) + 1})
    k = OEF.code_bits(csr.num_nodes)
    for a in range(0, csr.num_nodes + 1, max(1, csr.num_nodes // 200)):
        vals.add(a << k)
    vals.update({0, u - 1, u, u + 1, -(1 << 40), 1 << 62})
    vals = np.array(sorted(vals), dtype=np.int64)
    got = g.rank(torch.from_numpy(vals)).cpu().numpy()
    assert got.tolist() == [want.rank(int(v)) for v in vals]


def test_select_out_of_range_sets_status():
    g = EFGraph.from_csr(store_graphs()["house"], quantum=8)
    out = g.select(torch.tensor([0, -1, 10 ** 6], dtype=torch.int64)).cpu().tolist()
    assert out[1] == -1 and out[2] == -1
    with pytest.raises(GrapeError):
        g.stream_status()
    g.stream_status()          # cleared


def check_walks(csr, starts, walk_len, wpn, p, q, seed, trial_cap=4096, quantum=64, g=None,
                undirected=True):
    g = g or EFGraph.from_csr(csr, quantum=quantum, undirected=undirected)
    st = None if starts is None else torch.as_tensor(np.asarray(starts, np.int32))
    got = ef_walks(g, st, walk_len, wpn, p, q, seed, trial_cap=trial_cap)
    torch.cuda.synchronize()
    g.stream_status()
    got = got.cpu().numpy()
    og = oracle.Graph(*csr.numpy())
    want, rc = oracle.walks(og, None if starts is None else np.asarray(starts), walk_len, wpn,
                            p, q, seed, trial_cap=trial_cap)
    assert rc == 0
    if not np.array_equal(got, want):
        bad = np.argwhere((got != want).any(axis=1))[:, 0]
        raise AssertionError(f"{len(bad)} rows differ, first {bad[:5].tolist()}:\n"
                             f"gpu    {got[bad[0]].tolist()}\noracle {want[bad[0]].tolist()}")


def tiny_graphs():
    out = {}
    n, e = _law.graph_house()
    out["house"] = csr_np(*_law.csr_from_edges(n, e, None, True))
    wts = [0.1 + 0.9 * ((7 * k + 3) % 11) / 10 for k in range(len(e))]
    out["house_w"] = csr_np(*_law.csr_from_edges(n, e, wts, True))
    n, e = _law.graph_directed()
    out["directed"] = csr_np(*_law.csr_from_edges(n, e, None, False))
    wd = [0.2 + 0.15 * (k % 6) for k in range(len(e))]
    out["directed_w"] = csr_np(*_law.csr_from_edges(n, e, wd, False))
    out["star"] = csr_np(*_law.csr_from_edges(9, [(0, i) for i in range(1, 9)]))
    kn = [(i, j) for i in range(8) for j in range(i + 1, 8)]
    out["k8"] = csr_np(*_law.csr_from_edges(8, kn))
    return out


@pytest.mark.parametrize("name", sorted(tiny_graphs()))
def test_walks_tiny_graphs_all_pq(name):
    csr = tiny_graphs()[name]
    g = EFGraph.from_csr(csr, quantum=2, undirected=name not in DIRECTED)
    for p in PQ5:
        for q in PQ5:
            check_walks(csr, None, 17, 9, p, q, seed=int(p * 100 + q * 10), g=g)


_RMAT12 = {}


def rmat12(weighted):
    if weighted not in _RMAT12:
        _RMAT12[weighted] = synth.rmat(12, 40000, seed=21, weighted=weighted)
    return _RMAT12[weighted]


def expected_directory_rows(csr):
    """Rows that get a bucket directory: deg + nb > 448 and deg >= 8 nb, with
    nb = 2^(k - l) buckets per row (computed here from the CSR)."""
    off, dst, _ = csr.numpy()
    d = np.diff(off)
    k = OEF.code_bits(csr.num_nodes)
    l = OEF.low_bits_count(len(dst), csr.num_nodes << k)
    if l > k or len(dst) == 0:
        return 0
    nb = 1 << (k - l)
    return int(((d + nb > 448) & (d >= 8 * nb)).sum())


@pytest.mark.parametrize("weighted", [False, True], ids=["unweighted", "weighted"])
@pytest.mark.parametrize("quantum", [64, 1024])
def test_walks_rmat12(weighted, quantum):
    csr = rmat12(weighted)
    g = EFGraph.from_csr(csr, quantum=quantum)
    assert g.info()["directory_rows"] == expected_directory_rows(csr) > 0
    for (p, q) in [(1.0, 1.0), (2.0, 1.0), (1.0, 0.5), (0.5, 2.0), (4.0, 0.25), (0.25, 4.0)]:
        check_walks(csr, None, 24, 2, p, q, seed=99, g=g)


@pytest.mark.parametrize("cap", [0, 2])
def test_walks_exact_fallback(cap):
    for weighted in (False, True):
        csr = rmat12(weighted)
        g = EFGraph.from_csr(csr, quantum=64)
        for (p, q) in [(0.5, 2.0), (4.0, 0.25)]:
            check_walks(csr, None, 12, 1, p, q, seed=5, trial_cap=cap, g=g)


def test_walks_ragged_lengths_starts_and_dead_ends():
    csr = synth.rmat(11, 9000, seed=31)     # leaves isolated nodes: dead starts
    g = EFGraph.from_csr(csr, quantum=32)
    rng = np.random.default_rng(1)
    starts = rng.integers(0, csr.num_nodes, 777).astype(np.int32)
    for L in (1, 2, 3, 5, 33):
        for wpn in (1, 3):
            check_walks(csr, starts, L, wpn, 0.5, 2.0, seed=L * 7 + wpn, g=g)
    n, e = _law.graph_directed()
    d = csr_np(*_law.csr_from_edges(n, e, None, False))
    check_walks(d, None, 40, 5, 1.0, 0.5, seed=3, quantum=1, undirected=False)


def test_walks_with_more_low_bits_than_code_bits():
    # 400 entries over 1000 nodes: l > k, rows do not start buckets, and the
    # walks fall back to rank and select on the whole store
    csr = store_graphs()["sparse_l_gt_k"]
    g = EFGraph.from_csr(csr, quantum=8)
    info = g.info()
    assert info["low_bits"] > info["code_bits"] and info["directory_rows"] == 0
    for (p, q) in [(1.0, 1.0), (0.5, 2.0), (4.0, 0.25)]:
        check_walks(csr, None, 12, 2, p, q, seed=21, g=g)


def test_walks_out_of_range_starts():
    csr = rmat12(False)
    g = EFGraph.from_csr(csr)
    st = torch.tensor([0, -4, 5, csr.num_nodes, 7], dtype=torch.int32)
    out = ef_walks(g, st, 6, 2, 1.0, 0.5, seed=1).cpu().numpy()
    with pytest.raises(GrapeError):
        g.stream_status()
    for r in (1, 3, 6, 8):
        assert (out[r] == -1).all()
    og = oracle.Graph(*csr.numpy())
    want, rc = oracle.walks(og, st.numpy(), 6, 2, 1.0, 0.5, 1)
    assert rc == -1 and np.array_equal(out, want)


def test_counters_equal_oracle_counts():
    for weighted in (False, True):
        csr = rmat12(weighted)
        g = EFGraph.from_csr(csr, quantum=64)
        og = oracle.Graph(*csr.numpy())
        for (p, q, cap) in [(0.5, 2.0, 4096), (4.0, 0.25, 4096), (1.0, 0.5, 2)]:
            g.counters(True)
            ef_walks(g, None, 20, 1, p, q, seed=17, trial_cap=cap)
            c = g.counters()
            g.counters(False)
            st = oracle.OracleStats()
            oracle.walks(og, None, 20, 1, p, q, 17, trial_cap=cap, stats=st)
            assert c["steps"] == st.steps
            assert c["trials"] == st.trials
            assert c["fallbacks"] == st.fallbacks
            # returns and certain rejections are decided without reading a code when
            # the return has the largest bias (p < 1 and p < q here); else every
            # proposal reads its code
            ret_largest = (1.0 / p) > max(1.0, 1.0 / q)
            if ret_largest:
                assert 0 < c["codes_read"] < st.trials
            else:
                assert c["codes_read"] == st.trials
            assert c["sectors"] > 0


def test_er1k_in_full():
    csr = synth.workload_graph("er1k")
    job = synth.WORKLOADS["er1k"]["job"]
    check_walks(csr, None, job.walk_len, job.walks_per_node, job.p, job.q, job.seed)


def test_rmat20w_full_job_equals_csr_engine_and_sampled_oracle_rows():
    csr = synth.workload_graph("rmat20w", device="cuda")
    job = synth.WORKLOADS["rmat20w"]["job"]
    g = EFGraph.from_csr(csr, quantum=64)
    got = ef_walks(g, None, job.walk_len, job.walks_per_node, job.p, job.q, job.seed)
    gc = Graph.from_csr(csr)
    ref = walks(gc, None, job.walk_len, job.walks_per_node, job.p, job.q, job.seed)
    torch.cuda.synchronize()
    g.stream_status()
    assert torch.equal(got, ref)
    del ref
    gc.close()
    og = oracle.Graph(*csr.to("cpu").numpy())
    ids = np.random.default_rng(3).choice(got.shape[0], 2000, replace=False)
    want = oracle.walk_rows(og, None, job.walk_len, job.walks_per_node, job.p, job.q, job.seed,
                            ids)
    assert np.array_equal(got[torch.from_numpy(ids).cuda()].cpu().numpy(), want)


@pytest.mark.parametrize("quantum", [64, 1024])
def test_walks_shorter_row_search_equals_directed_search(quantum):
    # an undirected graph walked with membership tests in N(t) only (directed
    # reading) and with the shorter of N(t), N(x): the same rows, both the oracle's
    csr = synth.rmat(13, 120000, seed=23)
    for und in (False, True):
        g = EFGraph.from_csr(csr, quantum=quantum, undirected=und)
        assert g.info()["directory_rows"] == expected_directory_rows(csr) > 0
        for (p, q) in [(1.0, 0.25), (0.5, 2.0)]:
            check_walks(csr, None, 30, 1, p, q, seed=13, g=g)


def test_undirected_store_rejects_asymmetric_csr():
    off, dst = [0, 2, 3, 5], [1, 2, 0, 0, 1]          # 2 -> 1 without 1 -> 2
    EFGraph.from_csr(csr_np(off, dst), quantum=4, undirected=False)
    with pytest.raises(GrapeError, match="INVALID_GRAPH"):
        EFGraph.from_csr(csr_np(off, dst), quantum=4, undirected=True)
    # symmetric rows, unequal weights
    with pytest.raises(GrapeError, match="INVALID_GRAPH"):
        EFGraph.from_csr(csr_np([0, 1, 2], [1, 0], [1.0, 0.5]), quantum=4, undirected=True)


@pytest.mark.parametrize("bad", ["unsorted_row", "id_out_of_range", "multi_edge", "bad_offsets",
                                 "negative_weight"])
def test_invalid_csr_rejected(bad):
    off = [0, 2, 3, 5]
    dst = [1, 2, 0, 0, 1]
    w = None
    if bad == "unsorted_row":
        dst = [2, 1, 0, 0, 1]
    elif bad == "id_out_of_range":
        dst = [1, 3, 0, 0, 1]
    elif bad == "multi_edge":
        dst = [1, 1, 0, 0, 1]
    elif bad == "bad_offsets":
        off = [0, 3, 2, 5]
    elif bad == "negative_weight":
        w = [1.0, 0.5, -1.0, 0.3, 0.2]
    with pytest.raises(GrapeError, match="INVALID_GRAPH"):
        EFGraph.from_csr(csr_np(off, dst, w), quantum=4, undirected=False)
