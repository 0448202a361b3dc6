"""GPU context windows (grape_contexts_from_rows, grape_walk_contexts) against
the oracle's windows of the oracle's walks: bit-exact int32, for windows 1 to
64, short and long rows (the tiled and the direct kernel), dead ends, dead
starts, shards of a job, unaligned outputs, and the R-MAT scale-20 weighted
workload's graph on sampled rows."""
import numpy as np
import pytest
import torch

import oracle
import _law
from paper_2110_06196_gb300 import Graph, contexts, contexts_from_rows, synth

pytestmark = pytest.mark.gpu


def csr_from_np(off, dst, w=None):
    return synth.CSRGraph(torch.from_numpy(off), torch.from_numpy(dst),
                          None if w is None else torch.from_numpy(w), len(off) - 1)


def random_rows(rng, n, L, nodes=1000):
    rows = rng.integers(0, nodes, (n, L)).astype(np.int32)
    for r in range(n):
        if rng.random() < 0.4:
            rows[r, int(rng.integers(0, L + 1)):] = -1
    return rows


@pytest.mark.parametrize("window", [1, 2, 5, 17, 64])
@pytest.mark.parametrize("L", [1, 2, 7, 100, 2500])
def test_contexts_from_rows_match_the_oracle(window, L):
    rng = np.random.default_rng(window * 1000 + L)
    n = max(3, 60000 // (L * window))
    rows = random_rows(rng, n, L)
    got = contexts_from_rows(torch.from_numpy(rows).cuda(), window).cpu().numpy()
    assert np.array_equal(got, oracle.contexts(rows, window))


def test_unaligned_output_and_row_offsets():
    rng = np.random.default_rng(5)
    rows = random_rows(rng, 301, 13)
    want = oracle.contexts(rows, 3)
    buf = torch.full((301 * 13 * 6 + 1,), 7, dtype=torch.int32, device="cuda")
    out = buf[1:].view(301, 13, 6)                   # 4-byte aligned, not 16
    contexts_from_rows(torch.from_numpy(rows).cuda(), 3, out=out)
    assert np.array_equal(out.cpu().numpy(), want)
    assert int(buf[0]) == 7


@pytest.mark.parametrize("weighted", [False, True], ids=["unweighted", "weighted"])
def test_walk_contexts_equal_oracle_windows_of_oracle_walks(weighted):
    csr = synth.rmat(11, 20000, seed=9, weighted=weighted)
    g = Graph.from_csr(csr)
    og = oracle.Graph(*csr.numpy())
    starts = np.random.default_rng(2).integers(0, csr.num_nodes, 700).astype(np.int32)
    for (p, q, L, wpn, window) in [(0.5, 2.0, 30, 2, 4), (1.0, 0.25, 9, 1, 10), (2.0, 1.0, 1, 1, 3)]:
        rows_want, rc = oracle.walks(og, starts, L, wpn, p, q, seed=31)
        assert rc == 0
        cen, ctx = contexts(g, starts, L, wpn, p, q, 31, window=window, centres=True)
        assert np.array_equal(cen.cpu().numpy(), rows_want)
        assert np.array_equal(ctx.cpu().numpy(), oracle.contexts(rows_want, window))
        _, ctx2 = contexts(g, starts, L, wpn, p, q, 31, window=window)     # rows in scratch
        assert torch.equal(ctx, ctx2)


def test_shards_and_dead_ends():
    n, e = _law.graph_directed()
    csr = csr_from_np(*_law.csr_from_edges(n, e, None, False))
    g = Graph.from_csr(csr, undirected=False)
    og = oracle.Graph(*csr.numpy())
    rows_want, _ = oracle.walks(og, None, 12, 40, 0.5, 2.0, seed=4)
    want = oracle.contexts(rows_want, 3)
    total = rows_want.shape[0]
    parts = []
    for b in range(0, total, 37):
        c = min(37, total - b)
        _, ctx = contexts(g, None, 12, 40, 0.5, 2.0, 4, window=3, walk_begin=b, walk_count=c)
        parts.append(ctx.cpu().numpy())
    assert np.array_equal(np.concatenate(parts), want)
    assert (rows_want == -1).any()                   # the graph has a dead end


def test_rmat20w_graph_sampled_rows():
    csr = synth.workload_graph("rmat20w", device="cuda")
    g = Graph.from_csr(csr, validate=False)
    og = oracle.Graph(*csr.numpy())
    job = synth.WORKLOADS["rmat20w"]["job"]
    b, c = 3_000_000, 200_000
    _, ctx = contexts(g, None, job.walk_len, job.walks_per_node, job.p, job.q, job.seed,
                      window=5, walk_begin=b, walk_count=c)
    ids = np.random.default_rng(1).choice(c, 300, replace=False)
    rows = oracle.walk_rows(og, None, job.walk_len, job.walks_per_node, job.p, job.q, job.seed,
                            b + ids)
    got = ctx[torch.from_numpy(ids).cuda()].cpu().numpy()
    assert np.array_equal(got, oracle.contexts(rows, 5))
