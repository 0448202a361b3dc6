"""GPU parity of grape_walks_cumsum (the paper's cumulative-sum sampler at every
step, through the C ABI) with the walk oracle run with trial_cap = 0, bit for
bit: tiny structured graphs over a (p, q) grid; R-MAT scale 12 weighted and
unweighted with powers of two for p and q (every row's sums exact, the warp's
shuffle scan) and with p, q that are not (products of 53 bits, sums in row
order); hub rows longer than the warp's product cache; ragged lengths, dead
and out-of-range starts, a directed graph; equality with grape_walks at
trial_cap = 0; and the R-MAT scale-20 weighted job, sampled.
"""
import numpy as np
import pytest
import torch

import oracle
import _law
from paper_2110_06196_gb300 import Graph, GrapeError, synth, walks, walks_cumsum

pytestmark = pytest.mark.gpu

PQ5 = (0.25, 0.5, 1.0, 2.0, 4.0)


def csr_np(off, dst, w=None):
    return synth.CSRGraph(torch.from_numpy(np.asarray(off, np.int64)),
                          torch.from_numpy(np.asarray(dst, np.int32)),
                          None if w is None else torch.from_numpy(np.asarray(w, np.float32)),
                          len(off) - 1)


def check(csr, starts, walk_len, wpn, p, q, seed, undirected=True, g=None):
    g = g or Graph.from_csr(csr, undirected=undirected)
    st = None if starts is None else torch.as_tensor(np.asarray(starts, np.int32))
    got = walks_cumsum(g, st, walk_len, wpn, p, q, seed)
    torch.cuda.synchronize()
    g.stream_status()
    got = got.cpu().numpy()
    og = oracle.Graph(*csr.numpy())
    want, rc = oracle.walks(og, None if starts is None else np.asarray(starts), walk_len, wpn, p,
                            q, seed, trial_cap=0)
    assert rc == 0
    if not np.array_equal(got, want):
        bad = np.argwhere((got != want).any(axis=1))[:, 0]
        raise AssertionError(f"{len(bad)} rows differ, first {bad[:5].tolist()}:\n"
                             f"gpu    {got[bad[0]].tolist()}\noracle {want[bad[0]].tolist()}")


def tiny():
    out = {}
    n, e = _law.graph_house()
    out["house"] = (csr_np(*_law.csr_from_edges(n, e, None, True)), True)
    wts = [0.1 + 0.9 * ((7 * k + 3) % 11) / 10 for k in range(len(e))]
    out["house_w"] = (csr_np(*_law.csr_from_edges(n, e, wts, True)), True)
    n, e = _law.graph_directed()
    out["directed"] = (csr_np(*_law.csr_from_edges(n, e, None, False)), False)
    wd = [0.2 + 0.15 * (k % 6) for k in range(len(e))]
    out["directed_w"] = (csr_np(*_law.csr_from_edges(n, e, wd, False)), False)
    out["star"] = (csr_np(*_law.csr_from_edges(9, [(0, i) for i in range(1, 9)])), True)
    kn = [(i, j) for i in range(8) for j in range(i + 1, 8)]
    out["k8"] = (csr_np(*_law.csr_from_edges(8, kn)), True)
    return out


@pytest.mark.parametrize("name", sorted(tiny()))
def test_tiny_graphs_all_pq(name):
    csr, und = tiny()[name]
    g = Graph.from_csr(csr, undirected=und)
    for p in PQ5:
        for q in PQ5:
            check(csr, None, 17, 9, p, q, seed=int(p * 100 + q * 10), g=g)


_RMAT12 = {}


def rmat12(weighted):
    if weighted not in _RMAT12:
        _RMAT12[weighted] = synth.rmat(12, 40000, seed=21, weighted=weighted)
    return _RMAT12[weighted]


@pytest.mark.parametrize("weighted", [False, True], ids=["unweighted", "weighted"])
def test_rmat12_exact_sums(weighted):
    csr = rmat12(weighted)
    assert int(np.diff(csr.numpy()[0]).max()) > 256          # rows beyond the product cache
    g = Graph.from_csr(csr)
    for (p, q) in [(1.0, 1.0), (0.5, 2.0), (4.0, 0.25), (0.25, 4.0), (2.0, 0.5)]:
        check(csr, None, 20, 2, p, q, seed=7, g=g)


@pytest.mark.parametrize("weighted", [False, True], ids=["unweighted", "weighted"])
def test_rmat12_sums_in_row_order(weighted):
    # 1/3, 1/0.7 and 1/1.3 are not powers of two: products carry 53 bits and
    # the cumulative sums round, so the warp adds in row order
    csr = rmat12(weighted)
    g = Graph.from_csr(csr)
    for (p, q) in [(3.0, 0.7), (0.7, 1.3), (1.0, 3.0)]:
        check(csr, None, 16, 1, p, q, seed=11, g=g)


def test_equals_rejection_path_with_trial_cap_zero():
    csr = synth.rmat(13, 120000, seed=23, weighted=True)
    g = Graph.from_csr(csr)
    g.set_tuning(trial_cap=0)
    for (p, q) in [(0.5, 2.0), (3.0, 0.7)]:
        a = walks(g, None, 30, 1, p, q, 5)
        b = walks_cumsum(g, None, 30, 1, p, q, 5)
        torch.cuda.synchronize()
        assert torch.equal(a, b)


def test_ragged_dead_and_bad_starts():
    csr = synth.rmat(11, 9000, seed=31)        # isolated nodes: dead starts
    g = Graph.from_csr(csr)
    rng = np.random.default_rng(2)
    starts = rng.integers(0, csr.num_nodes, 500).astype(np.int32)
    for L in (1, 2, 3, 33):
        for wpn in (1, 3):
            check(csr, starts, L, wpn, 0.5, 2.0, seed=L + wpn, g=g)
    st = torch.tensor([0, -1, 3, csr.num_nodes], dtype=torch.int32)
    out = walks_cumsum(g, st, 5, 1, 1.0, 0.5, 3).cpu().numpy()
    with pytest.raises(GrapeError):
        g.stream_status()
    assert (out[1] == -1).all() and (out[3] == -1).all()
    n, e = _law.graph_directed()
    check(csr_np(*_law.csr_from_edges(n, e, None, False)), None, 40, 5, 1.0, 0.5, 3,
          undirected=False)


def test_rmat20w_sampled():
    csr = synth.workload_graph("rmat20w", device="cuda")
    job = synth.WORKLOADS["rmat20w"]["job"]
    g = Graph.from_csr(csr)
    ids = np.random.default_rng(4).choice(csr.num_nodes * job.walks_per_node, 300, replace=False)
    # the rows of the sampled walk ids, from a job of 1 walk per start over those starts
    starts = (ids % csr.num_nodes).astype(np.int32)
    got = walks_cumsum(g, torch.from_numpy(starts), 40, 1, job.p, job.q, job.seed).cpu().numpy()
    og = oracle.Graph(*csr.to("cpu").numpy())
    want, rc = oracle.walks(og, starts, 40, 1, job.p, job.q, job.seed, trial_cap=0)
    assert rc == 0 and np.array_equal(got, want)
