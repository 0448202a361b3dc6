"""Approximated walks (grape_walks_approx, SUSS sub-sampling at nodes of degree
above k) against the oracle's approximated walks: bit-exact rows on small
graphs (weighted and unweighted, every class, trial caps 0, 2 and the
default), R-MAT scale 12, and sampled rows of the R-MAT scale-20 weighted
workload's graph; k >= the largest degree gives the exact walks."""
import numpy as np
import pytest
import torch

import oracle
import _law
from paper_2110_06196_gb300 import Graph, GrapeError, synth, walks, walks_approx

pytestmark = pytest.mark.gpu


def csr_from_np(off, dst, w=None):
    return synth.CSRGraph(torch.from_numpy(off), torch.from_numpy(dst),
                          None if w is None else torch.from_numpy(w), len(off) - 1)


def hub_csr(weighted):
    edges = [(0, x) for x in range(1, 8)] + [(1, 2), (1, 3), (2, 4), (5, 6)]
    w = [0.15 + 0.1 * k for k in range(len(edges))] if weighted else None
    return csr_from_np(*_law.csr_from_edges(8, edges, w, True))


def check(csr, starts, L, wpn, p, q, seed, k, cap=None, undirected=True):
    g = Graph.from_csr(csr, undirected=undirected)
    if cap is not None:
        g.set_tuning(trial_cap=cap)
    got = walks_approx(g, starts, L, wpn, p, q, seed, suss_k=k).cpu().numpy()
    og = oracle.Graph(*csr.numpy())
    want, rc = oracle.walks(og, starts, L, wpn, p, q, seed, suss_k=k,
                            trial_cap=g.get_tuning().trial_cap)
    assert rc == 0
    assert np.array_equal(got, want), np.argwhere((got != want).any(axis=1))[:5].ravel()


@pytest.mark.parametrize("weighted", [False, True], ids=["unweighted", "weighted"])
@pytest.mark.parametrize("cap", [None, 0, 2])
def test_hub_graph_all_pq(weighted, cap):
    csr = hub_csr(weighted)
    for (p, q) in [(0.5, 2.0), (2.0, 0.5), (1.0, 1.0), (4.0, 0.25)]:
        for k in (1, 2, 3, 6):
            check(csr, None, 15, 40, p, q, 17, k, cap)


@pytest.mark.parametrize("weighted", [False, True], ids=["unweighted", "weighted"])
def test_rmat12(weighted):
    csr = synth.rmat(12, 40000, seed=21, weighted=weighted)
    for (p, q, k) in [(0.5, 2.0, 8), (1.0, 0.25, 4), (2.0, 1.0, 16), (0.25, 4.0, 32)]:
        check(csr, None, 20, 2, p, q, 5, k)


def test_directed_graph():
    n, e = _law.graph_directed()
    csr = csr_from_np(*_law.csr_from_edges(n, e, [0.2 + 0.1 * j for j in range(len(e))], False))
    check(csr, None, 12, 30, 0.5, 2.0, 3, 1, undirected=False)


def test_large_k_is_the_exact_walk():
    csr = synth.rmat(12, 40000, seed=21, weighted=True)
    g = Graph.from_csr(csr)
    exact = walks(g, None, 25, 2, 0.5, 2.0, 7).cpu()
    for k in (0, int(np.diff(csr.offsets.numpy()).max())):
        assert torch.equal(walks_approx(g, None, 25, 2, 0.5, 2.0, 7, suss_k=k).cpu(), exact)
    with pytest.raises(GrapeError):
        walks_approx(g, None, 25, 2, 0.5, 2.0, 7, suss_k=-1)


def test_rmat20w_graph_sampled_rows():
    csr = synth.workload_graph("rmat20w", device="cuda")
    g = Graph.from_csr(csr, validate=False)
    og = oracle.Graph(*csr.numpy())
    job = synth.WORKLOADS["rmat20w"]["job"]
    rows = walks_approx(g, None, job.walk_len, 1, job.p, job.q, job.seed, suss_k=16)
    ids = np.random.default_rng(4).choice(rows.shape[0], 400, replace=False)
    got = rows[torch.from_numpy(ids).cuda()].cpu().numpy()
    want = np.stack([oracle.walks(og, None, job.walk_len, 1, job.p, job.q, job.seed,
                                  walk_ids=(int(w), int(w) + 1), suss_k=16)[0][0] for w in ids])
    assert np.array_equal(got, want)
