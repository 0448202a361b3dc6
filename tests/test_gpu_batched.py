"""Batched walks (one persistent launch replayed from a CUDA graph): each
request's rows are byte-identical to the per-call path and to the oracle, for
any queue granularity and search threshold, and on the 512-request mix (every
request in full against the oracle) over the
R-MAT scale-20 weighted graph."""
import numpy as np
import pytest
import torch

import oracle
from paper_2110_06196_gb300 import BatchPlan, Graph, autotune_batched, synth, walks, walks_batched

pytestmark = pytest.mark.gpu


def _reqs_from_mix(mix, wpn=1):
    return [dict(starts=torch.from_numpy(r.starts).cuda(), walk_len=r.walk_len, walks_per_node=wpn,
                 p=r.p, q=r.q, seed=r.seed) for r in mix]


def _per_call(g, r):
    return walks(g, r["starts"], r["walk_len"], r.get("walks_per_node", 1), r["p"], r["q"], r["seed"])


@pytest.fixture(scope="module")
def small():
    csr = synth.rmat(13, 60000, seed=31, weighted=True)
    return csr, Graph.from_csr(csr)


def test_batched_equals_per_call_and_oracle(small):
    csr, g = small
    mix = synth.request_mix(csr.num_nodes, 40, gen_seed=5, max_starts=3000, len_lo=1, len_hi=60)
    reqs = _reqs_from_mix(mix, wpn=2)
    # a request with no start list (all nodes) too
    reqs.append(dict(starts=None, num_starts=csr.num_nodes, walk_len=7, walks_per_node=1,
                     p=2.0, q=0.5, seed=77))
    outs = walks_batched(g, reqs)
    torch.cuda.synchronize()
    g.stream_status()
    og = oracle.Graph(*csr.numpy())
    for r, o in zip(reqs, outs):
        alone = _per_call(g, r)
        assert torch.equal(o, alone)
        st = None if r["starts"] is None else r["starts"].cpu().numpy()
        want, _ = oracle.walks(og, st, r["walk_len"], r["walks_per_node"], r["p"], r["q"], r["seed"])
        assert np.array_equal(o.cpu().numpy(), want)


@pytest.mark.parametrize("chunk", [1, 7, 64, 1000])
@pytest.mark.parametrize("shorter_min", [0, 16, 0x7fffffff])
@pytest.mark.parametrize("hub", [(0x7fffffff, 0x7fffffff), (32, 0x7fffffff), (0x7fffffff, 32)],
                         ids=["plain", "pivots32", "warp32"])
def test_batched_independent_of_granularity(small, chunk, shorter_min, hub):
    csr, g = small
    mix = synth.request_mix(csr.num_nodes, 16, gen_seed=6, max_starts=2000, len_lo=5, len_hi=40)
    g.set_tuning(pivot_min=0x7fffffff, warp_search_min=0x7fffffff)
    ref = [_per_call(g, r) for r in _reqs_from_mix(mix)]
    g.set_tuning(chunk_walks=chunk, shorter_min=shorter_min, pivot_min=hub[0],
                 warp_search_min=hub[1])
    try:
        reqs = _reqs_from_mix(mix)
        plan = BatchPlan(g, reqs)
        for _ in range(2):          # replay the captured graph
            for r in reqs:
                r["out"].fill_(-7)
            plan.launch()
            torch.cuda.synchronize()
            for a, b in zip(plan.outputs(), ref):
                assert torch.equal(a, b)
        plan.close()
    finally:
        g.set_tuning(chunk_walks=64, shorter_min=8, pivot_min=0x7fffffff,
                     warp_search_min=0x7fffffff)


def test_autotune_picks_a_grid_point_and_keeps_bytes(small):
    csr, g = small
    mix = synth.request_mix(csr.num_nodes, 24, gen_seed=8, max_starts=4000, len_lo=10, len_hi=50)
    reqs = _reqs_from_mix(mix)
    ref = [_per_call(g, r) for r in reqs]
    best = autotune_batched(g, reqs)
    assert best["chunk_walks"] in (16, 32, 64, 128, 256)
    assert best["pivot_min"] in (0x7fffffff, 32, 128, 512, 2048)
    assert best["warp_search_min"] in (0x7fffffff, 1024, 8192)
    t = g.get_tuning()
    assert (t.chunk_walks, t.pivot_min, t.warp_search_min) == \
        (best["chunk_walks"], best["pivot_min"], best["warp_search_min"])
    outs = walks_batched(g, _reqs_from_mix(mix))
    for a, b in zip(outs, ref):
        assert torch.equal(a, b)


def test_rmat20_512_request_mix():
    csr = synth.workload_graph("rmat20w", device="cuda")
    g = Graph.from_csr(csr, validate=False)
    mix = synth.request_mix(csr.num_nodes, 512, gen_seed=1234, max_starts=100_000, len_lo=10,
                            len_hi=200)
    reqs = _reqs_from_mix(mix)
    plan = BatchPlan(g, reqs)
    plan.launch()
    torch.cuda.synchronize()
    g.stream_status()
    outs = plan.outputs()
    og = oracle.Graph(*csr.numpy())
    checked = 0
    for j, (r, o) in enumerate(zip(mix, outs)):
        if j % 8 == 0:      # every 8th request also against the per-call path
            assert torch.equal(o, walks(g, reqs[j]["starts"], r.walk_len, 1, r.p, r.q, r.seed))
        # every request in full against the oracle (its walk ids over the host cores)
        want = oracle.walks_parallel(og, r.starts, r.walk_len, 1, r.p, r.q, r.seed)
        assert np.array_equal(o.cpu().numpy(), want), j
        checked += len(r.starts)
    assert checked == sum(len(r.starts) for r in mix)
    plan.close()
