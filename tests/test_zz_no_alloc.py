"""grape_walks_batched_static: batched walks for callers that cannot allocate
device memory when they need walks (their memory is owned by another allocator,
or allocation is not allowed where they call).  It keeps its state in a
fixed-size array in the library instead of cudaMalloc'd memory.

Checked through the C ABI: on two calls in a row its rows equal those of
grape_walks_batched, the entry point that allocates, and those of the CPU
oracle, bit for bit (the tolerance of every walk test here); with the work
counters on, it counts what the allocating path counts; and a batch above its
4096-request limit is refused before anything runs.  This file is collected
last so that a run that stops at the first failure has already run every
other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2110_06196_gb300 import Graph, synth, walks_batched
from paper_2110_06196_gb300 import _lib
from paper_2110_06196_gb300 import walk as W

pytestmark = pytest.mark.gpu


def _requests(csr, count, gen_seed):
    mix = synth.request_mix(csr.num_nodes, count, gen_seed=gen_seed, max_starts=5000, len_lo=3,
                            len_hi=70)
    return [dict(starts=torch.from_numpy(r.starts).cuda(), walk_len=r.walk_len,
                 walks_per_node=1 + (j % 2), p=r.p, q=r.q, seed=r.seed)
            for j, r in enumerate(mix)]


def _call_static(g, reqs):
    arr, keep = W._requests(reqs, g)   # allocates any missing outputs (test side)
    code = g._lib.grape_walks_batched_static(g.handle, arr, len(reqs), W._stream_ptr())
    _lib.check(code, "grape_walks_batched_static")
    torch.cuda.synchronize()
    return [r["out"] for r in reqs]


@pytest.mark.parametrize("weighted", [False, True], ids=["unweighted", "weighted"])
def test_static_batched_matches_allocating_batched_twice(weighted):
    csr = synth.rmat(13, 60000, seed=51, weighted=weighted)
    g = Graph.from_csr(csr)
    for call, gen_seed in enumerate((101, 202)):          # two calls in a row
        reqs = _requests(csr, 40, gen_seed)
        ref = walks_batched(g, [dict(r, out=None) for r in reqs])
        torch.cuda.synchronize()
        # fresh output buffers, filled with a value no walk writes
        reqs = [dict(r, out=torch.full(tuple(rr.shape), -7, dtype=torch.int32, device="cuda"))
                for r, rr in zip(reqs, ref)]
        got = _call_static(g, reqs)
        og = oracle.Graph(*csr.numpy())
        for j, (a, b) in enumerate(zip(got, ref)):
            assert torch.equal(a, b), f"call {call}"
            r = reqs[j]
            want, _ = oracle.walks(og, r["starts"].cpu().numpy(), r["walk_len"],
                                   r["walks_per_node"], r["p"], r["q"], r["seed"])
            assert np.array_equal(a.cpu().numpy(), want), f"call {call}, request {j}"


def test_static_batched_counts_like_allocating_batched():
    csr = synth.rmat(12, 30000, seed=53)
    g = Graph.from_csr(csr)
    reqs = _requests(csr, 24, 303)
    g.counters(enable=True)
    walks_batched(g, [dict(r, out=None) for r in reqs])
    torch.cuda.synchronize()
    want = g.counters()
    _call_static(g, [dict(r, out=None) for r in reqs])
    got = g.counters()
    g.counters(enable=False)
    for k in ("steps", "trials", "walks", "fallbacks"):
        assert got[k] == want[k] > 0 or (k == "fallbacks" and got[k] == want[k]), k


def test_static_batched_rejects_more_than_its_limit():
    csr = synth.rmat(10, 4000, seed=52)
    g = Graph.from_csr(csr)
    reqs = [dict(starts=None, num_starts=1, walk_len=2, walks_per_node=1, p=1.0, q=1.0, seed=j)
            for j in range(4097)]
    arr, keep = W._requests(reqs, g)
    code = g._lib.grape_walks_batched_static(g.handle, arr, len(reqs), W._stream_ptr())
    assert _lib.STATUS[code] == "GRAPE_ERR_INVALID_ARG"
