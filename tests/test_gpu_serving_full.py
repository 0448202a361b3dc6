"""The served path at its full size: the R-MAT scale-26 graph (2^30 undirected
edges, 2.1 G CSR entries) resident on the device, requests drawn as the
serving workload draws them (starts log-uniform in [1, 1e6], lengths uniform in
[20, 120], p and q from {0.25 .. 4}) arriving as a Poisson stream, admitted
under a 40 GB output cap.  All 50 requests are checked in full against the
CPU oracle (the oracle's walk ids split over the host cores, byte-identical to
its single-threaded run), and the server's device-counted transitions equal
the rows' own.
"""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2110_06196_gb300 import Graph, Server, synth

pytestmark = pytest.mark.gpu


def test_rmat26_served_requests_equal_oracle():
    csr = synth.workload_graph("rmat26", device="cuda")
    g = Graph.from_csr(csr, validate=False)
    host = csr.to("cpu").numpy()
    del csr
    torch.cuda.empty_cache()
    n = g.num_nodes
    mix = synth.request_mix(n, 50, gen_seed=2026, max_starts=1_000_000, len_lo=20, len_hi=120,
                            first_seed=70_000)
    arrivals = synth.poisson_arrivals(200.0, len(mix), seed=12)
    srv = Server(g, output_cap_bytes=40 << 30, max_inflight=4096, chunk_walks=0,
                 max_chunks=1 << 24, idle_exit_us=2000)
    tickets = {}
    t0 = time.perf_counter()
    for j, r in enumerate(mix):
        delay = arrivals[j] - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        tickets[srv.submit(r.starts, r.walk_len, r.p, r.q, r.seed)] = j
    got = {}
    while len(got) < len(mix):
        t, _, rows = srv.wait_any(timeout_ms=600_000)
        got[tickets[t]] = rows
    steps = srv.stats()["steps"]
    srv.close()
    og = oracle.Graph(*host)
    total = 0
    for j, r in enumerate(mix):
        rows = got[j]
        assert rows.shape == (len(r.starts), r.walk_len)
        want = oracle.walks_parallel(og, r.starts, r.walk_len, 1, r.p, r.q, r.seed)
        assert np.array_equal(rows, want), j
        total += int((rows >= 0).sum()) - int((rows[:, 0] >= 0).sum())
    assert steps == total
    g.close()
