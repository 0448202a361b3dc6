"""Continuous-batching server: every request's rows equal the same request run
alone through grape_walks (and the oracle on samples), whatever else is in
flight; admission by output bytes queues requests that do not fit yet; the
resident kernel's bounded idle wait runs out and it is relaunched; cancel,
timeouts, oversize requests and shutdown with work in flight."""
import threading
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2110_06196_gb300 import GrapeError, Graph, Server, synth, walks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def graph():
    csr = synth.rmat(14, 120000, seed=41, weighted=False)
    return csr, Graph.from_csr(csr)


def _alone(g, starts, L, p, q, seed, wpn=1):
    return walks(g, torch.from_numpy(starts).cuda(), L, wpn, p, q, seed).cpu().numpy()


def test_mixed_stream_equals_alone_and_oracle(graph):
    csr, g = graph
    mix = synth.request_mix(csr.num_nodes, 120, gen_seed=3, max_starts=20000, len_lo=5,
                            len_hi=90)
    srv = Server(g, output_cap_bytes=256 << 20, max_inflight=64, chunk_walks=32,
                 idle_exit_us=500)
    arrivals = synth.poisson_arrivals(2000.0, len(mix), seed=9)
    tickets = {}
    t0 = time.perf_counter()
    for j, r in enumerate(mix):
        while time.perf_counter() - t0 < arrivals[j]:
            time.sleep(0.0002)
        tickets[srv.submit(r.starts, r.walk_len, r.p, r.q, r.seed)] = j
    got = {}
    lat = []
    while len(got) < len(mix):
        t, l, rows = srv.wait_any(timeout_ms=60000)
        got[tickets[t]] = rows
        lat.append(l)
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(mix) and st["inflight"] == 0
    # the server's device-side count of transitions equals the rows' own
    assert st["steps"] == sum(int((got[j] >= 0).sum()) - int((got[j][:, 0] >= 0).sum())
                              for j in range(len(mix)))
    og = oracle.Graph(*csr.numpy())
    for j, r in enumerate(mix):
        assert np.array_equal(got[j], _alone(g, r.starts, r.walk_len, r.p, r.q, r.seed)), j
        if j % 10 == 0:
            ids = np.arange(min(3, len(r.starts)))
            want = oracle.walk_rows(og, r.starts, r.walk_len, 1, r.p, r.q, r.seed, ids)
            assert np.array_equal(got[j][ids], want)
    assert all(x > 0 for x in lat)


def test_admission_by_output_bytes(graph):
    csr, g = graph
    L = 50
    per = 20000 * L * 4                       # 4 MB of rows per request
    srv = Server(g, output_cap_bytes=3 * per, max_inflight=16, chunk_walks=64)
    rng = np.random.default_rng(1)
    reqs = [rng.integers(0, csr.num_nodes, 20000).astype(np.int32) for _ in range(12)]
    ts = [srv.submit(s, L, 0.5, 2.0, 100 + j) for j, s in enumerate(reqs)]
    peak = 0
    for _ in range(2000):
        st = srv.stats()
        peak = max(peak, st["bytes_reserved"])
        if st["completed"] == len(reqs):
            break
        time.sleep(0.001)
    outs = [srv.wait(t, timeout_ms=60000) for t in ts]
    srv.close()
    assert peak <= 3 * per + 3 * 256 * 4
    for j, (s, o) in enumerate(zip(reqs, outs)):
        assert np.array_equal(o, _alone(g, s, L, 0.5, 2.0, 100 + j))


def test_oversize_request_is_rejected(graph):
    csr, g = graph
    srv = Server(g, output_cap_bytes=1 << 20, max_inflight=4)
    with pytest.raises(GrapeError) as ei:
        srv.submit(np.zeros(100000, np.int32), 10, 1.0, 1.0, 0)
    assert ei.value.name == "GRAPE_ERR_NOMEM"
    srv.close()


def test_idle_exit_and_relaunch(graph):
    csr, g = graph
    srv = Server(g, output_cap_bytes=64 << 20, max_inflight=8, idle_exit_us=200)
    s = np.arange(500, dtype=np.int32)
    a = srv.wait(srv.submit(s, 20, 2.0, 0.5, 1), timeout_ms=30000)
    time.sleep(0.05)                     # the server stops the idle resident kernel
    b = srv.wait(srv.submit(s, 20, 2.0, 0.5, 2), timeout_ms=30000)
    st = srv.stats()
    srv.close()
    assert st["kernel_launches"] >= 2
    assert np.array_equal(a, _alone(g, s, 20, 2.0, 0.5, 1))
    assert np.array_equal(b, _alone(g, s, 20, 2.0, 0.5, 2))


def test_cancel_timeout_and_shutdown(graph):
    csr, g = graph
    srv = Server(g, output_cap_bytes=8 << 20, max_inflight=2, chunk_walks=16)
    big = np.random.default_rng(2).integers(0, csr.num_nodes, 30000).astype(np.int32)
    t1 = srv.submit(big, 60, 0.25, 4.0, 5)
    t2 = srv.submit(big, 60, 0.25, 4.0, 6)      # waits for memory behind t1
    t3 = srv.submit(big[:10], 5, 1.0, 1.0, 7)
    srv.cancel(t2)
    with pytest.raises(GrapeError) as ei:
        srv.wait(t2, timeout_ms=60000)
    assert ei.value.name == "GRAPE_ERR_CANCELLED"
    with pytest.raises(GrapeError) as ei:
        srv.wait(999999, timeout_ms=0)
    assert ei.value.name == "GRAPE_ERR_NOT_FOUND"
    r1 = srv.wait(t1, timeout_ms=60000)
    assert np.array_equal(r1, _alone(g, big, 60, 0.25, 4.0, 5))
    r3 = srv.wait(t3, timeout_ms=60000)
    assert np.array_equal(r3, _alone(g, big[:10], 5, 1.0, 1.0, 7))
    # shutdown with work still queued and running
    for j in range(6):
        srv.submit(big, 60, 0.5, 2.0, 50 + j)
    srv.close()


def test_concurrent_submitters(graph):
    csr, g = graph
    srv = Server(g, output_cap_bytes=128 << 20, max_inflight=32, chunk_walks=32)
    results = {}
    errors = []

    def client(k):
        try:
            rng = np.random.default_rng(k)
            for j in range(6):
                s = rng.integers(0, csr.num_nodes, int(rng.integers(1, 4000))).astype(np.int32)
                t = srv.submit(s, 25, 1.0, 0.5, 1000 * k + j)
                results[(k, j)] = (s, srv.wait(t, timeout_ms=60000))
        except Exception as e:  # pragma: no cover
            errors.append(e)

    th = [threading.Thread(target=client, args=(k,)) for k in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    srv.close()
    assert not errors
    for (k, j), (s, rows) in results.items():
        assert np.array_equal(rows, _alone(g, s, 25, 1.0, 0.5, 1000 * k + j))


def test_burst_larger_than_the_entry_stage_keeps_one_kernel(graph):
    """One burst whose queue entries exceed the host staging of a single copy
    (2^18 entries): the server publishes it in pieces without synchronising the
    device, so the resident kernel never runs out of work and is launched
    once; rows equal the requests run alone."""
    csr, g = graph
    rng = np.random.default_rng(12)
    reqs = [(rng.integers(0, csr.num_nodes, n).astype(np.int32), 6, 0.5, 2.0, 100 + j)
            for j, n in enumerate((300000, 5000, 70000))]
    srv = Server(g, output_cap_bytes=1 << 30, max_inflight=16, chunk_walks=1,
                 max_chunks=1 << 20, idle_exit_us=200000)
    t0 = time.perf_counter()
    tickets = [srv.submit(st, L, p, q, seed) for (st, L, p, q, seed) in reqs]
    got = [srv.wait(t, timeout_ms=60000) for t in tickets]
    elapsed = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    assert st["kernel_launches"] == 1, st
    assert elapsed < 1.5, elapsed        # the kernel's idle bound is about 2 s
    for (starts, L, p, q, seed), rows in zip(reqs, got):
        assert np.array_equal(rows, _alone(g, starts, L, p, q, seed))


def test_held_rows_reuse_slots(graph):
    """Requests submitted without a host buffer keep their rows in the device
    arena until wait (or wait_any) hands them over; with two slots, every later
    request reuses the slot of a retired one.  Rows equal the requests alone."""
    csr, g = graph
    rng = np.random.default_rng(4)
    reqs = [(rng.integers(0, csr.num_nodes, int(rng.integers(1, 3000))).astype(np.int32),
             int(rng.integers(2, 40)), float(rng.choice([0.25, 1.0, 4.0])),
             float(rng.choice([0.5, 1.0, 2.0])), 500 + j) for j in range(24)]
    srv = Server(g, output_cap_bytes=64 << 20, max_inflight=2, chunk_walks=0,
                 idle_exit_us=1000)
    got = {}
    for j in range(0, len(reqs), 4):
        batch = reqs[j:j + 4]
        tks = [srv.submit(st, L, p, q, seed, hold=True) for (st, L, p, q, seed) in batch]
        for k, t in enumerate(tks[:2]):
            got[j + k] = srv.wait(t, timeout_ms=60000)
        for _ in range(2):
            t, _, rows = srv.wait_any(timeout_ms=60000)
            got[j + 2 + tks[2:].index(t)] = rows
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["inflight"] == 0
    for j, (starts, L, p, q, seed) in enumerate(reqs):
        assert np.array_equal(got[j], _alone(g, starts, L, p, q, seed)), j


def test_requests_around_the_idle_exit(graph):
    """Requests arriving just before, at and after the moment the server stops
    an idle resident kernel: each is served by the leaving kernel or by the
    next one, never lost, and its rows equal the request alone."""
    csr, g = graph
    srv = Server(g, output_cap_bytes=64 << 20, max_inflight=8, idle_exit_us=300)
    rng = np.random.default_rng(8)
    got = []
    for j in range(40):
        st = rng.integers(0, csr.num_nodes, int(rng.integers(1, 200))).astype(np.int32)
        got.append((st, srv.wait(srv.submit(st, 12, 1.0, 0.5, 900 + j), timeout_ms=30000)))
        time.sleep(float(rng.uniform(0.0, 0.005)))   # the driver looks every <= 2 ms
    s = srv.stats()
    srv.close()
    assert s["completed"] == 40 and s["kernel_launches"] >= 2, s
    for j, (st, rows) in enumerate(got):
        assert np.array_equal(rows, _alone(g, st, 12, 1.0, 0.5, 900 + j)), j


def test_kernel_wait_runs_out_without_heartbeat(graph):
    """The resident kernel's own bounded wait: with the host heartbeat stopped
    (a host that no longer answers, injected on the host side), every idle warp
    gives up after kernel_wait_ms, raises bit 2 of the graph's status word and
    leaves.  The server counts the timed-out launch, and the next request
    relaunches the kernel and comes back equal to the oracle's rows."""
    csr, g = graph
    try:                                               # start from a clear status word
        g.stream_status()
    except GrapeError:
        pass
    og = oracle.Graph(*csr.numpy())
    srv = Server(g, output_cap_bytes=64 << 20, max_inflight=8, idle_exit_us=60_000_000,
                 kernel_wait_ms=50)
    try:
        starts = np.arange(0, csr.num_nodes, 97, dtype=np.int32)
        a = srv.wait(srv.submit(starts, 21, 0.5, 2.0, 123), timeout_ms=30000)
        want, _ = oracle.walks(og, starts, 21, 1, 0.5, 2.0, 123)
        assert np.array_equal(a, want)
        st = srv.stats()
        assert st["kernel_launches"] == 1 and st["kernel_timeouts"] == 0
        srv.inject_fault(no_heartbeat=True)
        deadline = time.time() + 20
        while srv.stats()["kernel_timeouts"] == 0 and time.time() < deadline:
            time.sleep(0.01)
        assert srv.stats()["kernel_timeouts"] == 1
        with pytest.raises(GrapeError) as ei:             # status bit 2 is up
            g.stream_status()
        assert ei.value.name == "GRAPE_ERR_DEVICE"
        srv.inject_fault(no_heartbeat=False)
        starts2 = np.arange(5, csr.num_nodes, 61, dtype=np.int32)
        b = srv.wait(srv.submit(starts2, 33, 2.0, 0.25, 456), timeout_ms=30000)
        want2, _ = oracle.walks(og, starts2, 33, 1, 2.0, 0.25, 456)
        assert np.array_equal(b, want2)
        st = srv.stats()
        assert st["kernel_launches"] == 2 and st["kernel_timeouts"] == 1
    finally:
        srv.close()
    g.stream_status()                                  # nothing else was raised
