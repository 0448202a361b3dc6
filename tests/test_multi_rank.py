"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1), each taking
its contiguous walk-id shard of a job N times the per-rank size (weak
scaling), with a barrier and a max of elapsed times as the only
communication.  The shards, computed per rank (here by the oracle, since this
host has no GPU), reassemble the whole job byte for byte: walks are pure
functions of (graph, walk id, seed), which is what lets grape_walks_range
shard a job with no data exchange."""
import importlib.util
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import _law

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def graph():
    n, e = _law.graph_house()
    w = [0.1 + 0.9 * ((7 * k + 3) % 11) / 10 for k in range(len(e))]
    return oracle.Graph(*_law.csr_from_edges(n, e, w, True))


def rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    bench = load_bench()
    d = bench.Dist(world)
    g = graph()
    wpn_per_rank, L = 6, 15
    total = g.num_nodes * wpn_per_rank * world          # weak scaling: fixed work per rank
    b, e = bench.shard(total, world, rank)
    rows, rc = oracle.walks(g, None, L, wpn_per_rank * world, 0.5, 2.0, seed=11,
                            walk_ids=(b, e))
    assert rc == 0
    d.barrier()
    m = d.max(float(rank + 1))                         # the bench's max over ranks
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), rows)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{b} {e} {m}\n")
    d.close()


def test_shards_cover_the_job_disjointly():
    bench = load_bench()
    for total in (1, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            spans = [bench.shard(total, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == total
            assert all(spans[r][1] == spans[r + 1][0] for r in range(world - 1))


def test_two_gloo_ranks_reassemble_the_job(tmp_path):
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=rank_main, args=(r, world, port, str(tmp_path)))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    parts, spans = [], []
    for r in range(world):
        parts.append(np.load(tmp_path / f"rank{r}.npy"))
        b, e, m = open(tmp_path / f"rank{r}.txt").read().split()
        spans.append((int(b), int(e)))
        assert float(m) == float(world)                # max over ranks seen by every rank
    g = graph()
    whole, rc = oracle.walks(g, None, 15, 6 * world, 0.5, 2.0, seed=11)
    assert rc == 0
    assert spans[0][0] == 0 and spans[1][0] == spans[0][1] and spans[1][1] == len(whole)
    assert np.array_equal(np.concatenate(parts), whole)
