"""Row sharding across ranks (host logic; CPU, gloo): contiguous row ranges
balanced by cell count, sharded workloads that reassemble the original, and a
world-size-2 run in which every rank steps its own rows (the FP64 oracle stands
in for the GPU step) with only scalar reductions between ranks: the gathered
rows equal the single-process result bit for bit and the global mass is
conserved (Eq. 10)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2305_05362_gb300 import shard, workloads as wl


def test_partition_covers_rows_and_balances_cells():
    rng = np.random.default_rng(3)
    for trial in range(40):
        n_rows = int(rng.integers(1, 60))
        lens = rng.integers(1, 5000, n_rows)
        ro = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        for world in (1, 2, 3, 4, 7, 8):
            parts = shard.partition_rows(ro, world)
            assert len(parts) == world
            assert parts[0][0] == 0 and parts[-1][1] == n_rows
            for (a, b), (c, d) in zip(parts, parts[1:]):
                assert b == c and a <= b
            cells = [int(ro[b] - ro[a]) for a, b in parts]
            assert sum(cells) == int(ro[-1])
            ideal = ro[-1] / world
            # whole rows: no rank exceeds the ideal share by more than one row
            assert max(cells) <= ideal + lens.max() + 1, (world, cells, ideal)


def test_partition_more_ranks_than_rows():
    ro = np.array([0, 10, 30], dtype=np.int64)
    parts = shard.partition_rows(ro, 5)
    assert sum(b - a for a, b in parts) == 2
    assert all(a <= b for a, b in parts)


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_shards_reassemble_the_workload(world):
    w = wl.batched(n_rows=23, n_max=3000, seed_len=4)
    parts = [shard.shard_workload(w, k, world) for k in range(world)]
    assert sum(p.n_rows for p in parts) == w.n_rows
    assert np.array_equal(np.concatenate([p.q0 for p in parts]), w.q0)
    assert np.array_equal(np.concatenate([p.v0 for p in parts]), w.v0)
    assert np.array_equal(np.concatenate([p.order for p in parts]), w.order)
    r = 0
    for p in parts:
        for rr in range(p.n_rows):
            assert np.array_equal(p.row_nodes(rr), w.row_nodes(r + rr))
            assert np.array_equal(p.q0[p.row_slice(rr)], w.q0[w.row_slice(r + rr)])
        r += p.n_rows


def _oracle_steps(w, steps):
    q = w.q0.copy()
    shifts = [oracle.shift_from_velocity(w.v0[r], w.dt) for r in range(w.n_rows)]
    for _ in range(steps):
        out = np.empty_like(q)
        for r in range(w.n_rows):
            sl = w.row_slice(r)
            dv = None if w.dv is None else w.dv[sl]
            out[sl] = oracle.step(w.row_nodes(r), q[sl], shifts[r], int(w.order[r]), w.limiter,
                                  dv, w.dt, w.scheme, int(w.nsub[r]))
        q = out
    return q


def _mass(w, q):
    return sum(oracle.mass(w.row_nodes(r), q[w.row_slice(r)]) for r in range(w.n_rows))


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = wl.disk(n_r=12, n_phi=256, seed_dv=4)
        mine = shard.shard_workload(w, rank, world)
        m0 = shard.global_sum(_mass(mine, mine.q0))
        q = _oracle_steps(mine, 3)
        m1 = shard.global_sum(_mass(mine, q))
        t = shard.global_max(float(rank + 1))
        np.save(os.path.join(out_dir, "q%d.npy" % rank), q)
        np.save(os.path.join(out_dir, "s%d.npy" % rank), np.array([m0, m1, t]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_gloo_match_single_process(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    w = wl.disk(n_r=12, n_phi=256, seed_dv=4)
    ref = _oracle_steps(w, 3)
    got = np.concatenate([np.load(tmp_path / ("q%d.npy" % k)) for k in range(world)])
    assert np.array_equal(got, ref)
    m_ref0, m_ref1 = _mass(w, w.q0), _mass(w, ref)
    for k in range(world):
        m0, m1, t = np.load(tmp_path / ("s%d.npy" % k))
        assert abs(m0 - m_ref0) <= 1e-13 * abs(m_ref0)
        assert abs(m1 - m_ref1) <= 1e-13 * abs(m_ref1)
        assert abs(m1 - m0) <= 1e-12 * abs(m0)
        assert t == float(world)
