"""Batch sharding of one system across ranks (host logic on CPU): the shards
of mlcc3_shard_batches partition the unique batches with balanced costs, and
two gloo ranks that each compute Omega, rho and sigma over their shard (the
oracle's batched form standing in for the GPU) and all-reduce the outputs get
the single-rank result."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2202_08612_gb300 import binding, build  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


@pytest.mark.parametrize("no,count", [(5, 2), (12, 3), (20, 8), (3, 16)])
def test_shards_partition_the_batches(no, count):
    full = [(i, j, k) for i in range(no) for j in range(i + 1) for k in range(j + 1)
            if not (i == j == k)]
    got = [binding.shard_batches(no, None, False, count, q) for q in range(count)]
    assert sorted(sum(got, [])) == sorted(full)
    assert len(set(sum(got, []))) == len(full)
    cost = [sum(6 if (i != j and j != k) else 3 for i, j, k in g) for g in got]
    assert max(cost) - min(cost) <= 6
    for g in got:   # each shard keeps the list order
        assert g == [t for t in full if t in set(g)]


def test_cvs_shards_hold_core_batches_only():
    mask = np.zeros(6, dtype=np.uint8)
    mask[0] = 1
    got = sum((binding.shard_batches(6, mask, True, 2, q) for q in range(2)), [])
    assert got and all(0 in t for t in got)
    assert len(got) == sum(1 for i in range(6) for j in range(i + 1) for k in range(j + 1)
                           if not (i == j == k) and 0 in (i, j, k))
    with pytest.raises(binding.MLCC3Error):
        binding.shard_batches(6, mask, True, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from oracle import batched as B
    from paper_2202_08612_gb300 import binding as bd, shard, synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = synth.make_system(5, 9, 4, 4, 12, seed=31)
        st = synth.make_states(s, 1, seed=32)
        b = B.make_bctx(s)
        mine = bd.shard_batches(4, None, False, world, rank)
        w = float(st.omega[0])
        parts = list(B.triples_omega(b, mine)) + list(B.jacobian_right(b, w, st.R1[0], st.R2[0], mine)) \
            + list(B.jacobian_left(b, w, st.L1[0], st.L2[0], mine))
        ts = [torch.from_numpy(np.ascontiguousarray(p)) for p in parts]
        shard.allreduce_sum(ts)
        if rank == 0:
            out["sharded"] = [t.numpy() for t in ts]
            out["full"] = list(B.triples_omega(b)) + list(B.jacobian_right(b, w, st.R1[0], st.R2[0])) \
                + list(B.jacobian_left(b, w, st.L1[0], st.L2[0]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_to_the_single_rank_result():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for x, y in zip(res["sharded"], res["full"]):
        assert np.abs(y).max() > 1e-8
        assert np.abs(x - y).max() <= 1e-13 * np.abs(y).max()
