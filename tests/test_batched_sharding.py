"""Splitting the batched workload across GPUs (host logic, on CPU).

The systems of a batch are independent, so N GPUs share one batch with no
exchange in the data path: the library's ebv_batch_partition pairs long
systems with short ones (Eq. 7's equalisation across systems) and hands the
pairs, longest first, to the least-loaded rank.  Checked here: every system
lands on exactly one rank, the ranks' costs are those of their systems and
stay within one pair's cost of the average, the split is the same on every
rank, and the one collective of the bench (putting the per-system info words
back in system order after the timed region) reassembles the batch.  Two
gloo ranks stand in for two GPUs.
"""
import importlib.util
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import paper_1907_05767_gb300 as ebv
import synthetic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1907_05767_gb300 import _build
    _build.build()
    return ebv.lib()


def _cost(ns, rs):
    ns = np.asarray(ns, dtype=np.float64)
    rs = np.asarray(rs, dtype=np.float64)
    return 2.0 * ns ** 3 / 3 + 2.0 * ns ** 2 * rs + 1.0


@pytest.mark.parametrize("nranks", [1, 2, 3, 8])
def test_partition_of_the_4096_system_batch(lib, nranks):
    ns, rs = synthetic.config3_sizes()
    rank_of, cost = ebv.ebv_batch_partition(ns, rs, nranks)
    assert rank_of.shape == ns.shape and rank_of.min() >= 0 and rank_of.max() < nranks
    c = _cost(ns, rs)
    for r in range(nranks):
        assert np.isclose(cost[r], c[rank_of == r].sum(), rtol=1e-12)
    # within one work item (at most the largest system) of the average
    assert cost.max() - cost.sum() / nranks <= c.max() * (1 + 1e-12)
    if nranks > 1:
        assert cost.max() / cost.min() < 1.01  # 4096 systems: the split is nearly even


def test_partition_small_cases_and_errors(lib):
    # more ranks than items: some ranks get nothing, no system is lost.  The
    # order-100 system is the most expensive, so nothing joins it; 50 and 10
    # form a pair (cheaper together than 100 alone) and stay on one rank.
    rank_of, cost = ebv.ebv_batch_partition([100, 10, 50], [1, 1, 1], 5)
    assert np.isclose(cost.sum(), _cost([100, 10, 50], [1, 1, 1]).sum())
    assert rank_of[1] == rank_of[2] != rank_of[0]
    assert np.count_nonzero(cost) == 2
    # equal systems round-robin over the ranks
    rank_of, cost = ebv.ebv_batch_partition([64] * 8, [2] * 8, 4)
    assert np.bincount(rank_of, minlength=4).tolist() == [2, 2, 2, 2]
    rank_of, cost = ebv.ebv_batch_partition([], [], 3)
    assert rank_of.size == 0 and np.all(cost == 0)
    with pytest.raises(ebv.EbvError):
        ebv.ebv_batch_partition([10], [1], 0)
    with pytest.raises(ebv.EbvError):
        ebv.ebv_batch_partition([5000], [1], 2)


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = _bench()
        ns, rs = synthetic.config3_sizes()
        idx, rank_of, cost = bench.shard_of_rank(ns, rs, world, rank)
        # the same split on every rank
        gathered = [None] * world
        dist.all_gather_object(gathered, rank_of.tolist())
        same = all(g == gathered[0] for g in gathered)
        # stand-in per-system results of this rank's share (what the GPU
        # writes into info): a value that names the system
        local = 1000 + idx.astype(np.int64)
        full = bench.gather_by_system(local, idx, len(ns), dist, "cpu")
        out[rank] = (same, idx.tolist(), full.tolist(), cost.tolist())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_split_the_batch_and_gather_in_system_order(lib, world):
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    ns, _ = synthetic.config3_sizes()
    assert all(out[r][0] for r in range(world))
    shares = [set(out[r][1]) for r in range(world)]
    assert sum(len(x) for x in shares) == len(ns)  # every system exactly once
    assert set().union(*shares) == set(range(len(ns)))
    want = [1000 + s for s in range(len(ns))]
    assert all(out[r][2] == want for r in range(world))
    c = out[0][3]
    assert max(c) / min(c) < 1.01
