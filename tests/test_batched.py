"""Batched factor + solve: the host schedule (CPU) and per-system parity with
the CPU oracle (GPU).  Tolerances: FP64 as the dense path (factors 1e-13, X
1e-11 relative, backward error 1e-14); FP32 factors 5e-5, X 1e-4 relative,
backward error 1e-5 (n * 2^-24 with margin, as for the dense FP32 path)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1907_05767_gb300 as ebv
import synthetic


@pytest.fixture(scope="module")
def lib():
    from paper_1907_05767_gb300 import _build
    _build.build()
    return ebv.lib()


def decode(sched):
    p = int(sched[0])
    items = sched[8:8 + 2 * p].reshape(p, 2)
    sys = np.where(items >= 0, items & ((1 << 28) - 1), -1)
    var = np.where(items >= 0, items >> 28, -1)
    return p, sys, var


def test_schedule_pairs_long_with_short(lib):
    ns, rs = synthetic.config3_sizes(1001)
    sched = ebv.ebv_batch_schedule(ns, rs)
    p, sys, var = decode(sched)
    assert sched[1] == 1001 and 501 <= p < 1001
    assert sys[:, 0].min() >= 0
    flat = sys[sys >= 0]
    assert sorted(flat.tolist()) == list(range(1001))  # every system exactly once
    cost = 2.0 * ns ** 3 / 3 + 2.0 * ns ** 2 * rs + 1
    pair_cost = np.where(sys >= 0, cost[np.maximum(sys, 0)], 0).sum(axis=1)
    assert np.all(np.diff(pair_cost) <= 0)  # items in decreasing cost
    assert pair_cost.max() <= cost.max()  # no item costs more than the largest system
    # the first slot of each pair holds the costlier system, the second the cheaper
    both = sys[:, 1] >= 0
    assert both.sum() > 200
    assert np.all(cost[sys[both, 0]] >= cost[sys[both, 1]])
    # pairing equalises: item costs spread far less than single-system costs
    assert pair_cost.max() / pair_cost.min() < (cost.max() / cost.min()) / 4
    # default variants: nb16 for n <= 64, nb32 above
    used = sys >= 0
    assert np.array_equal(var[used] == 0, ns[sys[used]] <= 64)


def test_schedule_equal_sizes_are_not_paired(lib):
    _, sys, _ = decode(ebv.ebv_batch_schedule([1024] * 256, [4] * 256))
    assert sys.shape[0] == 256 and np.all(sys[:, 1] == -1)


def test_schedule_variant_map_and_errors(lib):
    vmap = np.ones(4096, dtype=np.int8)
    sched = ebv.ebv_batch_schedule([10, 20, 30], [1, 1, 1], vmap)
    _, sys, var = decode(sched)
    assert np.all(var[sys >= 0] == 1)
    for bad in ([5000], [-1]):
        with pytest.raises(ebv.EbvError):
            ebv.ebv_batch_schedule(bad, [1])
    with pytest.raises(ebv.EbvError):
        ebv.ebv_batch_schedule([10], [65])
    assert int(lib.ebv_batch_schedule_len(0)) == 8
    assert int(lib.ebv_batch_schedule_len(5)) == 8 + 2 * 5


def fill(batch, seed_base, w=0.5):
    xs = []
    for s in range(batch.batch):
        n, r = int(batch.n[s]), int(batch.nrhs[s])
        a = synthetic.dense_dd(n, w, seed_base + s)
        x = synthetic.planted_x(n, r, seed_base + s)
        batch.a_view(s).copy_(torch.from_numpy(a))
        if r:
            batch.b_view(s).copy_(torch.from_numpy(synthetic.rhs_for(a, x)))
        xs.append((a, synthetic.rhs_for(a, x) if r else None))
    return xs


def check_system(batch, s, a, b, prec):
    tol_f, tol_x, tol_b = (1e-13, 1e-11, 1e-14) if prec == "fp64" else (5e-5, 1e-4, 1e-5)
    lu_ref, info_ref = oracle.lu(a)
    lu = batch.a_view(s).cpu().numpy().astype(np.float64)
    assert int(batch.info[s]) == info_ref
    assert np.abs(lu - lu_ref).max() <= tol_f, (s, np.abs(lu - lu_ref).max())
    if b is None:
        return
    x = batch.b_view(s).cpu().numpy().astype(np.float64)
    x_ref = oracle.solve(lu_ref, b)
    assert np.abs(x - x_ref).max() / np.abs(x_ref).max() <= tol_x
    r = oracle.residual(a, x, b)
    assert np.abs(r).max() / (np.abs(a).sum(axis=1).max() * np.abs(x).max()) <= tol_b


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_matches_oracle(prec):
    ns = [1, 2, 3, 15, 16, 17, 31, 32, 33, 63, 64, 65, 100, 129, 200, 257, 300, 5, 48, 96]
    rs = [1, 2, 4, 3, 1, 0, 2, 4, 1, 1, 3, 2, 4, 1, 2, 3, 1, 4, 2, 1]
    batch = ebv.Batch(ns, rs, prec)
    data = fill(batch, 123_000)
    batch.run()
    torch.cuda.synchronize()
    for s, (a, b) in enumerate(data):
        check_system(batch, s, a, b, prec)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5])
def test_batched_each_variant_matches_oracle(variant, prec):
    # every block width (16, 32, 64 in FP32) and tile edge (64, 32), on orders
    # that leave ragged blocks and tiles; in FP64 ids 2 and 5 run as id 1
    ns = [1, 7, 31, 40, 77, 129, 150, 300]
    rs = [1, 2, 1, 1, 3, 2, 4, 1]
    batch = ebv.Batch(ns, rs, prec, variant_of_n=np.full(4096, variant, dtype=np.int8))
    data = fill(batch, 322_000 + variant, w=0.9)
    batch.run()
    for s, (a, b) in enumerate(data):
        check_system(batch, s, a, b, prec)


@pytest.mark.gpu
@pytest.mark.parametrize("variant", [0, 1])
def test_batched_each_variant(variant):
    ns = [7, 40, 77, 150]
    rs = [2, 1, 3, 4]
    batch = ebv.Batch(ns, rs, "fp64", variant_of_n=np.full(4096, variant, dtype=np.int8))
    data = fill(batch, 321_000, w=0.9)
    batch.run()
    for s, (a, b) in enumerate(data):
        check_system(batch, s, a, b, "fp64")


@pytest.mark.gpu
def test_batched_zero_pivot_per_system():
    batch = ebv.Batch([20, 50, 33], [1, 1, 1], "fp64")
    data = fill(batch, 555)
    a = data[1][0].copy()
    k = 37
    a[k, :k] = 0.0
    a[:k, k] = 0.0
    a[k, k] = 0.0
    batch.a_view(1).copy_(torch.from_numpy(a))
    batch.run()
    info = batch.info.cpu().numpy()
    assert info[0] == 0 and info[2] == 0 and info[1] == k + 1


@pytest.mark.gpu
def test_batched_config3_sampled_and_graph_replay():
    # The 4096-system workload (n ~ U{16..512}, 1-4 RHS): every system's
    # residual is checked on the GPU side against its own b through the oracle
    # for a seeded sample, all info words must be 0, and a CUDA-graph replay
    # must reproduce the direct call bit for bit.
    ns, rs = synthetic.config3_sizes()
    batch = ebv.Batch(ns, rs, "fp64")
    pick = synthetic.pick_indices(99, 24, [len(ns)])[:, 0]
    data = {}
    for s in range(batch.batch):
        n, r = int(ns[s]), int(rs[s])
        a, x, b = synthetic.config3_system(s, n, r)
        batch.a_view(s).copy_(torch.from_numpy(a))
        batch.b_view(s).copy_(torch.from_numpy(b))
        if s in set(pick.tolist()):
            data[s] = (a, b)
    a0, b0 = batch.a_buf.clone(), batch.b_buf.clone()
    batch.run()
    torch.cuda.synchronize()
    assert int(batch.info.abs().max()) == 0
    for s, (a, b) in data.items():
        check_system(batch, s, a, b, "fp64")
    first_a, first_b = batch.a_buf.clone(), batch.b_buf.clone()
    g = torch.cuda.CUDAGraph()
    batch.a_buf.copy_(a0)
    batch.b_buf.copy_(b0)
    with torch.cuda.graph(g):
        batch.run()
    batch.a_buf.copy_(a0)
    batch.b_buf.copy_(b0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(batch.a_buf, first_a) and torch.equal(batch.b_buf, first_b)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_autotune_returns_valid_variants(tmp_path, prec):
    vmap, ms = ebv.batch_autotune([16, 100, 300], prec, reps=8, cache_path=str(tmp_path / "tune.json"))
    offered = {0, 1, 2, 3, 4, 5} if prec == "fp32" else {0, 1, 3, 4}
    assert vmap.shape == (4096,) and set(np.unique(vmap).tolist()) <= offered
    assert set(ms) == {16, 100, 300}
    for v in ms.values():  # a time for every offered variant, -1 for the others
        assert len(v) == 6
        assert all((t > 0) == (i in offered) for i, t in enumerate(v))
    # the chosen variant is the fastest one timed
    for o, v in ms.items():
        assert v[vmap[o - 1]] == min(t for t in v if t > 0)
    vmap2, _ = ebv.batch_autotune([16, 100, 300], prec, reps=8, cache_path=str(tmp_path / "tune.json"))
    assert np.array_equal(vmap, vmap2)  # served from the cache


@pytest.mark.gpu
def test_autotune_buckets_cover_the_batched_orders(tmp_path):
    vmap, table = ebv.batch_autotune_buckets("fp32", reps=16, cache_path=str(tmp_path / "tune.json"))
    assert sorted(table) == [32, 64, 96, 128, 160, 192, 224, 256, 288, 320, 352, 384, 416, 448, 480, 512]
    for mid, row in table.items():  # every order of a bucket takes its middle order's choice
        assert row["best"] == ebv.BATCH_VARIANTS[int(vmap[mid - 1])]
    assert vmap[16 - 1] == vmap[32 - 1] and vmap[47 - 1] == vmap[32 - 1]
