"""The FP64 panels' two diagonal-block kernels (the register-resident one,
default, and the blocked 16 x 16 sub-block one behind
ebv_debug_set_diag_lu(0)) against the CPU oracle.

They factor the 64 x 64 diagonal block of every panel of the banded
factorisations and of dense FP64 systems of order <= 256.  Cases: blocks
narrower than 64 (the last panel), pivots at every position class of the
register layout (slot boundaries 15/16, the last row), zero pivots reported at
the same index by both kernels, and planted few-bit factors that every
summation order must reproduce bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1907_05767_gb300 as ebv
import synthetic

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture
def diag_kernel():
    lib = ebv.lib()
    yield lambda on: lib.ebv_debug_set_diag_lu(1 if on else 0)
    lib.ebv_debug_set_diag_lu(1)


@pytest.mark.parametrize("n", [1, 2, 17, 64, 65, 100, 200, 256])
def test_dense_small_both_kernels(diag_kernel, n):
    a = synthetic.dense_dd(n, 0.9, 91_000 + n)
    b = synthetic.rhs_for(a, synthetic.planted_x(n, 2, 91_100 + n))
    lu_ref, _ = oracle.lu(a)
    x_ref = oracle.solve(lu_ref, b)
    out = {}
    for on in (True, False):
        diag_kernel(on)
        f = ebv.factor(torch.from_numpy(a).to(DEV), "fp64")
        x = ebv.solve(f, torch.from_numpy(b).to(DEV)).cpu().numpy()
        lu = f.lu.cpu().numpy()
        assert int(f.info.item()) == 0
        assert np.abs(lu - lu_ref).max() <= 1e-13, on
        assert np.abs(x - x_ref).max() / np.abs(x_ref).max() <= 1e-11
        out[on] = lu
    assert np.abs(out[True] - out[False]).max() <= 2e-13


@pytest.mark.parametrize("n,kl,ku", [(300, 3, 70), (500, 90, 5), (257, 64, 64), (700, 130, 200), (129, 0, 0)])
def test_band_both_kernels(diag_kernel, n, kl, ku):
    a = synthetic.dense_dd(n, 0.9, 92_000 + n + kl)
    d = np.subtract.outer(np.arange(n), np.arange(n))
    a[(d > kl) | (d < -ku)] = 0.0
    ab = synthetic.dense_to_band(a, kl, ku)
    fb, _ = oracle.band_lu(ab, kl, ku)
    for on in (True, False):
        diag_kernel(on)
        f = ebv.band_factor(torch.from_numpy(ab).to(DEV), kl, ku, "fp64")
        assert int(f.info.item()) == 0
        assert np.abs(f.lu.cpu().numpy() - fb).max() <= 1e-13, on


@pytest.mark.parametrize("k", [0, 1, 15, 16, 17, 31, 48, 63, 64, 100, 199])
def test_zero_pivot_same_index(diag_kernel, k):
    n = 200
    a = synthetic.dense_dd(n, 0.5, 93_000 + k)
    a[k, :k] = 0.0
    a[:k, k] = 0.0
    a[k, k] = 0.0  # no earlier step touches a_kk: it reaches the elimination as 0
    for on in (True, False):
        diag_kernel(on)
        f = ebv.factor(torch.from_numpy(a).to(DEV), "fp64")
        assert int(f.info.item()) == k + 1, on


def test_planted_dyadic_factors_exact(diag_kernel):
    rng = np.random.default_rng(11)
    n = 192
    lo = np.eye(n)
    up = np.diag(rng.choice([1.0, 2.0, 0.5, -1.0], size=n))
    for _ in range(3 * n):
        i, j = rng.integers(0, n, 2)
        if i > j:
            lo[i, j] = rng.choice([0.25, -0.5, 0.125])
        elif j > i:
            up[i, j] = rng.choice([0.5, -0.25, 1.0])
    a = lo @ up
    for on in (True, False):
        diag_kernel(on)
        f = ebv.factor(torch.from_numpy(a).to(DEV), "fp64")
        lu = f.lu.cpu().numpy()
        assert np.array_equal(np.tril(lu, -1), np.tril(lo, -1)) and np.array_equal(np.triu(lu), up), on


def _with_bad_pivot(n, k, bad, seed):
    a = synthetic.dense_dd(n, 0.5, seed)
    a[k, :k] = 0.0
    a[:k, k] = 0.0
    a[k, k] = bad  # no earlier step touches a_kk: it reaches the elimination as is
    return a


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf, 0.0])
@pytest.mark.parametrize("prec,n", [("fp64", 200), ("fp64", 700), ("fp32", 200), ("fp32", 700), ("bf16", 700)])
def test_nonfinite_pivot_reported_first(bad, prec, n):
    # every path of the dense factorisation (panels and registers in FP64,
    # the cluster or blocked binary32 leaves, the mixed precisions) reports the
    # first zero / non-finite pivot; later pivots may be NaN too (it spreads)
    k = 77
    a = _with_bad_pivot(n, k, bad, 97_000 + n)
    f = ebv.factor(torch.from_numpy(a).to(DEV), prec)
    assert int(f.info.item()) == k + 1, (prec, n, bad)


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_nonfinite_pivot_band_and_batched(bad):
    n, kl, k = 600, 40, 333
    a = _with_bad_pivot(n, k, bad, 98_000)
    d = np.subtract.outer(np.arange(n), np.arange(n))
    a[np.abs(d) > kl] = 0.0
    ab = synthetic.dense_to_band(a, kl, kl)
    f = ebv.band_factor(torch.from_numpy(ab).to(DEV), kl, kl, "fp64")
    assert int(f.info.item()) == k + 1
    batch = ebv.Batch([50, 120], [1, 1], "fp64")
    for s, m in enumerate((50, 120)):
        sysa = _with_bad_pivot(m, 31, bad, 98_100 + m) if s == 1 else synthetic.dense_dd(m, 0.5, 98_200)
        batch.a_view(s).copy_(torch.from_numpy(sysa))
        batch.b_view(s).copy_(torch.ones((m, 1), dtype=torch.float64))
    batch.run()
    info = batch.info.cpu().numpy()
    assert info[0] == 0 and info[1] == 32
