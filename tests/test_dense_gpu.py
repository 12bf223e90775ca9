"""Dense path on the GPU against the CPU oracle (same seeded inputs).

Tolerances (FP64): factors within 1e-13 of the oracle's (entries are O(1);
the two differ only in summation order and fused multiply-adds), X within
1e-11 max-norm relative, backward error ||b - Ax||/(||A|| ||x||) <= 1e-14.
FP32: the same quantities within bounds derived from n * 2^-24 (factors 5e-5,
X 1e-4 relative, backward error 1e-5).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1907_05767_gb300 as ebv
import synthetic

pytestmark = pytest.mark.gpu
DEV = "cuda"


def backward_error(a, x, b):
    r = oracle.residual(a, x, b)
    return np.abs(r).max() / (np.abs(a).sum(axis=1).max() * np.abs(x).max())


def relerr(x, ref):
    return np.abs(x - ref).max() / np.abs(ref).max()


SIZES = [1, 2, 3, 17, 31, 63, 64, 65, 100, 127, 128, 129, 200, 256, 300, 511, 777]


@pytest.mark.parametrize("n", SIZES)
def test_fp64_factor_solve_matches_oracle(n):
    a = synthetic.dense_dd(n, 0.9, 10_000 + n)
    x_true = synthetic.planted_x(n, 3, 10_000 + n)
    b = synthetic.rhs_for(a, x_true)
    f = ebv.factor(torch.from_numpy(a).to(DEV), "fp64")
    x = ebv.solve(f, torch.from_numpy(b).to(DEV)).cpu().numpy()
    assert int(f.info.item()) == 0
    lu_ref, _ = oracle.lu(a)
    x_ref = oracle.solve(lu_ref, b)
    assert np.abs(f.lu.cpu().numpy() - lu_ref).max() <= 1e-13
    assert relerr(x, x_ref) <= 1e-11
    assert backward_error(a, x, b) <= 1e-14


def test_fp64_factor_large_rows_sampled():
    # n = 10000: the two-leaf panel update launches 156 row blocks, more CTAs
    # than FP64 tiles fit on the GPU at once, so later CTAs run after the first
    # ones have finished.  |A - LU| on sampled rows (the last ones included,
    # which the last CTAs own) stays at the level of FP64 rounding.
    n = 10_000
    a = synthetic.dense_dd(n, 0.9, 10_000 + n)
    x_true = synthetic.planted_x(n, 2, 10_000 + n)
    b = synthetic.rhs_for(a, x_true)
    f = ebv.factor(torch.from_numpy(a).to(DEV), "fp64")
    x = ebv.solve(f, torch.from_numpy(b).to(DEV)).cpu().numpy()
    assert int(f.info.item()) == 0
    lu = f.lu.cpu().numpy()
    rng = np.random.default_rng(7)
    rows = np.unique(np.concatenate([rng.integers(0, n, 16), np.arange(n - 260, n, 13), [0, 63, 64, 127, 128]]))
    lrows = np.where(np.arange(n)[None, :] < rows[:, None], lu[rows], 0.0)  # strict lower part of L's rows
    lrows[np.arange(len(rows)), rows] = 1.0
    lu_rows = lrows @ np.triu(lu)
    assert np.abs(a[rows] - lu_rows).max() <= 1e-13
    r = b[rows] - a[rows] @ x
    assert np.abs(r).max() / (np.abs(a[rows]).sum(axis=1).max() * np.abs(x).max()) <= 1e-14
    assert np.abs(x - x_true).max() <= 1e-11


@pytest.mark.parametrize("n", [5, 64, 130, 333])
def test_fp32_factor_solve_matches_oracle(n):
    a = synthetic.dense_dd(n, 0.9, 20_000 + n)
    x_true = synthetic.planted_x(n, 2, 20_000 + n)
    b = synthetic.rhs_for(a, x_true)
    f = ebv.factor(torch.from_numpy(a).to(DEV), "fp32")
    x = ebv.solve(f, torch.from_numpy(b).to(DEV)).cpu().numpy().astype(np.float64)
    lu_ref, _ = oracle.lu(a)
    x_ref = oracle.solve(lu_ref, b)
    assert np.abs(f.lu.cpu().numpy().astype(np.float64) - lu_ref).max() <= 5e-5
    assert relerr(x, x_ref) <= 1e-4
    assert backward_error(a, x, b) <= 1e-5


def test_config0_n256_single_rhs():
    a, x_true, b = synthetic.config0()
    f = ebv.factor(torch.from_numpy(a).to(DEV), "fp64")
    x = ebv.solve(f, torch.from_numpy(b).to(DEV)).cpu().numpy()
    lu_ref, _ = oracle.lu(a)
    x_ref = oracle.solve(lu_ref, b)
    assert relerr(x, x_ref) <= 1e-11
    assert backward_error(a, x, b) <= 1e-14
    assert np.abs(x - x_true).max() <= 1e-12


def test_planted_dyadic_factors_are_exact():
    # Every intermediate is a short dyadic number, so any summation order (and
    # FMA) must reproduce the planted factors bit for bit.
    from oracle_pins import _planted_dyadic
    for n in (7, 64, 65, 150):
        lo, up, a = _planted_dyadic(n, 900 + n) if n <= 13 else _big_dyadic(n)
        for prec, dt in (("fp64", np.float64), ("fp32", np.float32)):
            f = ebv.factor(torch.from_numpy(a).to(DEV), prec)
            lu = f.lu.cpu().numpy().astype(np.float64)
            assert np.array_equal(np.tril(lu, -1), np.tril(lo, -1)), (n, prec)
            assert np.array_equal(np.triu(lu), up), (n, prec)


def _big_dyadic(n):
    """Planted unit-lower L and upper U with few-bit dyadic entries, sparse
    enough that A = LU and every Schur complement stay exact in binary32."""
    rng = np.random.default_rng(n)
    lo = np.eye(n)
    up = np.diag(rng.choice([1.0, 2.0, 0.5, -1.0], size=n))
    for _ in range(3 * n):
        i, j = rng.integers(0, n, 2)
        if i > j:
            lo[i, j] = rng.choice([0.25, -0.5, 0.125])
        elif j > i:
            up[i, j] = rng.choice([0.5, -0.25, 1.0])
    a = lo @ up
    return lo, up, a


def test_padded_leading_dimension():
    n, ld = 150, 160
    a = synthetic.dense_dd(n, 0.9, 31)
    b = synthetic.rhs_for(a, synthetic.planted_x(n, 2, 31))
    big = torch.zeros((n, ld), dtype=torch.float64, device=DEV)
    big[:, :n] = torch.from_numpy(a)
    big[:, n:] = 7.0  # must stay untouched
    info = ebv.ebv_factor(big, "fp64")
    assert int(info.item()) == 0
    assert torch.all(big[:, n:] == 7.0)
    lu_ref, _ = oracle.lu(a)
    assert np.abs(big[:, :n].cpu().numpy() - lu_ref).max() <= 1e-13
    x = torch.from_numpy(b).to(DEV).clone()
    ebv.ebv_solve(big, x, "fp64", ld=ld)
    assert relerr(x.cpu().numpy(), oracle.solve(lu_ref, b)) <= 1e-11


@pytest.mark.parametrize("prec,ld", [("fp64", 701), ("fp32", 703)])
def test_unaligned_leading_dimension(prec, ld):
    """Rows of an odd leading dimension are not 16-byte aligned: the block
    substitution copies their tiles element by element (n = 700, above the
    one-CTA small-system solve)."""
    n, nrhs = 700, 3
    dt = torch.float64 if prec == "fp64" else torch.float32
    a = synthetic.dense_dd(n, 0.9, 33)
    x_true = synthetic.planted_x(n, nrhs, 33)
    b = synthetic.rhs_for(a, x_true)
    big = torch.zeros((n, ld), dtype=dt, device=DEV)
    big[:, :n] = torch.from_numpy(a).to(dt)
    big[:, n:] = 7.0  # must stay untouched
    info = ebv.ebv_factor(big, prec)
    assert int(info.item()) == 0
    assert torch.all(big[:, n:] == 7.0)
    lu_ref, _ = oracle.lu(a)
    x = torch.from_numpy(b).to(DEV).to(dt).clone()  # the right-hand sides in the factors' precision
    ebv.ebv_solve(big, x, prec, ld=ld)
    assert torch.all(big[:, n:] == 7.0)
    xs = x.cpu().numpy().astype(np.float64)
    if prec == "fp64":
        assert np.abs(big[:, :n].cpu().numpy() - lu_ref).max() <= 1e-13
        assert relerr(xs, oracle.solve(lu_ref, b)) <= 1e-11
    else:
        assert np.abs(big[:, :n].cpu().numpy().astype(np.float64) - lu_ref).max() <= 5e-5
        assert relerr(xs, oracle.solve(lu_ref, b)) <= 1e-4
        assert backward_error(a, xs, b) <= 1e-5


@pytest.mark.parametrize("n,k", [(10, 4), (100, 70), (300, 1)])
def test_zero_pivot_reported(n, k):
    a = synthetic.dense_dd(n, 0.5, 41)
    # Row k and column k are zero left of / above the diagonal, so no step
    # before k changes a_kk: it reaches the elimination as an exact 0.
    a[k, :k] = 0.0
    a[:k, k] = 0.0
    a[k, k] = 0.0
    _, info_ref = oracle.lu(a)
    f = ebv.factor(torch.from_numpy(a).to(DEV), "fp64")
    assert int(f.info.item()) == info_ref == k + 1


def test_nan_pivot_reported():
    a = synthetic.dense_dd(80, 0.5, 43)
    a[70, 70] = np.nan
    _, info_ref = oracle.lu(a)
    f = ebv.factor(torch.from_numpy(a).to(DEV), "fp64")
    assert int(f.info.item()) == info_ref == 71


def test_empty_system_and_zero_rhs():
    info = ebv.ebv_factor(torch.zeros((0, 1), dtype=torch.float64, device=DEV), "fp64")
    assert int(info.item()) == 0
    a2 = torch.from_numpy(synthetic.dense_dd(20, 0.5, 5)).to(DEV)
    f = ebv.factor(a2, "fp64")
    b = torch.zeros((20, 1), dtype=torch.float64, device=DEV)[:, :0]
    ebv.ebv_solve(f.lu, b, "fp64", ld=20)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("n", [64, 200, 1000, 2048])
def test_mixed_refined_matches_fp64_oracle(prec, n):
    a = synthetic.dense_dd(n, 0.9, 50_000 + n)
    x_true = synthetic.planted_x(n, 4, 50_000 + n)
    b = synthetic.rhs_for(a, x_true)
    f = ebv.factor(torch.from_numpy(a).to(DEV), prec)
    rep = torch.zeros(3, dtype=torch.float64, device=DEV)
    x = ebv.solve(f, torch.from_numpy(b).to(DEV), refine=(1e-12, 10), report=rep).cpu().numpy()
    r = ebv.read_report(rep)
    lu_ref, _ = oracle.lu(a)
    x_ref = oracle.solve(lu_ref, b)
    # the unrefined FP32 factors carry the bfloat16 / half rounding of the
    # update operands: relative residual of the first solve well below 1
    assert r["resid_first"] < 1e-2
    assert r["status"] == ebv.OK and r["resid_final"] <= 1e-12, r
    assert relerr(x, x_ref) <= 1e-11
    rel_res = np.abs(oracle.residual(a, x, b)).max(axis=0) / np.abs(b).max(axis=0)
    assert rel_res.max() <= 1e-12


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_mixed_refined_to_fp64_backward_error(prec):
    # With a tighter stop test the refined solution reaches the FP64 path's
    # backward-error bound as well.
    n = 1500
    a = synthetic.dense_dd(n, 0.9, 70_000)
    b = synthetic.rhs_for(a, synthetic.planted_x(n, 3, 70_000))
    f = ebv.factor(torch.from_numpy(a).to(DEV), prec)
    rep = torch.zeros(3, dtype=torch.float64, device=DEV)
    x = ebv.solve(f, torch.from_numpy(b).to(DEV), refine=(1e-15, 8), report=rep).cpu().numpy()
    assert backward_error(a, x, b) <= 1e-14
    assert ebv.read_report(rep)["iters"] <= 8


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_mixed_factors_close_to_oracle(prec):
    n = 512
    a = synthetic.dense_dd(n, 0.9, 60_000)
    f = ebv.factor(torch.from_numpy(a).to(DEV), prec)
    lu_ref, _ = oracle.lu(a)
    lu = f.lu.cpu().numpy().astype(np.float64)
    # each Schur update is a sum of products of 8-bit (bf16) / 11-bit (half)
    # operands; with |l|,|u| <= 1.8e-3 here the accumulated error is far below 1e-4
    assert np.abs(lu - lu_ref).max() <= 1e-4
    # a(0,:) and the first column only need the FP32 rounding of A
    np.testing.assert_allclose(lu[0], lu_ref[0], rtol=1e-7, atol=1e-9)
