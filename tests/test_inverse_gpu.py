"""Explicit inverse (the product form of Eq. 4c, A^{-1} = U^{-1} L^{-1})
against the FP64 oracle, element by element.

Tolerances.  FP64 from the oracle's own factors: only the summation order
differs (each entry sums at most n products of entries of W = U^{-1} and
Z = L^{-1}), so |X - X_oracle| <= 1e-12 max|X_oracle| (n u ~ 1e-13 for
n ~ 1000).  FP64 end to end from the GPU's factors: 1e-11, the bar of the FP64
solve (X = A^{-1} I).  Exact cases (diagonal, dyadic bidiagonal L or U: every
product has a single non-zero term) match bit for bit.  FP32 (binary32 factors
and products): 1e-4 relative; from the binary32 factors of a bf16
mixed-precision factorisation: 1e-3 (those factors carry the bf16 rounding of
the trailing updates).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1907_05767_gb300 as ebv
import synthetic

pytestmark = pytest.mark.gpu

# one leaf, ragged leaves, several tree levels with ragged last nodes
SIZES = [1, 5, 64, 65, 129, 200, 449, 777, 1100]


def relerr(x, ref):
    return float(np.abs(x - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("n", SIZES)
def test_inverse_fp64_from_oracle_factors(n):
    a = synthetic.dense_dd(n, 0.9, 70_000 + n)
    f, info = oracle.lu(a)
    assert info == 0
    x_ref = oracle.inverse(f)
    x = ebv.ebv_inverse(torch.from_numpy(f).cuda(), prec="fp64").cpu().numpy()
    assert relerr(x, x_ref) <= 1e-12, relerr(x, x_ref)


@pytest.mark.parametrize("n", [300, 1100])
def test_inverse_fp64_end_to_end(n):
    a = synthetic.dense_dd(n, 0.9, 71_000 + n)
    fac = ebv.factor(torch.from_numpy(a).cuda(), "fp64")
    x = ebv.inverse(fac).cpu().numpy()
    assert int(fac.info.item()) == 0
    x_ref = oracle.inverse(oracle.lu(a)[0])
    assert relerr(x, x_ref) <= 1e-11, relerr(x, x_ref)
    assert np.abs(a @ x - np.eye(n)).max() <= 1e-13


def test_inverse_padded_leading_dimensions():
    n = 333
    a = synthetic.dense_dd(n, 0.9, 72_000)
    f, _ = oracle.lu(a)
    lu = torch.zeros((n, n + 7), dtype=torch.float64, device="cuda")
    lu[:, :n] = torch.from_numpy(f).cuda()
    xt = torch.full((n, n + 5), float("nan"), dtype=torch.float64, device="cuda")
    ebv.ebv_inverse(lu[:, :n], xt[:, :n], prec="fp64")
    xs = xt.cpu().numpy()
    assert relerr(xs[:, :n], oracle.inverse(f)) <= 1e-12
    assert np.isnan(xs[:, n:]).all()  # the padding of x is not written


@pytest.mark.parametrize("n", [70, 300])
def test_inverse_exact_cases(n):
    i, j = np.indices((n, n))
    d = np.resize(np.array([2.0, -4.0, 0.5, 8.0, 1.0, -0.25]), n)
    cases = [
        (np.diag(d), np.diag(1.0 / d)),
        (np.eye(n) - 0.5 * np.eye(n, k=-1), np.where(i >= j, 0.5 ** (i - j), 0.0)),
        (2.0 * np.eye(n) + np.eye(n, k=1), np.where(j >= i, 0.5 * (-0.5) ** (j - i), 0.0)),
    ]
    for a, expected in cases:
        f, info = oracle.lu(a)
        assert info == 0
        assert np.array_equal(oracle.inverse(f), expected)
        x = ebv.ebv_inverse(torch.from_numpy(f).cuda(), prec="fp64").cpu().numpy()
        assert np.array_equal(x, expected)


@pytest.mark.parametrize("n", [65, 449, 1100])
def test_inverse_fp32(n):
    a = synthetic.dense_dd(n, 0.9, 73_000 + n)
    f = oracle.lu(a)[0].astype(np.float32)
    x = ebv.ebv_inverse(torch.from_numpy(f).cuda(), prec="fp32").cpu().numpy()
    assert x.dtype == np.float32
    assert relerr(x.astype(np.float64), oracle.inverse(f.astype(np.float64))) <= 1e-4
    fac = ebv.factor(torch.from_numpy(a).cuda(), "fp32")
    x = ebv.inverse(fac).cpu().numpy().astype(np.float64)
    assert relerr(x, oracle.inverse(oracle.lu(a)[0])) <= 1e-4


def test_inverse_from_mixed_precision_factors():
    n = 640
    a = synthetic.dense_dd(n, 0.9, 74_000)
    fac = ebv.factor(torch.from_numpy(a).cuda(), "bf16")
    x = ebv.inverse(fac)
    assert x.dtype == torch.float32 and int(fac.info.item()) == 0
    assert relerr(x.cpu().numpy().astype(np.float64), oracle.inverse(oracle.lu(a)[0])) <= 1e-3


def test_inverse_large_sampled():
    # several full tree levels (n = 4096: six of them): sampled rows of A X - I
    # and X A - I, and sampled columns against the oracle's substitutions
    n = 4096
    a = synthetic.dense_dd(n, 0.9, 75_000)
    fac = ebv.factor(torch.from_numpy(a).cuda(), "fp64")
    x = ebv.inverse(fac).cpu().numpy()
    rows = synthetic.pick_indices(17, 24, [n])[:, 0]
    eye = np.eye(n)[rows]
    assert np.abs(a[rows] @ x - eye).max() <= 1e-13
    assert np.abs(x[rows] @ a - eye).max() <= 1e-13
    cols = synthetic.pick_indices(18, 4, [n])[:, 0]
    lu, _ = oracle.lu(a)
    ref = oracle.solve(lu, np.eye(n)[:, cols])
    assert np.abs(x[:, cols] - ref).max() <= 1e-11 * np.abs(ref).max()
