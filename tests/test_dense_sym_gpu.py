"""Dense symmetric storage (EBV_DENSE_SYM) against the CPU oracle's dense
Doolittle on the full matrix.

For symmetric A the Doolittle factors satisfy U = D L^T (D the pivots; the
oracle's pins check this against Cholesky), so the lower triangle carries all
of them: the GPU leaves L below the diagonal and D on it, forms only the
block-lower part of each trailing update and never touches the entries above
the diagonal (the test fills them with a sentinel and checks it survives).
Checked: the lower triangle against the oracle's L and diagonal of U (1e-13),
X against the oracle's substitutions (1e-11 relative) and the backward error
over every row (<= 1e-14) for FP64; FP32 factors (5e-5); FP64 refinement;
zero pivots; both the side-stream look-ahead and the serial order.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1907_05767_gb300 as ebv
import synthetic

pytestmark = pytest.mark.gpu
DEV = "cuda"
SENTINEL = 12345.0


def sym_dd(n, seed, w=0.9):
    a = synthetic.dense_dd(n, w, seed)
    return np.tril(a) + np.tril(a, -1).T  # symmetric, still strictly diagonally dominant


def _factor(a, prec):
    # the upper triangle holds a sentinel: the factorisation must neither read nor write it
    stored = np.tril(a) + np.triu(np.full_like(a, SENTINEL), 1)
    f = ebv.factor(torch.from_numpy(stored).to(DEV), prec, sym=True, keep_a=False)
    f.a = torch.from_numpy(stored).to(DEV)  # A's lower triangle for the refinement's residual
    return f


@pytest.mark.parametrize("n", [1, 2, 5, 63, 64, 65, 130, 200, 777, 2000])
def test_fp64_matches_oracle(n):
    a = sym_dd(n, 80_000 + n)
    x_true = synthetic.planted_x(n, 3, 81_000 + n)
    b = synthetic.rhs_for(a, x_true)
    lu_ref, _ = oracle.lu(a)
    x_ref = oracle.solve(lu_ref, b)
    f = _factor(a, "fp64")
    x = ebv.solve(f, torch.from_numpy(b).to(DEV)).cpu().numpy()
    assert int(f.info.item()) == 0
    lu = f.lu.cpu().numpy()
    assert np.all(np.triu(lu, 1) == np.triu(np.full_like(lu, SENTINEL), 1))
    lo = np.tril(lu)
    assert np.abs(lo - np.tril(lu_ref)).max() <= 1e-13  # L below the diagonal, the pivots on it
    assert np.abs(x - x_ref).max() / np.abs(x_ref).max() <= 1e-11
    r = oracle.residual(a, x, b)
    assert np.abs(r).max() / (np.abs(a).sum(axis=1).max() * np.abs(x).max()) <= 1e-14


def test_fp64_without_lookahead_same_factors():
    n = 900
    a = sym_dd(n, 82_000)
    lib = ebv.lib()
    f1 = _factor(a, "fp64")
    lib.ebv_debug_set_band_lookahead(0)
    try:
        f0 = _factor(a, "fp64")
    finally:
        lib.ebv_debug_set_band_lookahead(2)
    # the same operations in the same order on each entry: bit for bit
    assert torch.equal(torch.tril(f1.lu), torch.tril(f0.lu))


def test_fp32_and_refined():
    n = 700
    a = sym_dd(n, 83_000)
    lu_ref, _ = oracle.lu(a)
    f = _factor(a, "fp32")
    assert int(f.info.item()) == 0
    assert np.abs(np.tril(f.lu.cpu().numpy().astype(np.float64)) - np.tril(lu_ref)).max() <= 5e-5
    x_true = synthetic.planted_x(n, 2, 83_100)
    b = synthetic.rhs_for(a, x_true)
    f64 = _factor(a, "fp64")
    rep = torch.zeros(3, dtype=torch.float64, device=DEV)
    x = ebv.solve(f64, torch.from_numpy(b).to(DEV), refine=(1e-15, 5), report=rep).cpu().numpy()
    r = oracle.residual(a, x, b)
    assert (np.abs(r).max(axis=0) / np.abs(b).max(axis=0)).max() <= 1e-14
    assert np.abs(x - x_true).max() <= 1e-12


@pytest.mark.parametrize("n,k", [(10, 4), (300, 77), (300, 299)])
def test_zero_pivot_index(n, k):
    a = sym_dd(n, 84_000 + k, w=0.5)
    a[k, :] = 0.0
    a[:, k] = 0.0  # no earlier step touches a_kk: it reaches the elimination as 0
    f = _factor(a, "fp64")
    assert int(f.info.item()) == k + 1


def test_mixed_precisions_rejected():
    a = torch.from_numpy(sym_dd(64, 85_000)).to(DEV)
    lowp = torch.empty((64, 64), dtype=torch.float32, device=DEV)
    with pytest.raises(ebv.EbvError) as e:
        ebv.ebv_factor(a, "bf16", lowp=lowp, storage=ebv.DENSE_SYM)
    assert e.value.status == ebv.ERR_UNSUPPORTED
