"""Symmetric band kept in its lower half (EBV_BAND_SYM_LOWER) against the CPU
oracle's banded Doolittle on the full band.

For symmetric A the Doolittle factors satisfy U = D L^T (D the pivots; the
oracle's pins check this against Cholesky), so the lower half carries all of
it: the GPU leaves L below the diagonal and D on it, in kl + 1 entries per
row.  Checked: those entries against the oracle's L and diagonal of U
(1e-13), X against the oracle's banded substitutions (1e-11 relative) and the
backward error over every row (<= 1e-14) for FP64; FP32 factors (5e-5); the
mixed precisions refined to a relative residual <= 1e-12; zero pivots.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1907_05767_gb300 as ebv
import synthetic

pytestmark = pytest.mark.gpu
DEV = "cuda"


def sym_band(n, kl, seed, w=0.9):
    a = synthetic.dense_dd(n, w, seed)
    a = np.tril(a) + np.tril(a, -1).T  # symmetric, still strictly diagonally dominant
    d = np.subtract.outer(np.arange(n), np.arange(n))
    a[np.abs(d) > kl] = 0.0
    return synthetic.dense_to_band(a, kl, kl)


CASES = [("lap", 8), ("lap", 33), ("lap", 64), ("rand", (500, 30)), ("rand", (300, 100)), ("rand", (130, 64)),
         ("rand", (257, 1)), ("rand", (700, 250))]


def _case(kind, arg):
    if kind == "lap":
        ab, kl, _ = synthetic.laplacian_band(arg)
        return ab, kl
    n, kl = arg
    return sym_band(n, kl, 70_000 + n + kl), kl


@pytest.mark.parametrize("kind,arg", CASES)
def test_lower_half_fp64_matches_oracle(kind, arg):
    ab, kl = _case(kind, arg)
    n = ab.shape[0]
    lower = np.ascontiguousarray(ab[:, :kl + 1])  # the stored half: kl + 1 entries per row
    x_true = synthetic.planted_x(n, 4, 71_000 + n)
    b = synthetic.band_rhs(ab, kl, kl, x_true)
    fb, _ = oracle.band_lu(ab, kl, kl)
    x_ref = oracle.band_solve(fb, kl, kl, b)
    f = ebv.band_factor(torch.from_numpy(lower).to(DEV), kl, kl, "fp64", sym="lower")
    assert f.lu.shape == (n, kl + 1)
    x = ebv.solve(f, torch.from_numpy(b).to(DEV)).cpu().numpy()
    assert int(f.info.item()) == 0
    lu = f.lu.cpu().numpy()
    assert np.abs(lu - fb[:, :kl + 1]).max() <= 1e-13  # L below the diagonal, the pivots on it
    assert np.abs(x - x_ref).max() / np.abs(x_ref).max() <= 1e-11
    r = oracle.band_residual(ab, kl, kl, x, b)
    assert np.abs(r).max() / (np.abs(ab).sum(axis=1).max() * np.abs(x).max()) <= 1e-14


def test_lower_half_fp32_and_mixed():
    ab, kl, _ = synthetic.laplacian_band(40)
    n = ab.shape[0]
    lower = np.ascontiguousarray(ab[:, :kl + 1])
    fb, _ = oracle.band_lu(ab, kl, kl)
    f = ebv.band_factor(torch.from_numpy(lower).to(DEV), kl, kl, "fp32", sym="lower")
    assert np.abs(f.lu.cpu().numpy().astype(np.float64) - fb[:, :kl + 1]).max() <= 5e-5
    x_true = synthetic.planted_x(n, 3, 72_000)
    b = synthetic.band_rhs(ab, kl, kl, x_true)
    for prec in ("bf16", "fp16"):  # band storage: FP32 factors, FP64 refinement
        f = ebv.band_factor(torch.from_numpy(lower).to(DEV), kl, kl, prec, sym="lower")
        rep = torch.zeros(3, dtype=torch.float64, device=DEV)
        x = ebv.solve(f, torch.from_numpy(b).to(DEV), refine=(1e-12, 10), report=rep).cpu().numpy()
        r_info = ebv.read_report(rep)
        assert int(f.info.item()) == 0 and r_info["status"] == 0
        r = oracle.band_residual(ab, kl, kl, x, b)
        assert (np.abs(r).max(axis=0) / np.abs(b).max(axis=0)).max() <= 1e-12


def test_lower_half_zero_pivot_and_cluster_path():
    ab = sym_band(200, 20, 73_000, w=0.5)
    kl = 20
    k = 77
    a = synthetic.band_to_dense(ab, kl, kl)
    a[k, :k] = 0.0
    a[:k, k] = 0.0
    a[k, k] = 0.0  # no earlier step touches a_kk: it reaches the elimination as 0
    lower = np.ascontiguousarray(synthetic.dense_to_band(a, kl, kl)[:, :kl + 1])
    f = ebv.band_factor(torch.from_numpy(lower).to(DEV), kl, kl, "fp64", sym="lower")
    assert int(f.info.item()) == k + 1
    # the cluster-panel factorisation of the same storage gives the same factors
    ab = sym_band(300, 40, 73_100)
    kl = 40
    lower = np.ascontiguousarray(ab[:, :kl + 1])
    fb, _ = oracle.band_lu(ab, kl, kl)
    lib = ebv.lib()
    lib.ebv_debug_set_band_cluster(1)
    try:
        f = ebv.band_factor(torch.from_numpy(lower).to(DEV), kl, kl, "fp64", sym="lower")
        assert int(f.info.item()) == 0
        assert np.abs(f.lu.cpu().numpy() - fb[:, :kl + 1]).max() <= 1e-13
    finally:
        lib.ebv_debug_set_band_cluster(0)
