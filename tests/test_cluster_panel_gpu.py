"""The thread-block-cluster panel kernel against the CPU oracle, and against
the default paths (one-CTA diagonal blocks with separate L21 / U12 launches).

Switched on (ebv_debug_set_band_cluster(1), ebv_debug_set_small_dense(0)) it
factors every 64-column panel of the banded factorisation (diagonal block,
L21 and U12 in one launch) and whole dense systems of order <= 256.  The
shapes below give panels narrower than 64 (the last one), odd widths (a
middle column without a partner), bands narrower and wider than a panel,
and kl != ku.  Tolerances as for the other FP64 paths: factors within 1e-13
of the oracle's, X within 1e-11 relative, backward error <= 1e-14; FP32
factors 5e-5.  Zero pivots must be reported at the same index by both paths.
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
def cluster_switch():
    lib = ebv.lib()

    def mode(on):  # on: the cluster panel wherever it can run; off: the defaults
        lib.ebv_debug_set_cluster_panel(1)
        lib.ebv_debug_set_band_cluster(1 if on else 0)
        lib.ebv_debug_set_small_dense(0 if on else 1)

    yield mode
    mode(0)


def _dense(a, prec):
    f = ebv.factor(torch.from_numpy(a).to(DEV), prec)
    return f, f.lu.cpu().numpy().astype(np.float64), int(f.info.item())


@pytest.mark.parametrize("n", [1, 2, 5, 33, 64, 127, 200, 255, 256])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_dense_small_both_paths_match_oracle(cluster_switch, n, prec):
    a = synthetic.dense_dd(n, 0.9, 60_000 + n)
    b = synthetic.rhs_for(a, synthetic.planted_x(n, 2, 60_000 + n))
    lu_ref, _ = oracle.lu(a)
    x_ref = oracle.solve(lu_ref, b)
    tol_f, tol_x = (1e-13, 1e-11) if prec == "fp64" else (5e-5, 1e-4)
    out = {}
    for on in (1, 0):
        cluster_switch(on)
        f, lu, info = _dense(a, prec)
        x = ebv.solve(f, torch.from_numpy(b).to(DEV)).cpu().numpy().astype(np.float64)
        assert info == 0
        assert np.abs(lu - lu_ref).max() <= tol_f, (on, np.abs(lu - lu_ref).max())
        assert np.abs(x - x_ref).max() / np.abs(x_ref).max() <= tol_x
        out[on] = lu
    assert np.abs(out[1] - out[0]).max() <= 2 * tol_f


@pytest.mark.parametrize("n,kl,ku", [(500, 3, 70), (300, 90, 5), (130, 64, 64), (257, 1, 1), (700, 200, 300),
                                     (200, 0, 20), (200, 20, 0), (1000, 130, 130)])
def test_band_panels_both_paths_match_oracle(cluster_switch, n, kl, ku):
    a = synthetic.dense_dd(n, 0.9, 61_000 + n + kl)
    d = np.subtract.outer(np.arange(n), np.arange(n))
    a[(d > kl) | (d < -ku)] = 0.0
    ab = synthetic.dense_to_band(a, kl, ku)
    x_true = synthetic.planted_x(n, 3, 61_000 + n)
    b = synthetic.band_rhs(ab, kl, ku, x_true)
    fb, _ = oracle.band_lu(ab, kl, ku)
    x_ref = oracle.band_solve(fb, kl, ku, b)
    for on in (1, 0):
        cluster_switch(on)
        for sym in ((False, True) if kl == ku else (False,)):
            if sym:  # the symmetric mode needs a symmetric matrix
                asym = np.tril(a) + np.tril(a, -1).T
                abs_ = synthetic.dense_to_band(asym, kl, ku)
                fref, _ = oracle.band_lu(abs_, kl, ku)
                f = ebv.band_factor(torch.from_numpy(abs_).to(DEV), kl, ku, "fp64", sym=True)
                assert int(f.info.item()) == 0
                assert np.abs(f.lu.cpu().numpy() - fref).max() <= 1e-13, (on, "sym")
                continue
            f = ebv.band_factor(torch.from_numpy(ab).to(DEV), kl, ku, "fp64")
            x = ebv.solve(f, torch.from_numpy(b).to(DEV)).cpu().numpy()
            assert int(f.info.item()) == 0
            assert np.abs(f.lu.cpu().numpy() - fb).max() <= 1e-13, on
            assert np.abs(x - x_ref).max() / np.abs(x_ref).max() <= 1e-11
            r = oracle.band_residual(ab, kl, ku, x, b)
            assert np.abs(r).max() / (np.abs(ab).sum(axis=1).max() * np.abs(x).max()) <= 1e-14


def test_band_fp32_panels(cluster_switch):
    ab, kl, ku = synthetic.laplacian_band(24)
    fb, _ = oracle.band_lu(ab, kl, ku)
    for on in (1, 0):
        cluster_switch(on)
        f = ebv.band_factor(torch.from_numpy(ab).to(DEV), kl, ku, "fp32")
        assert np.abs(f.lu.cpu().numpy().astype(np.float64) - fb).max() <= 5e-5


@pytest.mark.parametrize("n,k", [(10, 4), (100, 70), (256, 255), (256, 31)])
def test_zero_pivot_index_same_on_both_paths(cluster_switch, n, k):
    a = synthetic.dense_dd(n, 0.5, 62_000 + k)
    a[k, :k] = 0.0
    a[:k, k] = 0.0
    a[k, k] = 0.0
    for on in (1, 0):
        cluster_switch(on)
        _, _, info = _dense(a, "fp64")
        assert info == k + 1, (on, info)


def test_planted_dyadic_factors_exact_on_the_cluster(cluster_switch):
    # few-bit dyadic factors: every product and sum is exact, so the cluster
    # kernel (any order of the rank-1 updates) must return them bit for bit
    rng = np.random.default_rng(5)
    n = 200
    lo = np.eye(n)
    up = np.diag(rng.choice([1.0, 2.0, 0.5, -1.0], size=n))
    for _ in range(3 * n):
        i, j = rng.integers(0, n, 2)
        if i > j:
            lo[i, j] = rng.choice([0.25, -0.5, 0.125])
        elif j > i:
            up[i, j] = rng.choice([0.5, -0.25, 1.0])
    a = lo @ up
    cluster_switch(1)
    for prec in ("fp64", "fp32"):
        _, lu, info = _dense(a, prec)
        assert np.array_equal(np.tril(lu, -1), np.tril(lo, -1)) and np.array_equal(np.triu(lu), up), prec
