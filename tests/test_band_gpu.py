"""Banded path on the GPU against the CPU oracle's banded Doolittle (same
seeded inputs).  Tolerances as for the dense FP64 path: factors within 1e-13
(O(1) entries), X within 1e-11 relative, backward error <= 1e-14."""
import numpy as np
import pytest
import torch

import oracle
import paper_1907_05767_gb300 as ebv
import synthetic

pytestmark = pytest.mark.gpu
DEV = "cuda"


def banded_dd(n, kl, ku, seed, w=0.9):
    a = synthetic.dense_dd(n, w, seed)
    d = np.subtract.outer(np.arange(n), np.arange(n))
    a[(d > kl) | (d < -ku)] = 0.0
    return synthetic.dense_to_band(a, kl, ku), a


def check(ab, kl, ku, nrhs, seed, prec="fp64", sym=False):
    n = ab.shape[0]
    x_true = synthetic.planted_x(n, nrhs, seed)
    b = synthetic.band_rhs(ab, kl, ku, x_true)
    f = ebv.band_factor(torch.from_numpy(ab).to(DEV), kl, ku, prec, sym=sym)
    x = ebv.solve(f, torch.from_numpy(b).to(DEV)).cpu().numpy().astype(np.float64)
    assert int(f.info.item()) == 0
    fb, _ = oracle.band_lu(ab, kl, ku)
    x_ref = oracle.band_solve(fb, kl, ku, b)
    lu = f.lu.cpu().numpy().astype(np.float64)
    tol_f, tol_x, tol_b = (1e-13, 1e-11, 1e-14) if prec == "fp64" else (5e-5, 1e-4, 1e-5)
    assert np.abs(lu - fb).max() <= tol_f
    assert np.abs(x - x_ref).max() / np.abs(x_ref).max() <= tol_x
    r = oracle.band_residual(ab, kl, ku, x, b)
    anorm = np.abs(ab).sum(axis=1).max()
    assert np.abs(r).max() / (anorm * np.abs(x).max()) <= tol_b
    return f, x


@pytest.mark.parametrize("g", [4, 8, 33, 64])
def test_laplacian_grid(g):
    ab, kl, ku = synthetic.laplacian_band(g)
    check(ab, kl, ku, 8, 100 + g)


@pytest.mark.parametrize("n,kl,ku", [(500, 3, 70), (300, 90, 5), (200, 0, 20), (200, 20, 0), (130, 64, 64),
                                     (257, 1, 1), (70, 69, 69)])
def test_unsymmetric_bands(n, kl, ku):
    ab, _ = banded_dd(n, kl, ku, 7 * n + kl)
    check(ab, kl, ku, 3, n)


def test_band_fp32():
    ab, kl, ku = synthetic.laplacian_band(20)
    check(ab, kl, ku, 2, 5, prec="fp32")


def test_padding_slots_untouched():
    n, kl, ku = 100, 7, 9
    ab, _ = banded_dd(n, kl, ku, 3)
    ld = kl + ku + 4
    big = np.full((n, ld), 5.0)
    big[:, : kl + ku + 1] = ab
    t = torch.from_numpy(big).to(DEV)
    info = ebv.ebv_factor(t, "fp64", kl=kl, ku=ku, storage=ebv.BAND)
    assert int(info.item()) == 0
    out = t.cpu().numpy()
    assert np.all(out[:, kl + ku + 1:] == 5.0)
    fb, _ = oracle.band_lu(ab, kl, ku)
    assert np.abs(out[:, : kl + ku + 1] - fb).max() <= 1e-13


def test_band_zero_pivot():
    ab, kl, ku = synthetic.laplacian_band(6)
    ab = ab.copy()
    k = 20
    ab[k, :] = 0.0  # row k empty: a_kk reaches the elimination as 0
    for i in range(max(0, k - ku), k):
        ab[i, k - i + kl] = 0.0
    _, info_ref = oracle.band_lu(ab, kl, ku)
    f = ebv.band_factor(torch.from_numpy(ab).to(DEV), kl, ku)
    assert int(f.info.item()) == info_ref == k + 1


def test_band_refined_solution():
    ab, kl, ku = synthetic.laplacian_band(32)
    n = ab.shape[0]
    b = synthetic.band_rhs(ab, kl, ku, synthetic.planted_x(n, 4, 9))
    f = ebv.band_factor(torch.from_numpy(ab).to(DEV), kl, ku, "fp64")
    rep = torch.zeros(3, dtype=torch.float64, device=DEV)
    x = ebv.solve(f, torch.from_numpy(b).to(DEV), refine=(1e-14, 3), report=rep).cpu().numpy()
    r = ebv.read_report(rep)
    assert r["status"] == ebv.OK and r["resid_final"] <= 1e-14
    fb, _ = oracle.band_lu(ab, kl, ku)
    x_ref = oracle.band_solve(fb, kl, ku, b)
    assert np.abs(x - x_ref).max() / np.abs(x_ref).max() <= 1e-12


def symmetric_banded_dd(n, k, seed, w=0.9):
    a = synthetic.dense_dd(n, w, seed)
    a = 0.5 * (a + a.T)  # still strictly diagonally dominant
    d = np.subtract.outer(np.arange(n), np.arange(n))
    a[np.abs(d) > k] = 0.0
    return synthetic.dense_to_band(a, k, k)


@pytest.mark.parametrize("g", [4, 8, 33, 64])
def test_symmetric_laplacian_grid(g):
    # EBV_BAND_SYM: U12 = D11 L21^T and the block-lower trailing update give
    # the same (unique) factors as the general band path, within rounding.
    ab, kl, ku = synthetic.laplacian_band(g)
    check(ab, kl, ku, 8, 300 + g, sym=True)


@pytest.mark.parametrize("n,k", [(500, 70), (130, 64), (257, 1), (70, 69), (300, 128), (200, 0)])
def test_symmetric_bands(n, k):
    ab = symmetric_banded_dd(n, k, 11 * n + k)
    f, _ = check(ab, k, k, 3, n + 1, sym=True)
    # the stored U vectors are the pivots times the L vectors: u_ij = u_ii l_ji
    lu = f.lu.cpu().numpy()
    for i in range(0, n, max(1, n // 17)):
        for j in range(i + 1, min(n, i + k + 1)):
            u = lu[i, j - i + k]
            l = lu[j, i - j + k]
            assert abs(u - lu[i, k] * l) <= 1e-13 * max(1.0, abs(u))


def test_symmetric_band_fp32():
    ab, kl, ku = synthetic.laplacian_band(20)
    check(ab, kl, ku, 2, 7, prec="fp32", sym=True)


def factors_without_envelope(ab, kl, ku, prec, sym):
    ebv.lib().ebv_debug_set_band_envelope(0)
    try:
        f = ebv.band_factor(torch.from_numpy(ab).to(DEV), kl, ku, prec, sym=sym)
        return f.lu.cpu().numpy()
    finally:
        ebv.lib().ebv_debug_set_band_envelope(1)


@pytest.mark.parametrize("sym", [False, True])
@pytest.mark.parametrize("r", [20, 45])
def test_profile_disc_laplacian(r, sym):
    # An irregular domain: the distance to the next grid row's neighbour follows
    # the chord, so the band's width varies and the factorisation skips the
    # tiles outside the profile.  Skipped tiles are exactly zero, so the factors
    # equal those of the full band window bit for bit.
    ab, kl, ku = synthetic.laplacian_disc_band(r)
    f, _ = check(ab, kl, ku, 4, 400 + r, sym=sym)
    assert np.array_equal(f.lu.cpu().numpy(), factors_without_envelope(ab, kl, ku, "fp64", sym))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_profile_random(prec):
    from oracle_pins import variable_profile_dd
    kl, ku = 90, 130
    a = variable_profile_dd(700, kl, ku, 3)
    a = (a + np.diag(np.abs(a).sum(axis=1))) / 128.0  # well conditioned, O(1) pivots: the FP32 tolerances
    ab = synthetic.dense_to_band(a, kl, ku)
    f, _ = check(ab, kl, ku, 3, 701, prec=prec)
    assert np.array_equal(f.lu.cpu().numpy(), factors_without_envelope(ab, kl, ku, prec, False))


@pytest.mark.parametrize("prec,sym,grid", [("bf16", False, 40), ("fp16", True, 40), ("bf16", True, 0)])
def test_band_mixed_refined(prec, sym, grid):
    # Mixed precision on a band: FP32 factors of the FP64 band (FP32 tolerances
    # against the oracle's factors), then refinement with the FP64-accurate
    # band residual to a relative residual of 1e-12.
    ab, kl, ku = synthetic.laplacian_band(grid) if grid else synthetic.laplacian_disc_band(30)
    n = ab.shape[0]
    x_true = synthetic.planted_x(n, 8, 800 + n)
    b = synthetic.band_rhs(ab, kl, ku, x_true)
    f = ebv.band_factor(torch.from_numpy(ab).to(DEV), kl, ku, prec, sym=sym)
    assert f.lu.dtype == torch.float32 and int(f.info.item()) == 0
    fb, _ = oracle.band_lu(ab, kl, ku)
    assert np.abs(f.lu.cpu().numpy().astype(np.float64) - fb).max() <= 5e-5
    rep = torch.zeros(3, dtype=torch.float64, device=DEV)
    x = ebv.solve(f, torch.from_numpy(b).to(DEV), refine=(1e-12, 10), report=rep).cpu().numpy()
    r = ebv.read_report(rep)
    assert r["status"] == ebv.OK and r["resid_final"] <= 1e-12 and r["iters"] >= 1, r
    x_ref = oracle.band_solve(fb, kl, ku, b)
    assert np.abs(x - x_ref).max() / np.abs(x_ref).max() <= 1e-11
    res = oracle.band_residual(ab, kl, ku, x, b)
    assert (np.abs(res).max(axis=0) / np.abs(b).max(axis=0)).max() <= 1e-12
