"""Profile (skyline) storage, EBV_PROFILE: each 64-row block keeps its part
from the first non-zero of its rows, each 64-column block its part from the
first non-zero of its columns; no row exchanges, so the factors stay inside
and ebv_factor works in place.  Checked against the CPU oracle's banded
Doolittle on the same matrices (the factors unpacked from the buffer,
element by element, 1e-13; X 1e-11 relative; backward error 1e-14; FP32
factors 5e-5), on an irregular-domain Laplacian, a random profile and a
narrow band with a few wide rows (where the profile stores far less than
the band).  The packer itself is checked on the host: the buffer unpacks
to the input matrix exactly.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1907_05767_gb300 as ebv
import synthetic
from oracle_pins import variable_profile_dd

DEV = "cuda"


def few_wide_rows(n, k, reach, seed):
    """Diagonally dominant band kl = ku = k, plus a handful of rows (and
    columns) reaching `reach` back: a widest band many times the typical one."""
    rng = np.random.default_rng(seed)
    a = np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - k), min(n, i + k + 1)):
            a[i, j] = rng.uniform(-1, 1)
    for i in (n // 3, 2 * n // 3, n - 5):
        j0 = max(0, i - reach)
        a[i, j0:i] = rng.uniform(-1, 1, i - j0)
        a[j0:i, i] = rng.uniform(-1, 1, i - j0)
    a += np.diag(np.abs(a).sum(axis=1) + 1.0)
    return a


def _band_of(a):
    d = np.subtract.outer(np.arange(a.shape[0]), np.arange(a.shape[0]))
    nz = a != 0
    kl = int(d[nz].max())
    ku = int((-d[nz]).max())
    return synthetic.dense_to_band(a, kl, ku), kl, ku


def _cases():
    ab, kl, ku = synthetic.laplacian_disc_band(20)
    yield "disc20", ab, kl, ku
    ab, kl, ku = synthetic.laplacian_disc_band(45)
    yield "disc45", ab, kl, ku
    ab, kl, ku = _band_of(variable_profile_dd(700, 40, 60, 3))
    yield "random", ab, kl, ku
    ab, kl, ku = _band_of(few_wide_rows(4000, 4, 400, 4))
    yield "wide_rows", ab, kl, ku


CASES = list(_cases())


@pytest.mark.parametrize("name,ab,kl,ku", CASES, ids=[c[0] for c in CASES])
def test_packer_round_trip(name, ab, kl, ku):
    n = ab.shape[0]
    buf, klp, kup = ebv.ebv_profile_from_band(ab, kl, ku, "fp64")
    assert klp <= kl + 63 and kup <= ku + 63
    back = ebv.profile_to_band(buf, n, klp, kup)
    assert np.array_equal(synthetic.band_to_dense(back, klp, kup), synthetic.band_to_dense(ab, kl, ku))
    if name == "wide_rows":  # a few wide rows: the profile stores far less than the widest band
        assert buf.nbytes < 0.25 * ab.nbytes


@pytest.mark.gpu
@pytest.mark.parametrize("name,ab,kl,ku", CASES, ids=[c[0] for c in CASES])
def test_profile_fp64_matches_oracle(name, ab, kl, ku):
    n = ab.shape[0]
    x_true = synthetic.planted_x(n, 3, 80_000 + n)
    b = synthetic.band_rhs(ab, kl, ku, x_true)
    fb, _ = oracle.band_lu(ab, kl, ku)
    x_ref = oracle.band_solve(fb, kl, ku, b)
    f = ebv.profile_factor(ab, kl, ku, "fp64")
    x = ebv.solve(f, torch.from_numpy(b).to(DEV)).cpu().numpy()
    assert int(f.info.item()) == 0
    lu = ebv.profile_to_band(f.lu.cpu().numpy(), n, f.kl, f.ku)
    ref = synthetic.band_to_dense(fb, kl, ku)
    assert np.abs(synthetic.band_to_dense(lu, f.kl, f.ku) - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())
    assert np.abs(x - x_ref).max() / np.abs(x_ref).max() <= 1e-11
    r = oracle.band_residual(ab, kl, ku, x, b)
    assert np.abs(r).max() / (np.abs(ab).sum(axis=1).max() * np.abs(x).max()) <= 1e-14
    # FP64 refinement against the profile-stored A (its residual kernel reads
    # the profile; triple-binary32, accurate to ~2^-44 sum |a x|)
    rep = torch.zeros(3, dtype=torch.float64, device=DEV)
    xr = ebv.solve(f, torch.from_numpy(b).to(DEV), refine=(1e-12, 3), report=rep).cpu().numpy()
    assert np.abs(xr - x_ref).max() / np.abs(x_ref).max() <= 1e-11
    r_info = ebv.read_report(rep)
    assert r_info["status"] == 0 and r_info["resid_final"] <= 1e-12


@pytest.mark.gpu
def test_profile_fp32_and_zero_pivot():
    ab, kl, ku = synthetic.laplacian_disc_band(30)
    n = ab.shape[0]
    fb, _ = oracle.band_lu(ab, kl, ku)
    f = ebv.profile_factor(ab, kl, ku, "fp32")
    lu = ebv.profile_to_band(f.lu.cpu().numpy(), n, f.kl, f.ku, "fp32")
    assert np.abs(synthetic.band_to_dense(lu, f.kl, f.ku) - synthetic.band_to_dense(fb, kl, ku)).max() <= 5e-5
    a = synthetic.band_to_dense(ab, kl, ku)
    k = 333
    a[k, :k] = 0.0
    a[:k, k] = 0.0
    a[k, k] = 0.0
    f = ebv.profile_factor(synthetic.dense_to_band(a, kl, ku), kl, ku, "fp64")
    assert int(f.info.item()) == k + 1


def test_profile_descriptor_errors():
    import ctypes
    lib = ebv.lib()
    d = ebv._desc(100, 0, 5, 7, ebv.PROFILE)
    assert lib.ebv_workspace_size(ctypes.byref(d), ebv.FP64, 1) > 0
    d = ebv._desc(100, 0, 100, 7, ebv.PROFILE)
    assert lib.ebv_workspace_size(ctypes.byref(d), ebv.FP64, 1) == 0
    with pytest.raises(ebv.EbvError):
        ebv.ebv_profile_from_band(np.zeros((10, 3)), 1, 2, "fp64")  # ldab < kl + ku + 1
