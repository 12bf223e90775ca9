"""Profile (skyline) storage, EBV_PROFILE: each 64-row block keeps its part
from the first non-zero of its rows, each 64-column block its part from the
first non-zero of its columns; no row exchanges, so the factors stay inside
and ebv_factor works in place.  Checked against the CPU oracle's banded
Doolittle on the same matrices (the factors unpacked from the buffer,
element by element, 1e-13; X 1e-11 relative; backward error 1e-14; FP32
factors 5e-5), on an irregular-domain Laplacian, a random profile and a
narrow band with a few wide rows (where the profile stores far less than
the band).  The packer itself is checked on the host: the buffer unpacks
to the input matrix exactly, through the package's decoder and through the
layout the C header documents (tight envelope, byte count, binary32 values).
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


def _decode_as_documented(buf, n, es):
    """The profile buffer read from the layout the C header states, without
    the package's own decoder: int32 lo[nb], int32 up[nb], int64 offL[nb],
    int64 offU[nb], values from byte align256(24 nb); row block b keeps
    columns lo[b] .. 64b+63 of its rows, column block c rows up[c] .. 64c-1
    of its 64 columns, both row-major.  Returns (dense A, stored mask, lo, up)."""
    nb = (n + 63) // 64
    raw = buf.tobytes()
    lo = np.frombuffer(raw, np.int32, nb, 0)
    up = np.frombuffer(raw, np.int32, nb, 4 * nb)
    offl = np.frombuffer(raw, np.int64, nb, 8 * nb)
    offu = np.frombuffer(raw, np.int64, nb, 16 * nb)
    v0 = -(-24 * nb // 256) * 256
    vals = np.frombuffer(raw[v0:], np.float64 if es == 8 else np.float32).astype(np.float64)
    a = np.zeros((n, n))
    stored = np.zeros((n, n), dtype=bool)
    for b in range(nb):
        w = 64 * (b + 1) - lo[b]
        for i in range(64 * b, min(n, 64 * b + 64)):
            cols = np.arange(lo[b], min(n, 64 * b + 64))
            a[i, cols] = vals[offl[b] + (i - 64 * b) * w + (cols - lo[b])]
            stored[i, cols] = True
        cols = np.arange(64 * b, min(n, 64 * b + 64))
        for i in range(up[b], 64 * b):
            a[i, cols] = vals[offu[b] + (i - up[b]) * 64 + (cols - 64 * b)]
            stored[i, cols] = True
    return a, stored, lo, up


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name,ab,kl,ku", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_packer_layout_as_documented(name, ab, kl, ku, prec):
    n = ab.shape[0]
    es = 8 if prec == "fp64" else 4
    buf, klp, kup = ebv.ebv_profile_from_band(ab, kl, ku, prec)
    a = synthetic.band_to_dense(ab, kl, ku)
    got, stored, lo, up = _decode_as_documented(buf, n, es)
    want = a if es == 8 else a.astype(np.float32).astype(np.float64)
    assert np.array_equal(got, np.where(stored, want, 0.0))
    assert not np.any(a[~stored])  # every non-zero lies inside the profile
    nb = (n + 63) // 64
    for b in range(nb):  # the envelope is tight: its first row / column holds a non-zero
        r0, r1 = 64 * b, min(n, 64 * b + 64)
        assert lo[b] == r0 or np.any(a[r0:r1, lo[b]])
        assert not np.any(a[r0:r1, :lo[b]])
        assert up[b] == r0 or np.any(a[up[b], r0:r1])
        assert not np.any(a[:up[b], r0:r1])
    assert klp == min(n - 1, max(min(n, 64 * b + 64) - 1 - lo[b] for b in range(nb)))
    assert kup == min(n - 1, max(min(n, 64 * b + 64) - 1 - up[b] for b in range(nb)))
    count = sum(64 * (64 * (b + 1) - lo[b]) + 64 * (64 * b - up[b]) for b in range(nb))
    assert buf.nbytes == -(-24 * nb // 256) * 256 + es * count


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
