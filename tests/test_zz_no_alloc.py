"""ebv_solve_static (the solve whose workspace is the library's fixed device
array) against ebv_solve with a caller-allocated workspace and against the
CPU oracle, on the same factors and right-hand sides.  Each case makes two
static calls in a row with different right-hand sides, so the second runs on
the array the first left behind.  Tolerances: X within 1e-11 max-norm
relative of ebv_solve's X (both run the same kernels) and of the oracle's X
(the FP64 bound of the dense tests; refined mixed-precision solves reach it
too); binary32 solves within 1e-4 of the oracle (n * 2^-24 with margin).

The file name makes pytest collect it last; it also passes alone.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1907_05767_gb300 as ebv
import synthetic

DEV = "cuda"


def relerr(x, ref):
    return np.abs(x - ref).max() / np.abs(ref).max()


def _rhs_pair(a, nrhs, seed):
    n = a.shape[0]
    return [synthetic.rhs_for(a, synthetic.planted_x(n, nrhs, seed + k)) for k in range(2)]


def _oracle_x(a, b, band=None):
    if band is None:
        return oracle.solve(oracle.lu(a)[0], b)
    ab, kl, ku = band
    return oracle.band_solve(oracle.band_lu(ab, kl, ku)[0], kl, ku, b)


def _compare(f, a, bs, refine=None, band=None):
    fp32 = f.prec == ebv.FP32
    dt = torch.float32 if fp32 else torch.float64
    for b in bs:
        x_ref = torch.from_numpy(b).to(DEV, dt).contiguous()
        x_st = x_ref.clone()
        rep_ref = rep_st = None
        if refine is not None:
            rep_ref = torch.zeros(3, dtype=torch.float64, device=DEV)
            rep_st = torch.zeros(3, dtype=torch.float64, device=DEV)
        ebv.ebv_solve(f.lu, x_ref, f.prec, a_orig=f.a, refine=refine, report=rep_ref, kl=f.kl, ku=f.ku,
                      storage=f.storage)
        ebv.ebv_solve_static(f.lu, x_st, f.prec, a_orig=f.a, refine=refine, report=rep_st, kl=f.kl, ku=f.ku,
                             storage=f.storage)
        torch.cuda.synchronize()
        xr, xs = x_ref.cpu().double().numpy(), x_st.cpu().double().numpy()
        assert np.isfinite(xs).all()
        assert relerr(xs, xr) <= 1e-11
        assert relerr(xs, _oracle_x(a, b, band)) <= (1e-4 if fp32 else 1e-11)
        if refine is not None:
            assert ebv.read_report(rep_st)["status"] == 0
            assert ebv.read_report(rep_ref)["status"] == 0


@pytest.mark.gpu
def test_static_solve_fp64_dense_matches_solve():
    n = 777
    a = synthetic.dense_dd(n, 0.9, 90_001)
    f = ebv.factor(torch.from_numpy(a).to(DEV), "fp64")
    assert int(f.info.item()) == 0
    _compare(f, a, _rhs_pair(a, 3, 90_011))


@pytest.mark.gpu
def test_static_solve_fp32_dense_matches_solve():
    n = 300
    a = synthetic.dense_dd(n, 0.9, 90_004)
    f = ebv.factor(torch.from_numpy(a).to(DEV), "fp32")
    assert int(f.info.item()) == 0
    _compare(f, a, _rhs_pair(a, 2, 90_051))


@pytest.mark.gpu
def test_static_solve_mixed_refined_matches_solve():
    n = 1000
    a = synthetic.dense_dd(n, 0.9, 90_002)
    f = ebv.factor(torch.from_numpy(a).to(DEV), "bf16")
    assert int(f.info.item()) == 0
    _compare(f, a, _rhs_pair(a, 5, 90_021), refine=(1e-12, 10))


@pytest.mark.gpu
def test_static_solve_at_limits_band_and_dense():
    n, nrhs = ebv.STATIC_MAX_N, ebv.STATIC_MAX_NRHS
    a = synthetic.dense_dd(n, 0.9, 90_003)
    for prec in ("fp64", "bf16"):  # bf16 with refinement: the largest workspace at the limits
        f = ebv.factor(torch.from_numpy(a).to(DEV), prec)
        assert int(f.info.item()) == 0
        _compare(f, a, _rhs_pair(a, nrhs, 90_031), refine=(1e-12, 5))
        del f
    band, kl, ku = synthetic.laplacian_band(64)  # n = 64^2 = 4096, kl = ku = 64
    assert band.shape[0] == n
    fb = ebv.band_factor(torch.from_numpy(band).to(DEV), kl, ku, "fp64")
    assert int(fb.info.item()) == 0
    dense = synthetic.band_to_dense(band, kl, ku)
    _compare(fb, dense, _rhs_pair(dense, 4, 90_041), band=(band, kl, ku))


def test_static_solve_rejects_sizes_beyond_its_array():
    d_big = ebv._desc(ebv.STATIC_MAX_N + 1, ebv.STATIC_MAX_N + 1)
    st = ebv.lib().ebv_solve_static(ctypes.byref(d_big), ebv.FP64, None, None, None, 1, 1, None, None, None)
    assert st == ebv.ERR_WORKSPACE
    d = ebv._desc(16, 16)
    st = ebv.lib().ebv_solve_static(ctypes.byref(d), ebv.FP64, None, None, None, ebv.STATIC_MAX_NRHS + 1,
                                    ebv.STATIC_MAX_NRHS + 1, None, None, None)
    assert st == ebv.ERR_WORKSPACE
    assert ebv.lib().ebv_solve_static(None, ebv.FP64, None, None, None, 1, 1, None, None, None) == ebv.ERR_ARG
