"""ebv_gesv_host (A, B in host memory, the copy of A overlapped with the
factorisation) against the device path ebv_factor + ebv_solve on the same
inputs: the same kernels run on the same data, so X agrees to the dense
tests' FP64 bound (1e-11 max-norm relative) and the refinement reports the
same convergence."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1907_05767_gb300 as ebv
import synthetic


def _report(raw: torch.Tensor) -> dict:
    return ebv.read_report(raw)


@pytest.mark.gpu
@pytest.mark.parametrize("n,nrhs,prec", [(1500, 3, "bf16"), (2500, 1, "fp16"), (4160, 5, "bf16")])
def test_gesv_host_matches_device_path(n, nrhs, prec):
    a = synthetic.dense_dd(n, 0.9, 95_000 + n)
    b = synthetic.rhs_for(a, synthetic.planted_x(n, nrhs, 95_000 + n))
    # device path
    f = ebv.factor(torch.from_numpy(a).cuda(), prec)
    rep_d = torch.zeros(3, dtype=torch.float64, device="cuda")
    x_dev = ebv.solve(f, torch.from_numpy(b).cuda(), refine=(1e-12, 10), report=rep_d).cpu().numpy()
    # host path, A with a padded leading dimension
    a_pad = torch.zeros((n, n + 7), dtype=torch.float64).pin_memory()
    a_pad[:, :n] = torch.from_numpy(a)
    a_host = a_pad[:, :n]
    b_host = torch.from_numpy(b.copy()).pin_memory()
    x_host = torch.zeros_like(b_host).pin_memory()
    rep_h = torch.zeros(32, dtype=torch.uint8).pin_memory()
    info_h = torch.full((1,), -1, dtype=torch.int32).pin_memory()
    ebv.ebv_gesv_host(a_host, b_host, x_host, prec=prec, refine=(1e-12, 10), report_host=rep_h, info_host=info_h)
    torch.cuda.synchronize()
    x = x_host.numpy()
    assert int(info_h[0]) == 0
    assert np.abs(x - x_dev).max() / np.abs(x_dev).max() <= 1e-11
    assert np.array_equal(b_host.numpy(), b)  # B is not modified
    r = _report(rep_h)
    assert r["status"] == 0 and r["resid_final"] <= 1e-12
    lu_ref, _ = oracle.lu(a)
    x_ref = oracle.solve(lu_ref, b)
    assert np.abs(x - x_ref).max() / np.abs(x_ref).max() <= 1e-11


def test_gesv_host_arguments():
    d = ebv._desc(64, 64)
    assert ebv.lib().ebv_gesv_host_workspace_size(ctypes.byref(d), ebv.FP64, 1) == 0
    assert ebv.lib().ebv_gesv_host_workspace_size(ctypes.byref(d), ebv.MIXED_BF16, 1) > 64 * 64 * 12
    st = ebv.lib().ebv_gesv_host(ctypes.byref(d), ebv.FP64, None, None, None, 1, 1, None, None, None, None, 0, None)
    assert st == ebv.ERR_UNSUPPORTED
    band = ebv._desc(64, 3, 1, 1, ebv.BAND)
    st = ebv.lib().ebv_gesv_host(ctypes.byref(band), ebv.MIXED_BF16, None, None, None, 1, 1, None, None, None, None,
                                 0, None)
    assert st == ebv.ERR_ARG
    st = ebv.lib().ebv_gesv_host(ctypes.byref(d), ebv.MIXED_BF16, None, None, None, 1, 1, None, None, None, None, 0,
                                 None)
    assert st == ebv.ERR_ARG  # null host pointers
