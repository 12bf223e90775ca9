"""Failure detection without faulting the GPU: a bounded device wait on a flag
that nothing sets must expire, record EBV_ERR_TIMEOUT in the workspace status
block and return; the context stays usable afterwards.  Numerical failures are
covered where they occur (info words in the dense, band and batched tests; the
not-converged refinement status below)."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1907_05767_gb300 as ebv
import synthetic

pytestmark = pytest.mark.gpu


def test_bounded_wait_expires_and_reports():
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    st = ebv.lib().ebv_debug_wait_probe(1000, ctypes.c_void_p(ws.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == ebv.OK
    torch.cuda.synchronize()
    words = ws[:16].cpu().view(torch.int32).tolist()
    assert words == [ebv.ERR_TIMEOUT, 77, 0, 1]
    # the context is still healthy: a normal solve runs and is correct
    a, x_true, b = synthetic.config0(64, 1)
    f = ebv.factor(torch.from_numpy(a).cuda(), "fp64")
    x = ebv.solve(f, torch.from_numpy(b).cuda()).cpu().numpy()
    assert np.abs(x - x_true).max() < 1e-12


def test_probe_rejects_bad_arguments():
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    assert ebv.lib().ebv_debug_wait_probe(0, ctypes.c_void_p(ws.data_ptr()), None) == ebv.ERR_ARG
    assert ebv.lib().ebv_debug_wait_probe(10, None, None) == ebv.ERR_WORKSPACE


def test_refinement_reports_not_converged():
    # max_iter = 0 with a bfloat16 factorisation cannot reach 1e-14: the
    # device report says so (no host synchronisation inside the call).
    n = 300
    a = synthetic.dense_dd(n, 0.9, 5)
    b = synthetic.rhs_for(a, synthetic.planted_x(n, 2, 5))
    f = ebv.factor(torch.from_numpy(a).cuda(), "bf16")
    rep = torch.zeros(3, dtype=torch.float64, device="cuda")
    ebv.solve(f, torch.from_numpy(b).cuda(), refine=(1e-14, 0), report=rep)
    r = ebv.read_report(rep)
    assert r["status"] == ebv.ERR_NOT_CONVERGED and r["iters"] == 0 and r["resid_final"] > 1e-14
