"""Adjoint kernels and EbvSolve autograd against the FP64 oracle gradient
(grad_B = A^{-T} G, grad_A = -grad_B X^T; tolerance 1e-10 relative) and
against central finite differences of the GPU forward path (h = 1e-6,
|fd - g| <= 1e-6 * max(|g|, 1e-3 ||G||_inf))."""
import numpy as np
import pytest
import torch

import oracle
import paper_1907_05767_gb300 as ebv
import synthetic

pytestmark = pytest.mark.gpu


def make(batch, n, nrhs, seed):
    a = np.stack([synthetic.dense_dd(n, 0.5, seed + s) for s in range(batch)])
    x = np.stack([synthetic.planted_x(n, nrhs, seed + s) for s in range(batch)])
    b = np.einsum("bij,bjk->bik", a, x)
    w = np.stack([synthetic.gaussian(seed + s, synthetic.STREAM_W, (n, nrhs)) for s in range(batch)])
    return a, b, w


@pytest.mark.parametrize("batch,n,nrhs", [(3, 1, 1), (2, 33, 2), (4, 100, 4), (2, 257, 3)])
def test_adjoint_matches_oracle(batch, n, nrhs):
    a, b, w = make(batch, n, nrhs, 40_000 + n)
    at = torch.from_numpy(a).cuda().requires_grad_(True)
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    x = ebv.EbvSolve.apply(at, bt)
    loss = (torch.from_numpy(w).cuda() * x).sum()
    loss.backward()
    ga, gb = at.grad.cpu().numpy(), bt.grad.cpu().numpy()
    for s in range(batch):
        lu, _ = oracle.lu(a[s])
        xs = oracle.solve(lu, b[s])
        gb_ref, ga_ref = oracle.adjoint(lu, xs, w[s])
        np.testing.assert_allclose(x[s].detach().cpu().numpy(), xs, rtol=0, atol=1e-11 * np.abs(xs).max())
        assert np.abs(gb[s] - gb_ref).max() <= 1e-10 * np.abs(gb_ref).max()
        assert np.abs(ga[s] - ga_ref).max() <= 1e-10 * np.abs(ga_ref).max()


@pytest.mark.parametrize("batch,n,nrhs", [(2, 300, 6), (2, 200, 12), (1, 1700, 9), (1, 97, 16)])
def test_adjoint_kernel_variants(batch, n, nrhs):
    # ebv_solve_adjoint from the oracle's factors: right-hand sides in shared
    # memory with 8 and 16 columns, and (n * 16 doubles above the on-chip
    # budget) the global-memory kernel.
    a, b, w = make(batch, n, nrhs, 42_000 + n)
    lus, xs = [], []
    for s in range(batch):
        lu, _ = oracle.lu(a[s])
        lus.append(lu)
        xs.append(oracle.solve(lu, b[s]))
    gb, ga = ebv.ebv_solve_adjoint(torch.from_numpy(np.stack(lus)).cuda(), torch.from_numpy(np.stack(xs)).cuda(),
                                   torch.from_numpy(w).cuda())
    gb, ga = gb.cpu().numpy(), ga.cpu().numpy()
    for s in range(batch):
        gb_ref, ga_ref = oracle.adjoint(lus[s], xs[s], w[s])
        assert np.abs(gb[s] - gb_ref).max() <= 1e-10 * np.abs(gb_ref).max()
        assert np.abs(ga[s] - ga_ref).max() <= 1e-10 * np.abs(ga_ref).max()


def test_adjoint_finite_differences():
    batch, n, nrhs = 2, 64, 4
    a, b, w = make(batch, n, nrhs, 41_000)
    at = torch.from_numpy(a).cuda().requires_grad_(True)
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    wt = torch.from_numpy(w).cuda()
    (wt * ebv.EbvSolve.apply(at, bt)).sum().backward()
    ga, gb = at.grad.cpu().numpy(), bt.grad.cpu().numpy()

    def loss(aa, bb):
        with torch.no_grad():
            return float((wt * ebv.EbvSolve.apply(torch.from_numpy(aa).cuda(), torch.from_numpy(bb).cuda())).sum())

    h = 1e-6
    gscale = np.abs(w).max()
    idx = synthetic.pick_indices(17, 16, [batch, n, n])
    for s, i, j in idx:
        e = np.zeros_like(a)
        e[s, i, j] = h
        fd = (loss(a + e, b) - loss(a - e, b)) / (2 * h)
        assert abs(fd - ga[s, i, j]) <= 1e-6 * max(abs(ga[s, i, j]), 1e-3 * gscale), (s, i, j, fd, ga[s, i, j])
    idx = synthetic.pick_indices(18, 16, [batch, n, nrhs])
    for s, i, c in idx:
        e = np.zeros_like(b)
        e[s, i, c] = h
        fd = (loss(a, b + e) - loss(a, b - e)) / (2 * h)
        assert abs(fd - gb[s, i, c]) <= 1e-6 * max(abs(gb[s, i, c]), 1e-3 * gscale), (s, i, c, fd, gb[s, i, c])


def test_adjoint_identities_and_no_grad_a():
    batch, n, nrhs = 3, 150, 2
    a, b, w = make(batch, n, nrhs, 42_000)
    lu = torch.from_numpy(a).cuda().contiguous().clone()
    x = torch.from_numpy(b).cuda().contiguous().clone()
    bt = ebv.uniform_batch(lu, x)
    bt.run()
    gb, ga = ebv.ebv_solve_adjoint(lu, x, torch.from_numpy(w).cuda(), want_grad_a=False)
    assert ga is None
    gbn = gb.cpu().numpy()
    for s in range(batch):
        # A^T grad_B = G
        np.testing.assert_allclose(a[s].T @ gbn[s], w[s], rtol=0, atol=1e-13 * np.abs(w[s]).max())
