"""The five workloads at their full sizes, on the GPU, against the CPU oracle.

Each test runs one workload in the configuration the benchmark times and
checks the GPU result against ``oracle/`` on the same seeded inputs:

* dense FP64 n = 256, 1 right-hand side: factors element by element (1e-13),
  X against the oracle's X (1e-11 max-norm relative), backward error
  ||b - Ax||_inf / (||A||_inf ||x||_inf) <= 1e-14 (Dot2 residual).
* banded FP64 5-point Laplacian on a 512 x 512 grid (n = 262144, kl = ku =
  512), 8 right-hand sides, general and symmetric band modes (the symmetric
  one also with only the lower half stored): every stored entry of the
  factors against the oracle's banded Doolittle (1e-13), X
  against the oracle's banded substitutions (1e-11), the full backward error
  (<= 1e-14) and the planted solution.
* dense n = 16384, 32 right-hand sides, plain FP64: the backward error over
  every row by the oracle's Dot2 residual (<= 1e-14), the planted solution,
  and the first 384 columns of L and rows of U against the oracle's partial
  elimination (the first 384 steps fix them; 1e-13).  bf16 and fp16
  tensor-core updates with refinement: the relative residual of every column
  (<= 1e-12, the refinement's stop test) by the oracle's Dot2, the device
  report's before/after figures, and the planted solution (1e-11).
* batched: 4096 systems, n ~ U{16..512}, 1-4 right-hand sides, FP64 and FP32
  in one launch: every system's info word and planted solution, and 48
  sampled systems element by element against the oracle (FP64: factors 1e-13,
  X 1e-11, backward error 1e-14; FP32: 5e-5, 1e-4, 1e-5).
* differentiable batch: 256 FP64 systems n = 1024, 4 right-hand sides, loss
  = sum(W * X): gradients of 4 sampled systems against the oracle's adjoint
  (1e-10 relative), and central finite differences (h = 1e-6) of the loss
  through the GPU solver on 64 seeded entries of A and 64 of B:
  |fd - g| <= 1e-6 max(|g|, 1e-3 ||G||_inf).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1907_05767_gb300 as ebv
import synthetic

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
DEV = "cuda"


def bwd_dense(a, x, b, rows=None):
    r = oracle.residual(a, x, b, rows=rows)
    return float(np.abs(r).max() / (np.abs(a).sum(axis=1).max() * np.abs(x).max()))


def relerr(x, ref):
    return float(np.abs(x - ref).max() / np.abs(ref).max())


# ---------------------------------------------------------------------------
# dense FP64 n = 256, one right-hand side
# ---------------------------------------------------------------------------
def test_dense_fp64_n256_one_rhs():
    a, x_true, b = synthetic.config0()
    f = ebv.factor(torch.from_numpy(a).to(DEV), "fp64")
    x = ebv.solve(f, torch.from_numpy(b).to(DEV)).cpu().numpy()
    assert int(f.info.item()) == 0
    lu_ref, info_ref = oracle.lu(a)
    assert info_ref == 0
    assert np.abs(f.lu.cpu().numpy() - lu_ref).max() <= 1e-13
    assert relerr(x, oracle.solve(lu_ref, b)) <= 1e-11
    assert bwd_dense(a, x, b) <= 1e-14
    assert np.abs(x - x_true).max() <= 1e-12


# ---------------------------------------------------------------------------
# banded FP64 Laplacian, 512 x 512 grid, 8 right-hand sides
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def laplacian_512():
    ab, kl, ku, x_true, b = synthetic.config1()
    fb, info = oracle.band_lu(ab, kl, ku)
    assert info == 0
    x_ref = oracle.band_solve(fb, kl, ku, b)
    return ab, kl, ku, x_true, b, fb, x_ref


@pytest.mark.parametrize("sym", [False, True, "lower"])
def test_band_laplacian_512x512(laplacian_512, sym):
    ab, kl, ku, x_true, b, fb, x_ref = laplacian_512
    stored = np.ascontiguousarray(ab[:, :kl + 1]) if sym == "lower" else ab  # lower half: kl + 1 per row
    f = ebv.band_factor(torch.from_numpy(stored).to(DEV), kl, ku, "fp64", sym=sym)
    x = ebv.solve(f, torch.from_numpy(b).to(DEV)).cpu().numpy()
    assert int(f.info.item()) == 0
    lu = f.lu.cpu().numpy()
    del f
    assert np.abs(lu - fb[:, :lu.shape[1]]).max() <= 1e-13
    assert relerr(x, x_ref) <= 1e-11
    r = oracle.band_residual(ab, kl, ku, x, b)
    assert np.abs(r).max() / (np.abs(ab).sum(axis=1).max() * np.abs(x).max()) <= 1e-14
    assert relerr(x, x_true) <= 1e-12


# ---------------------------------------------------------------------------
# dense n = 16384, 32 right-hand sides
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def dense_16384():
    a, x_true, b = synthetic.config2()
    return a, x_true, b


def test_dense_16384_plain_fp64(dense_16384):
    a, x_true, b = dense_16384
    n = a.shape[0]
    A = torch.from_numpy(a).to(DEV)
    f = ebv.factor(A, "fp64", keep_a=False)
    del A
    x = ebv.solve(f, torch.from_numpy(b).to(DEV)).cpu().numpy()
    assert int(f.info.item()) == 0
    # backward error over every row (Dot2 residual)
    assert bwd_dense(a, x, b) <= 1e-14
    assert relerr(x, x_true) <= 1e-12
    # The first k elimination steps fix columns 0..k-1 of L and rows 0..k-1
    # of U: compare those entries with the oracle's partial elimination.
    k = 384
    part, info = oracle.lu(a, kstop=k)
    assert info == 0
    lu = f.lu.cpu().numpy()
    assert np.abs(np.tril(lu[:, :k], -1) - np.tril(part[:, :k], -1)).max() <= 1e-13
    assert np.abs(np.triu(lu[:k, :]) - np.triu(part[:k, :])).max() <= 1e-13
    assert n == 16384


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_dense_16384_mixed_refined(dense_16384, prec):
    a, x_true, b = dense_16384
    f = ebv.factor(torch.from_numpy(a).to(DEV), prec)
    rep = torch.zeros(3, dtype=torch.float64, device=DEV)
    x = ebv.solve(f, torch.from_numpy(b).to(DEV), refine=(1e-12, 10), report=rep).cpu().numpy()
    r_info = ebv.read_report(rep)
    assert int(f.info.item()) == 0
    assert r_info["status"] == 0 and r_info["resid_final"] <= 1e-12
    assert r_info["resid_first"] > r_info["resid_final"]  # the unrefined solve was the low-precision one
    # the stop test's own figure, recomputed by the oracle: max over columns
    # of ||b - Ax||_inf / ||b||_inf (refinement stops once it is <= 1e-12)
    r = oracle.residual(a, x, b)
    rel = (np.abs(r).max(axis=0) / np.abs(b).max(axis=0)).max()
    assert rel <= 1e-12, rel
    assert relerr(x, x_true) <= 1e-11  # ||A^-1||_inf <= 10 here: 10 x the residual bound


# ---------------------------------------------------------------------------
# batched: 4096 systems of uneven order in one launch
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def batched_4096():
    ns, rs = synthetic.config3_sizes()
    systems = [synthetic.config3_system(s, int(ns[s]), int(rs[s])) for s in range(len(ns))]
    return ns, rs, systems


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_4096_systems(batched_4096, prec):
    ns, rs, systems = batched_4096
    tol_f, tol_x, tol_b, tol_t = (1e-13, 1e-11, 1e-14, 1e-12) if prec == "fp64" else (5e-5, 1e-4, 1e-5, 1e-4)
    bt = ebv.Batch(ns, rs, prec)
    for s, (a, _, b) in enumerate(systems):
        bt.a_view(s).copy_(torch.from_numpy(a))
        bt.b_view(s).copy_(torch.from_numpy(b))
    bt.run()
    torch.cuda.synchronize()
    assert int(bt.info.abs().max()) == 0
    a_all = bt.a_buf.double().cpu().numpy()
    b_all = bt.b_buf.double().cpu().numpy()

    def factors(s):
        o, n = int(bt.a_off[s]), int(ns[s])
        return a_all[o:o + n * n].reshape(n, n)

    def solution(s):
        o, n, r = int(bt.b_off[s]), int(ns[s]), int(rs[s])
        return b_all[o:o + n * r].reshape(n, r)

    for s, (_, xt, _) in enumerate(systems):  # every system's planted solution
        assert relerr(solution(s), xt) <= tol_t, s
    for s in synthetic.pick_indices(303, 48, [len(ns)])[:, 0]:
        a, _, b = systems[int(s)]
        lu_ref, info_ref = oracle.lu(a)
        assert info_ref == 0
        x = solution(int(s))
        assert np.abs(factors(int(s)) - lu_ref).max() <= tol_f, s
        assert relerr(x, oracle.solve(lu_ref, b)) <= tol_x, s
        assert bwd_dense(a, x, b) <= tol_b, s


# ---------------------------------------------------------------------------
# differentiable batch: 256 FP64 systems n = 1024, 4 right-hand sides
# ---------------------------------------------------------------------------
def test_adjoint_batch_256_n1024():
    nb, n, nrhs = 256, 1024, 4
    data = [synthetic.config4_system(i, n, nrhs) for i in range(nb)]
    a = np.stack([d[0] for d in data])
    b = np.stack([d[2] for d in data])
    w = np.stack([d[3] for d in data])
    at = torch.from_numpy(a).to(DEV).requires_grad_(True)
    bt = torch.from_numpy(b).to(DEV).requires_grad_(True)
    wt = torch.from_numpy(w).to(DEV)
    x = ebv.EbvSolve.apply(at, bt)
    (wt * x).sum().backward()
    ga, gb = at.grad.cpu().numpy(), bt.grad.cpu().numpy()
    xs = x.detach().cpu().numpy()
    for s in (0, 97, 200, 255):
        lu, _ = oracle.lu(a[s])
        x_ref = oracle.solve(lu, b[s])
        assert relerr(xs[s], x_ref) <= 1e-11
        gb_ref, ga_ref = oracle.adjoint(lu, x_ref, w[s])
        assert np.abs(gb[s] - gb_ref).max() <= 1e-10 * np.abs(gb_ref).max()
        assert np.abs(ga[s] - ga_ref).max() <= 1e-10 * np.abs(ga_ref).max()

    # Central differences of the loss through the GPU solver.  The loss is a
    # sum over systems, so perturbing system s changes only its own term:
    # each difference re-solves system s alone.  A plain FP64 solve carries
    # ~1e-15 of rounding in each of the 4096 entries of X_s, ~6e-14 in the
    # loss, which h = 1e-6 turns into ~3e-8 of noise in a difference, above
    # the 1e-6 relative bound for gradients of a few 1e-2; so the loss is
    # evaluated from the FP64 factors with refinement (FP64-accurate
    # residual on the GPU), whose X is correct to about one rounding.
    def loss_s(s, aa, bb):
        f = ebv.factor(torch.from_numpy(aa).to(DEV), "fp64")
        xx = ebv.solve(f, torch.from_numpy(bb).to(DEV), refine=(1e-16, 3))
        return float((wt[s] * xx).sum())

    h = 1e-6
    gscale = np.abs(w).max()
    for s, i, j in synthetic.pick_indices(404, 64, [nb, n, n]):
        e = np.zeros((n, n))
        e[i, j] = h
        fd = (loss_s(s, a[s] + e, b[s]) - loss_s(s, a[s] - e, b[s])) / (2 * h)
        assert abs(fd - ga[s, i, j]) <= 1e-6 * max(abs(ga[s, i, j]), 1e-3 * gscale), (s, i, j, fd, ga[s, i, j])
    for s, i, c in synthetic.pick_indices(405, 64, [nb, n, nrhs]):
        e = np.zeros((n, nrhs))
        e[i, c] = h
        fd = (loss_s(s, a[s], b[s] + e) - loss_s(s, a[s], b[s] - e)) / (2 * h)
        assert abs(fd - gb[s, i, c]) <= 1e-6 * max(abs(gb[s, i, c]), 1e-3 * gscale), (s, i, c, fd, gb[s, i, c])
