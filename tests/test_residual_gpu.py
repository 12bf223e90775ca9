"""The refinement residual B - A X (tensor-core evaluation by exact digit
splitting) against the oracle's Dot2 residual.  Bound: every digit product and
every 1024-column partial sum is exact; what is dropped (digit pairs of weight
below 2^-60 and the fixed-point truncation of A and X at 2^-59 of their row /
column scale) stays far below 2^-44 * sum_j |a_ij x_j| for these
diagonally dominant rows, i.e. a few units of the FP64 working precision."""
import numpy as np
import pytest
import torch

import oracle
import paper_1907_05767_gb300 as ebv
import synthetic

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,nrhs", [(1, 1), (33, 2), (1500, 3), (4099, 32), (2000, 40)])
def test_residual_matches_dot2(n, nrhs):
    a = synthetic.dense_dd(n, 0.9, 80_000 + n)
    b = synthetic.uniform(80_000 + n, 5, (n, nrhs), -1.0, 1.0)
    x = np.linalg.solve(a, b)  # near-exact solution: heavy cancellation in b - A x
    r_ref = oracle.residual(a, x, b)
    r = ebv.debug_residual(torch.from_numpy(a).cuda(), torch.from_numpy(x).cuda(),
                           torch.from_numpy(b).cuda()).cpu().numpy()
    mag = np.abs(a) @ np.abs(x)
    err = np.abs(r - r_ref)
    assert np.all(err <= 2.0 ** -44 * mag + 1e-300), (err.max(), (err / mag).max())


def test_residual_of_exact_dyadic_solution_is_zero():
    n = 300
    a = np.round(synthetic.dense_dd(n, 0.9, 3) * 2 ** 20) / 2 ** 20
    np.fill_diagonal(a, 1.0)
    x = np.round(synthetic.planted_x(n, 2, 3) * 2 ** 10) / 2 ** 10
    b = a @ x  # exact: every product and partial sum fits in binary64
    r = ebv.debug_residual(torch.from_numpy(a).cuda(), torch.from_numpy(x).cuda(),
                           torch.from_numpy(b).cuda()).cpu().numpy()
    assert np.all(r == 0.0)
