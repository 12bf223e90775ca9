"""Pins that tie the CPU oracle to things other than itself.

Each ``pin_*`` takes a loaded oracle library (``oracle.load()`` or a copy built
with a planted mistake) and raises AssertionError when the oracle disagrees with
what the paper or the mathematics fixes:

* hand-worked fixtures under tests/golden/ (Eq. 1, Eq. 6a/6c);
* planted exact dyadic factors (the no-pivot LU is unique, so any correct
  elimination returns them bit for bit);
* closed forms: diagonal, triangular, tridiagonal (Thomas recurrence),
  block-diagonal matrices;
* brute force: Leibniz determinants and Cramer's rule in exact rationals;
* a library routine: LAPACK partial-pivoting LU (scipy) on a column-dominant
  matrix, where partial pivoting takes no row exchange and so must return the
  same factors; LAPACK banded solve; numpy's dense solve for A^T;
* invariants: A = LU to 1e-13, structural zeros/ones, fill confined to the band,
  central finite differences for the adjoint, exact-rational residuals;
* the product-form inverse (Eq. 4c): a hand-worked 3 x 3, adjugates of Leibniz
  cofactors in exact rationals, closed forms (diagonal, bidiagonal with exact
  dyadic inverses, block diagonal), A X = X A = I and LAPACK's inverse.
"""
from __future__ import annotations

import itertools
import os
from fractions import Fraction

import numpy as np

import oracle
import synthetic

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name: str) -> dict:
    """Parse a golden fixture: '#' comments, then blocks 'NAME' + rows of numbers."""
    out, cur, rows = {}, None, []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            toks = line.split()
            if len(toks) == 1 and not _is_number(toks[0]):
                if cur is not None:
                    out[cur] = np.array(rows, dtype=np.float64)
                cur, rows = toks[0], []
            else:
                rows.append([float(t) for t in toks])
    if cur is not None:
        out[cur] = np.array(rows, dtype=np.float64)
    return out


def _is_number(t: str) -> bool:
    try:
        float(t)
        return True
    except ValueError:
        return False


def _exact_matmul(x, y):
    """Exact rational product of two float matrices (returns Fractions)."""
    xf = [[Fraction(float(v)) for v in row] for row in x]
    yf = [[Fraction(float(v)) for v in row] for row in y]
    n, k, m = len(xf), len(yf), len(yf[0])
    return [[sum((xf[i][p] * yf[p][j] for p in range(k)), Fraction(0)) for j in range(m)] for i in range(n)]


def _leibniz_det(m) -> Fraction:
    """det by the Leibniz permutation expansion, in exact rationals."""
    n = len(m)
    total = Fraction(0)
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        prod = Fraction(1)
        for i in range(n):
            prod *= m[i][perm[i]]
        total += -prod if inv % 2 else prod
    return total


def _frac_matrix(a):
    return [[Fraction(float(v)) for v in row] for row in a]


# ----------------------------------------------------------------------------
# Pins
# ----------------------------------------------------------------------------

def pin_golden_factor_and_solve(lib):
    for name in ("doolittle_2x2.txt", "doolittle_3x3_integer.txt", "doolittle_3x3_dyadic.txt"):
        g = read_golden(name)
        f, info = oracle.lu(g["A"], lib=lib)
        assert info == 0, name
        lo, up = oracle.unpack(f)
        assert np.array_equal(lo, g["L"]), (name, lo)
        assert np.array_equal(up, g["U"]), (name, up)
        x = oracle.solve(f, g["b"], lib=lib)
        assert np.array_equal(x, g["x"]), (name, x)


def pin_golden_adjoint(lib):
    g = read_golden("adjoint_3x3.txt")
    f, _ = oracle.lu(g["A"], lib=lib)
    gb, ga = oracle.adjoint(f, g["x"], g["G"], lib=lib)
    assert np.array_equal(gb, g["grad_b"]), gb
    assert np.array_equal(ga, g["grad_A"]), ga


def _planted_dyadic(n: int, seed: int):
    rng = np.random.default_rng(seed)
    lvals = np.array([0.0, 0.125, -0.125, 0.25, -0.25, 0.5, -0.5])
    uvals = np.array([0.0, 0.25, -0.25, 0.5, -0.5, 1.0, -1.0])
    dvals = np.array([1.0, 2.0, 4.0, -2.0, 0.5])
    lo = np.tril(rng.choice(lvals, size=(n, n)), -1) + np.eye(n)
    up = np.triu(rng.choice(uvals, size=(n, n)), 1) + np.diag(rng.choice(dvals, size=n))
    exact = _exact_matmul(lo, up)
    a = np.array([[float(v) for v in row] for row in exact])
    assert all(Fraction(a[i, j]) == exact[i][j] for i in range(n) for j in range(n))
    return lo, up, a


def pin_planted_dyadic_factors(lib):
    for n in (1, 2, 3, 5, 8, 13):
        for seed in range(3):
            lo, up, a = _planted_dyadic(n, 100 * n + seed)
            f, info = oracle.lu(a, lib=lib)
            assert info == 0
            l2, u2 = oracle.unpack(f)
            assert np.array_equal(l2, lo), (n, seed)
            assert np.array_equal(u2, up), (n, seed)
            xint = np.arange(1, n + 1, dtype=np.float64)[:, None] * np.array([[1.0, -2.0]])
            bx = _exact_matmul(a, xint)
            b = np.array([[float(v) for v in row] for row in bx])
            x = oracle.solve(f, b, lib=lib)
            assert np.array_equal(x, xint), (n, seed, x)


def pin_closed_forms(lib):
    rng = np.random.default_rng(7)
    n = 9
    # diagonal: L = I, U = A
    d = np.diag(rng.uniform(0.5, 2.0, n))
    f, _ = oracle.lu(d, lib=lib)
    assert np.array_equal(f, d)
    # upper triangular: L = I, U = A
    up = np.triu(rng.uniform(-1, 1, (n, n)), 1) + np.diag(rng.uniform(1, 2, n))
    f, _ = oracle.lu(up, lib=lib)
    assert np.array_equal(f, up)
    # lower triangular: U = diag(A), L = A diag(A)^{-1}
    lw = np.tril(rng.uniform(-1, 1, (n, n)), -1) + np.diag(rng.uniform(1, 2, n))
    f, _ = oracle.lu(lw, lib=lib)
    lo, u2 = oracle.unpack(f)
    assert np.array_equal(u2, np.diag(np.diag(lw)))
    assert np.array_equal(lo, lw / np.diag(lw)[None, :])
    # tridiagonal: Thomas recurrence u_i = a_ii - (a_{i,i-1}/u_{i-1}) a_{i-1,i}
    sub, dia, sup = rng.uniform(-1, 1, n - 1), rng.uniform(3, 4, n), rng.uniform(-1, 1, n - 1)
    t = np.diag(dia) + np.diag(sub, -1) + np.diag(sup, 1)
    uu = np.empty(n)
    ll = np.empty(n - 1)
    uu[0] = dia[0]
    for i in range(1, n):
        ll[i - 1] = sub[i - 1] / uu[i - 1]
        uu[i] = dia[i] - ll[i - 1] * sup[i - 1]
    f, _ = oracle.lu(t, lib=lib)
    np.testing.assert_allclose(np.diag(f), uu, rtol=1e-15, atol=0)
    np.testing.assert_allclose(np.diag(f, -1), ll, rtol=1e-15, atol=0)
    assert np.array_equal(np.diag(f, 1), sup)
    assert not np.any(np.tril(f, -2)) and not np.any(np.triu(f, 2))
    # block diagonal: factors of the blocks, independently
    a1 = synthetic.dense_dd(4, 0.5, 11)
    a2 = synthetic.dense_dd(5, 0.5, 12)
    blk = np.zeros((9, 9))
    blk[:4, :4] = a1
    blk[4:, 4:] = a2
    f, _ = oracle.lu(blk, lib=lib)
    f1, _ = oracle.lu(a1, lib=lib)
    f2, _ = oracle.lu(a2, lib=lib)
    assert np.array_equal(f[:4, :4], f1) and np.array_equal(f[4:, 4:], f2)
    assert not np.any(f[:4, 4:]) and not np.any(f[4:, :4])


def pin_reconstruction(lib):
    for n, w in ((50, 0.5), (97, 0.9), (128, 0.9)):
        a = synthetic.dense_dd(n, w, 1000 + n)
        f, info = oracle.lu(a, lib=lib)
        assert info == 0
        lo, up = oracle.unpack(f)
        assert np.array_equal(np.diag(lo), np.ones(n))
        err = np.abs(a - lo @ up).sum(axis=1).max() / np.abs(a).sum(axis=1).max()
        assert err <= 1e-13, err


def pin_det_leibniz(lib):
    for n in range(1, 7):
        a = synthetic.dense_dd(n, 0.9, 2000 + n) + np.triu(np.full((n, n), 0.25), 1)
        f, _ = oracle.lu(a, lib=lib)
        det_lu = float(np.prod(np.diag(f)))
        det_ex = float(_leibniz_det(_frac_matrix(a)))
        assert abs(det_lu - det_ex) <= 1e-14 * abs(det_ex), (n, det_lu, det_ex)


def pin_cramer(lib):
    for n in range(1, 7):
        a = synthetic.dense_dd(n, 0.9, 3000 + n)
        b = synthetic.uniform(3000 + n, 9, (n, 1), -1.0, 1.0)
        f, _ = oracle.lu(a, lib=lib)
        x = oracle.solve(f, b, lib=lib)
        af = _frac_matrix(a)
        det = _leibniz_det(af)
        for i in range(n):
            ai = [row[:] for row in af]
            for r in range(n):
                ai[r][i] = Fraction(float(b[r, 0]))
            xi = float(_leibniz_det(ai) / det)
            assert abs(x[i, 0] - xi) <= 1e-14 * max(1.0, abs(xi)), (n, i, x[i, 0], xi)


def pin_lapack_lu_column_dominant(lib):
    import scipy.linalg
    for n in (6, 40, 75):
        # transpose of a strictly row-dominant matrix: strictly column dominant, so
        # partial pivoting keeps every diagonal pivot and LAPACK's factors are the
        # no-pivot factors
        a = np.ascontiguousarray(synthetic.dense_dd(n, 0.9, 4000 + n).T)
        p, lo_ref, up_ref = scipy.linalg.lu(a)
        assert np.array_equal(p, np.eye(n))
        f, _ = oracle.lu(a, lib=lib)
        lo, up = oracle.unpack(f)
        # blocked LAPACK and the plain loop round in different orders: a few ulps
        np.testing.assert_allclose(lo, lo_ref, rtol=4e-15, atol=1e-17)
        np.testing.assert_allclose(up, up_ref, rtol=4e-15, atol=1e-17)


def pin_planted_solution(lib):
    a, x_true, b = synthetic.config0(256, 3)
    f, _ = oracle.lu(a, lib=lib)
    x = oracle.solve(f, b, lib=lib)
    assert np.abs(x - x_true).max() <= 1e-13
    np.testing.assert_allclose(x, np.linalg.solve(a, b), rtol=0, atol=1e-14)


def pin_band(lib):
    import scipy.linalg
    ab, kl, ku = synthetic.laplacian_band(8)
    a = synthetic.band_to_dense(ab, kl, ku)
    fb, info = oracle.band_lu(ab, kl, ku, lib=lib)
    assert info == 0
    fd, _ = oracle.lu(a, lib=lib)
    # fill confined to the band, and the band equals the dense factors there
    n = a.shape[0]
    outside = np.abs(np.subtract.outer(np.arange(n), np.arange(n)))
    outside = (np.subtract.outer(np.arange(n), np.arange(n)) > kl) | (np.subtract.outer(np.arange(n), np.arange(n)) < -ku)
    assert not np.any(fd[outside])
    assert np.array_equal(synthetic.band_to_dense(fb, kl, ku), fd)
    x_true = synthetic.planted_x(n, 3, 77)
    b = synthetic.band_rhs(ab, kl, ku, x_true)
    np.testing.assert_allclose(b, a @ x_true, rtol=0, atol=1e-14)
    x = oracle.band_solve(fb, kl, ku, b, lib=lib)
    # LAPACK banded solver (partial pivoting; this Laplacian is strictly column
    # dominant, so no row is exchanged)
    lap = np.zeros((kl + ku + 1, n))
    for j in range(n):
        for i in range(max(0, j - ku), min(n, j + kl + 1)):
            lap[ku + i - j, j] = a[i, j]
    xr = scipy.linalg.solve_banded((kl, ku), lap, b)
    np.testing.assert_allclose(x, xr, rtol=0, atol=1e-14)
    np.testing.assert_allclose(x, x_true, rtol=0, atol=1e-13)
    # unsymmetric band with kl != ku
    n2, kl2, ku2 = 30, 2, 5
    a2 = synthetic.dense_dd(n2, 0.9, 5001)
    mask = (np.subtract.outer(np.arange(n2), np.arange(n2)) > kl2) | (np.subtract.outer(np.arange(n2), np.arange(n2)) < -ku2)
    a2[mask] = 0.0
    fb2, _ = oracle.band_lu(synthetic.dense_to_band(a2, kl2, ku2), kl2, ku2, lib=lib)
    fd2, _ = oracle.lu(a2, lib=lib)
    assert np.array_equal(synthetic.band_to_dense(fb2, kl2, ku2), fd2)
    x2 = oracle.band_solve(fb2, kl2, ku2, np.ones((n2, 1)), lib=lib)
    np.testing.assert_allclose(x2, np.linalg.solve(a2, np.ones((n2, 1))), rtol=0, atol=1e-14)


def profile_of(a):
    """First non-zero column left of the diagonal per row (i when none) and
    first non-zero row above the diagonal per column (j when none)."""
    n = a.shape[0]
    lo = np.array([next((j for j in range(i) if a[i, j] != 0.0), i) for i in range(n)])
    up = np.array([next((i for i in range(j) if a[i, j] != 0.0), j) for j in range(n)])
    return lo, up


def variable_profile_dd(n: int, kl: int, ku: int, seed: int):
    """Strictly row-dominant matrix whose row / column profile is drawn at random
    inside a kl / ku band (test input for the profile pins and tests)."""
    rng = np.random.default_rng(seed)
    a = np.zeros((n, n))
    for i in range(n):
        f = i - int(rng.integers(0, min(i, kl) + 1))
        a[i, f:i] = rng.uniform(-1.0, 1.0, i - f)
        if f < i:
            a[i, f] = 0.5
    for j in range(n):
        g = j - int(rng.integers(0, min(j, ku) + 1))
        a[g:j, j] = rng.uniform(-1.0, 1.0, j - g)
        if g < j:
            a[g, j] = -0.5
    a += np.diag(np.abs(a).sum(axis=1) + 1.0)
    return a


def pin_band_profile(lib):
    # Without row exchanges the factors stay inside the profile: L_ij = 0 left of
    # row i's first non-zero and U_ij = 0 above column j's first non-zero, and the
    # band factors equal the dense ones (irregular-domain Laplacian and a random
    # variable profile).
    ab, kl, ku = synthetic.laplacian_disc_band(7)
    cases = [(synthetic.band_to_dense(ab, kl, ku), kl, ku), (variable_profile_dd(70, 9, 13, 8), 9, 13)]
    for c, (a, kl, ku) in enumerate(cases):
        n = a.shape[0]
        lo, up = profile_of(a)
        assert (lo < np.arange(n)).any() and (lo > np.arange(n) - kl).any()  # the profile is uneven
        fb, info = oracle.band_lu(synthetic.dense_to_band(a, kl, ku), kl, ku, lib=lib)
        assert info == 0
        f = synthetic.band_to_dense(fb, kl, ku)
        assert np.array_equal(f, oracle.lu(a, lib=lib)[0])
        i, j = np.indices((n, n))
        assert not np.any(f[(j < i) & (j < lo[:, None])])
        assert not np.any(f[(i < j) & (i < up[None, :])])
        if c == 0:  # the Laplacian is sparse inside its profile, and the factors fill it
            inner = (j < i) & (j >= lo[:, None])
            assert np.count_nonzero(f[inner]) > np.count_nonzero(a[inner])


def pin_symmetric_ldlt(lib):
    # Symmetric A (the reading of eq. 6a-b that scales both vectors by the same
    # pivot): Doolittle's U is D L^T with D the pivots.  For symmetric,
    # strictly diagonally dominant A with a positive diagonal A is positive
    # definite, and the Cholesky factor R (A = R R^T, numpy) gives the same
    # L = R diag(1/r_ii) and D = diag(r_ii^2) independently.
    n = 40
    a = synthetic.dense_dd(n, 0.9, 6001)
    a = 0.5 * (a + a.T)
    f, info = oracle.lu(a, lib=lib)
    assert info == 0
    L = np.tril(f, -1) + np.eye(n)
    U = np.triu(f)
    d = np.diag(U)
    np.testing.assert_allclose(U, np.diag(d) @ L.T, rtol=0, atol=1e-15)
    r = np.linalg.cholesky(a)
    np.testing.assert_allclose(L, r / np.diag(r), rtol=0, atol=1e-14)
    np.testing.assert_allclose(d, np.diag(r) ** 2, rtol=1e-14, atol=0)
    # the symmetric band: the 2-D Laplacian (symmetric, kl == ku)
    ab, kl, ku = synthetic.laplacian_band(7)
    fb, info = oracle.band_lu(ab, kl, ku, lib=lib)
    assert info == 0
    fd = synthetic.band_to_dense(fb, kl, ku)
    Lb = np.tril(fd, -1) + np.eye(fd.shape[0])
    Ub = np.triu(fd)
    np.testing.assert_allclose(Ub, np.diag(np.diag(Ub)) @ Lb.T, rtol=0, atol=1e-14)


def pin_adjoint(lib):
    n, nrhs = 12, 3
    a = synthetic.dense_dd(n, 0.9, 6001)
    b = synthetic.uniform(6001, 5, (n, nrhs), -1.0, 1.0)
    w = synthetic.gaussian(6001, synthetic.STREAM_W, (n, nrhs))
    f, _ = oracle.lu(a, lib=lib)
    x = oracle.solve(f, b, lib=lib)
    gb, ga = oracle.adjoint(f, x, w, lib=lib)
    np.testing.assert_allclose(a.T @ gb, w, rtol=0, atol=1e-14)
    np.testing.assert_allclose(gb, np.linalg.solve(a.T, w), rtol=0, atol=1e-14)
    np.testing.assert_allclose(ga, -gb @ x.T, rtol=0, atol=1e-15)

    def loss(am, bm):
        fm, _ = oracle.lu(am, lib=lib)
        return float(np.sum(w * oracle.solve(fm, bm, lib=lib)))

    h = 1e-6
    for (i, j) in ((0, 0), (3, 7), (11, 2), (5, 5)):
        e = np.zeros_like(a)
        e[i, j] = h
        fd = (loss(a + e, b) - loss(a - e, b)) / (2 * h)
        assert abs(fd - ga[i, j]) <= 1e-7 * max(1.0, abs(ga[i, j])), (i, j, fd, ga[i, j])
    for (i, c) in ((0, 0), (6, 2), (11, 1)):
        e = np.zeros_like(b)
        e[i, c] = h
        fd = (loss(a, b + e) - loss(a, b - e)) / (2 * h)
        assert abs(fd - gb[i, c]) <= 1e-7 * max(1.0, abs(gb[i, c])), (i, c, fd, gb[i, c])


def pin_residual(lib):
    # residual of a nearly exact solution: heavy cancellation, which plain
    # binary64 evaluation gets wrong in its leading digits
    n = 7
    a = synthetic.dense_dd(n, 0.9, 7001) + 0.3
    b = synthetic.uniform(7001, 5, (n, 2), -1.0, 1.0)
    x = np.linalg.solve(a, b)
    r = oracle.residual(a, x, b, lib=lib)
    af = _frac_matrix(a)
    for c in range(2):
        for i in range(n):
            ex = Fraction(float(b[i, c])) - sum(af[i][j] * Fraction(float(x[j, c])) for j in range(n))
            mag = sum(abs(af[i][j] * Fraction(float(x[j, c]))) for j in range(n))
            assert abs(Fraction(r[i, c]) - ex) <= Fraction(1.2e-16) * abs(ex) + Fraction(1e-30) * mag, (i, c)
    rows = np.array([5, 0, 3])
    np.testing.assert_array_equal(oracle.residual(a, x, b, rows=rows, lib=lib), r[rows])
    # band residual on the grid Laplacian equals the dense one
    ab, kl, ku = synthetic.laplacian_band(4)
    ad = synthetic.band_to_dense(ab, kl, ku)
    xx = synthetic.planted_x(16, 2, 9)
    bb = synthetic.uniform(9, 5, (16, 2), -1, 1)
    np.testing.assert_array_equal(oracle.band_residual(ab, kl, ku, xx, bb, lib=lib),
                                  oracle.residual(ad, xx, bb, lib=lib))


def pin_partial_factorisation(lib):
    n, k = 40, 13
    a = synthetic.dense_dd(n, 0.9, 8001)
    full, _ = oracle.lu(a, lib=lib)
    part, _ = oracle.lu(a, kstop=k, lib=lib)
    assert np.array_equal(part[:, :k], full[:, :k])
    assert np.array_equal(part[:k, :], full[:k, :])
    l21 = part[k:, :k]
    u12 = part[:k, k:]
    l11 = np.tril(part[:k, :k], -1) + np.eye(k)
    np.testing.assert_allclose(l11 @ u12, a[:k, k:], rtol=0, atol=1e-15)
    np.testing.assert_allclose(part[k:, k:], a[k:, k:] - l21 @ u12, rtol=0, atol=1e-15)


def pin_info(lib):
    _, info = oracle.lu(np.array([[0.0, 1.0], [1.0, 0.0]]), lib=lib)
    assert info == 1
    _, info = oracle.lu(np.array([[1.0, 1.0, 0.0], [1.0, 1.0, 2.0], [0.0, 3.0, 1.0]]), lib=lib)
    assert info == 2
    _, info = oracle.lu(np.array([[1.0, 0.0], [0.0, np.nan]]), lib=lib)
    assert info == 2
    ab = np.array([[0.0, 2.0, 1.0], [1.0, 0.5, 1.0], [1.0, 1.0, 0.0]])
    _, info = oracle.band_lu(ab, 1, 1, lib=lib)
    assert info == 2  # 0.5 - (1/2) * 1 = 0


def _adjugate_inverse(a):
    """A^{-1} = adj(A) / det A from Leibniz cofactors, in exact rationals."""
    m = _frac_matrix(a)
    n = len(m)
    det = _leibniz_det(m)
    out = [[Fraction(0)] * n for _ in range(n)]
    for i in range(n):
        for j in range(n):
            minor = [row[:i] + row[i + 1:] for r, row in enumerate(m) if r != j]
            c = _leibniz_det(minor) if n > 1 else Fraction(1)
            out[i][j] = (c if (i + j) % 2 == 0 else -c) / det
    return out


def pin_golden_inverse(lib):
    g = read_golden("inverse_3x3.txt")
    f, info = oracle.lu(g["A"], lib=lib)
    assert info == 0
    x = oracle.inverse(f, lib=lib)
    assert np.array_equal(x, g["Ainv"]), x
    lo, up = oracle.unpack(f)
    assert np.array_equal(oracle.inverse(lo, lib=lib), g["Linv"])
    assert np.array_equal(oracle.inverse(up, lib=lib), g["Uinv"])


def pin_inverse_leibniz(lib):
    for n in range(1, 7):
        for seed in range(2):
            a = synthetic.dense_dd(n, 0.9, 5000 + 10 * n + seed) + np.triu(np.full((n, n), 0.125), 1)
            f, info = oracle.lu(a, lib=lib)
            assert info == 0
            x = oracle.inverse(f, lib=lib)
            ex = _adjugate_inverse(a)
            scale = max(abs(v) for row in ex for v in row)
            err = max(abs(Fraction(float(x[i, j])) - ex[i][j]) for i in range(n) for j in range(n))
            assert float(err) <= 1e-14 * float(scale), (n, seed, float(err))


def pin_inverse_closed_forms(lib):
    # diagonal: 1 / a_ii
    d = np.array([2.0, -4.0, 0.5, 8.0, 1.0, -0.25])
    f, _ = oracle.lu(np.diag(d), lib=lib)
    assert np.array_equal(oracle.inverse(f, lib=lib), np.diag(1.0 / d))
    n = 14
    i, j = np.indices((n, n))
    # unit lower bidiagonal, -1/2 below the diagonal: (A^{-1})_ij = 2^{-(i-j)} for i >= j
    lo = np.eye(n) - 0.5 * np.eye(n, k=-1)
    f, _ = oracle.lu(lo, lib=lib)
    assert np.array_equal(oracle.inverse(f, lib=lib), np.where(i >= j, 0.5 ** (i - j), 0.0))
    # upper bidiagonal 2I + N: A^{-1} = (1/2) sum_k (-N/2)^k, (A^{-1})_ij = (1/2)(-1/2)^{j-i} for j >= i
    up = 2.0 * np.eye(n) + np.eye(n, k=1)
    f, _ = oracle.lu(up, lib=lib)
    assert np.array_equal(oracle.inverse(f, lib=lib), np.where(j >= i, 0.5 * (-0.5) ** (j - i), 0.0))
    # block diagonal: the inverses of the blocks
    a1 = synthetic.dense_dd(5, 0.7, 21)
    a2 = synthetic.dense_dd(4, 0.7, 22)
    blk = np.zeros((9, 9))
    blk[:5, :5] = a1
    blk[5:, 5:] = a2
    x = oracle.inverse(oracle.lu(blk, lib=lib)[0], lib=lib)
    assert np.array_equal(x[:5, :5], oracle.inverse(oracle.lu(a1, lib=lib)[0], lib=lib))
    assert np.array_equal(x[5:, 5:], oracle.inverse(oracle.lu(a2, lib=lib)[0], lib=lib))
    assert not np.any(x[:5, 5:]) and not np.any(x[5:, :5])
    # tridiag(-1, 2, -1) of order m (1-based indices): (A^{-1})_ij = min(i, j) (m + 1 - max(i, j)) / (m + 1)
    # (its pivots (k+1)/k never vanish, so the no-pivot factors exist)
    m = 24
    t = 2.0 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
    i1, j1 = np.indices((m, m)) + 1
    closed = np.minimum(i1, j1) * (m + 1 - np.maximum(i1, j1)) / (m + 1.0)
    x = oracle.inverse(oracle.lu(t, lib=lib)[0], lib=lib)
    assert np.abs(x - closed).max() <= 1e-13 * np.abs(closed).max()
    # 2 x 2: [[a, b], [c, d]]^{-1} = [[d, -b], [-c, a]] / (ad - bc)
    a = np.array([[4.0, 3.0], [6.0, 3.0]])
    x = oracle.inverse(oracle.lu(a, lib=lib)[0], lib=lib)
    np.testing.assert_allclose(x, np.array([[3.0, -3.0], [-6.0, 4.0]]) / -6.0, rtol=2e-16, atol=0)


def pin_inverse_invariants(lib):
    for n, w in ((33, 0.5), (100, 0.9)):
        a = synthetic.dense_dd(n, w, 6000 + n)
        x = oracle.inverse(oracle.lu(a, lib=lib)[0], lib=lib)
        e = np.eye(n)
        assert np.abs(a @ x - e).max() <= 1e-14 and np.abs(x @ a - e).max() <= 1e-14
        np.testing.assert_allclose(x, np.linalg.inv(a), rtol=0, atol=1e-14)


ALL_PINS = [
    pin_golden_factor_and_solve,
    pin_golden_adjoint,
    pin_planted_dyadic_factors,
    pin_closed_forms,
    pin_reconstruction,
    pin_det_leibniz,
    pin_cramer,
    pin_lapack_lu_column_dominant,
    pin_planted_solution,
    pin_band,
    pin_band_profile,
    pin_symmetric_ldlt,
    pin_adjoint,
    pin_residual,
    pin_partial_factorisation,
    pin_info,
    pin_golden_inverse,
    pin_inverse_leibniz,
    pin_inverse_closed_forms,
    pin_inverse_invariants,
]
