"""Seeded synthetic inputs for the EbV solver and for its CPU oracle.

This module only draws inputs.  It holds none of the method's arithmetic (no
factorisation, no substitution); both the CUDA path's tests/bench and the oracle
take their matrices and right-hand sides from here, so the two see bit-identical
inputs.

Random numbers come from the counter-based SplitMix64 finaliser (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): value i of
stream s under seed k is ``mix64(key(k, s) + (i + 1) * GAMMA)``, turned into a
53-bit uniform double in [0, 1).  Everything is numpy uint64 arithmetic, so the
same numbers come out on x86 and Arm.

The matrix classes follow the paper's input class: a unit-diagonal, strictly
row-diagonally-dominant coefficient matrix (Eq. 2).  Recipes:

* ``dense_dd(n, w, seed)``: a_ii = 1, a_ij ~ U[-w, w] / (n - 1) for i != j, so
  every row's off-diagonal sum is below w < 1 (strict row dominance).
* ``laplacian_band(g)``: 2D 5-point Laplacian on a g x g grid, natural ordering,
  Dirichlet boundary (edge nodes lack their outside neighbours), diagonal 4.1,
  neighbours -1, stored as a row band with kl = ku = g.
* ``laplacian_disc_band(r)``: the same operator on the grid points of a disc of
  radius r (an irregular domain), ordered row by row; the distance to a node's
  neighbour in the next grid row follows the chord length, so the band's width
  varies from row to row (a profile, or skyline, matrix stored in its widest
  band, kl = ku = the largest distance).
* planted solutions ``x_true ~ U[-1, 1]`` with ``b = A @ x_true``.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Streams inside one seed.
STREAM_A = 0
STREAM_X = 1
STREAM_META = 2
STREAM_W = 3
STREAM_PICK = 4

BASE_SEED = 1907057670


def seed_for(config: int, system: int = 0) -> int:
    """Seed of system ``system`` of workload ``config`` (0..4)."""
    return BASE_SEED + 1000 * config + system


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        k = np.array([(seed & 0xFFFFFFFFFFFFFFFF)], dtype=np.uint64)
        k ^= np.uint64(stream) * GAMMA
        return _mix64(k)[0]


def uniform01(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Counter-based uniforms in [0, 1): values ``start .. start+count-1`` of a stream."""
    key = _key(seed, stream)
    with np.errstate(over="ignore"):
        ctr = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = _mix64(key + ctr * GAMMA)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(seed: int, stream: int, shape, lo: float, hi: float, start: int = 0) -> np.ndarray:
    count = int(np.prod(shape))
    u = uniform01(seed, stream, start, count)
    return (lo + (hi - lo) * u).reshape(shape)


def dense_dd(n: int, w: float, seed: int, dtype=np.float64) -> np.ndarray:
    """Unit-diagonal, strictly row-diagonally-dominant n x n matrix (row-major).

    Off-diagonals are U[-w, w] / (n - 1), drawn in row-major order from stream
    STREAM_A; the diagonal is exactly 1.
    """
    a = np.empty((n, n), dtype=np.float64)
    if n == 0:
        return a.astype(dtype)
    scale = w / (n - 1) if n > 1 else 0.0
    rows_per_chunk = max(1, (1 << 24) // max(n, 1))
    for r0 in range(0, n, rows_per_chunk):
        r1 = min(n, r0 + rows_per_chunk)
        u = uniform01(seed, STREAM_A, r0 * n, (r1 - r0) * n).reshape(r1 - r0, n)
        a[r0:r1] = (2.0 * u - 1.0) * scale
    np.fill_diagonal(a, 1.0)
    return a.astype(dtype, copy=False)


def planted_x(n: int, nrhs: int, seed: int) -> np.ndarray:
    """x_true ~ U[-1, 1], shape (n, nrhs), row-major."""
    return uniform(seed, STREAM_X, (n, nrhs), -1.0, 1.0)


def rhs_for(a: np.ndarray, x: np.ndarray) -> np.ndarray:
    """b = A @ x_true in FP64 (a plain library matvec; input preparation only)."""
    return np.ascontiguousarray(a.astype(np.float64) @ x)


def gaussian(seed: int, stream: int, shape) -> np.ndarray:
    """N(0, 1) by Box-Muller on pairs of counter-based uniforms."""
    count = int(np.prod(shape))
    u = uniform01(seed, stream, 0, 2 * count)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)).reshape(shape)


# ----------------------------------------------------------------------------
# Banded 5-point Laplacian (row-band storage)
# ----------------------------------------------------------------------------

def laplacian_band(g: int, diag: float = 4.1) -> tuple[np.ndarray, int, int]:
    """2D 5-point Laplacian on a g x g grid as a row band.

    Node (gy, gx) is row i = gy * g + gx.  Band storage: ``ab[i, j - i + kl]``
    holds a_ij for i - kl <= j <= i + ku, kl = ku = g; entries outside the matrix
    and the structural zeros inside the band are 0.
    Returns ``(ab, kl, ku)`` with ab of shape (n, kl + ku + 1).
    """
    n = g * g
    kl = ku = g
    ab = np.zeros((n, kl + ku + 1), dtype=np.float64)
    i = np.arange(n)
    gx = i % g
    gy = i // g
    ab[:, kl] = diag
    ab[gx > 0, kl - 1] = -1.0
    ab[gx < g - 1, kl + 1] = -1.0
    ab[gy > 0, kl - g] = -1.0
    ab[gy < g - 1, kl + g] = -1.0
    return ab, kl, ku


def laplacian_disc_band(r: int, diag: float = 4.1) -> tuple[np.ndarray, int, int]:
    """2D 5-point Laplacian on the grid points (x, y) with x^2 + y^2 <= r^2.

    Nodes are numbered row by row (y, then x); a node's neighbours are the grid
    points next to it that lie in the disc (Dirichlet boundary: the others are
    left out).  Diagonal 4.1, neighbours -1.  Returns ``(ab, kl, ku)``, the row
    band with kl = ku = the largest index distance between neighbours.
    """
    ys, xs = np.mgrid[-r:r + 1, -r:r + 1]
    inside = xs * xs + ys * ys <= r * r
    idx = np.full(inside.shape, -1, dtype=np.int64)
    n = int(inside.sum())
    idx[inside] = np.arange(n)
    east = inside[:, :-1] & inside[:, 1:]
    south = inside[:-1, :] & inside[1:, :]
    i = np.concatenate([idx[:, :-1][east], idx[:-1, :][south]])
    j = np.concatenate([idx[:, 1:][east], idx[1:, :][south]])
    d = int((j - i).max()) if i.size else 0
    ab = np.zeros((n, 2 * d + 1), dtype=np.float64)
    ab[:, d] = diag
    ab[i, d + (j - i)] = -1.0
    ab[j, d - (j - i)] = -1.0
    return ab, d, d


def band_to_dense(ab: np.ndarray, kl: int, ku: int) -> np.ndarray:
    n = ab.shape[0]
    a = np.zeros((n, n), dtype=ab.dtype)
    for d in range(-kl, ku + 1):
        i = np.arange(max(0, -d), min(n, n - d))
        a[i, i + d] = ab[i, d + kl]
    return a


def dense_to_band(a: np.ndarray, kl: int, ku: int) -> np.ndarray:
    n = a.shape[0]
    ab = np.zeros((n, kl + ku + 1), dtype=a.dtype)
    for d in range(-kl, ku + 1):
        i = np.arange(max(0, -d), min(n, n - d))
        ab[i, d + kl] = a[i, i + d]
    return ab


def band_rhs(ab: np.ndarray, kl: int, ku: int, x: np.ndarray) -> np.ndarray:
    """b = A @ x for a row band (input preparation only)."""
    n = ab.shape[0]
    b = np.zeros_like(x, dtype=np.float64)
    for d in range(-kl, ku + 1):
        col = ab[:, d + kl]
        if not np.any(col):
            continue
        i = np.arange(max(0, -d), min(n, n - d))
        b[i] += col[i, None] * x[i + d]
    return b


# ----------------------------------------------------------------------------
# The five workloads
# ----------------------------------------------------------------------------

def config0(n: int = 256, nrhs: int = 1):
    """Dense FP64 n=256, one RHS, off-diagonals U[-0.5, 0.5]/(n-1)."""
    s = seed_for(0)
    a = dense_dd(n, 0.5, s)
    x = planted_x(n, nrhs, s)
    return a, x, rhs_for(a, x)


def config1(g: int = 512, nrhs: int = 8):
    """Banded 5-point Laplacian on a g x g grid, nrhs planted right-hand sides."""
    s = seed_for(1)
    ab, kl, ku = laplacian_band(g)
    x = planted_x(g * g, nrhs, s)
    return ab, kl, ku, x, band_rhs(ab, kl, ku, x)


def config2(n: int = 16384, nrhs: int = 32):
    """Dense n=16384, 32 RHS, off-diagonals U[-0.9, 0.9]/(n-1)."""
    s = seed_for(2)
    a = dense_dd(n, 0.9, s)
    x = planted_x(n, nrhs, s)
    return a, x, rhs_for(a, x)


def config3_sizes(batch: int = 4096, nmin: int = 16, nmax: int = 512, rmin: int = 1, rmax: int = 4):
    """Per-system (n, nrhs) of the batched workload: n ~ U{nmin..nmax}, nrhs ~ U{rmin..rmax}."""
    s = seed_for(3)
    u = uniform01(s, STREAM_META, 0, 2 * batch)
    ns = nmin + np.floor(u[0::2] * (nmax - nmin + 1)).astype(np.int64)
    rs = rmin + np.floor(u[1::2] * (rmax - rmin + 1)).astype(np.int64)
    return ns, rs


def config3_system(i: int, n: int, nrhs: int):
    """System i of the batched workload (same distribution as the n=256 case)."""
    s = seed_for(3, 1 + i)
    a = dense_dd(n, 0.5, s)
    x = planted_x(n, nrhs, s)
    return a, x, rhs_for(a, x)


def config4_system(i: int, n: int = 1024, nrhs: int = 4):
    """System i of the differentiable batch: A, x_true, b and loss weights W ~ N(0,1)."""
    s = seed_for(4, 1 + i)
    a = dense_dd(n, 0.5, s)
    x = planted_x(n, nrhs, s)
    wts = gaussian(s, STREAM_W, (n, nrhs))
    return a, x, rhs_for(a, x), wts


def pick_indices(seed: int, count: int, bounds) -> np.ndarray:
    """``count`` seeded index tuples, entry k drawn uniformly from range(bounds[k])."""
    u = uniform01(seed, STREAM_PICK, 0, count * len(bounds)).reshape(count, len(bounds))
    return np.floor(u * np.asarray(bounds, dtype=np.float64)).astype(np.int64)
