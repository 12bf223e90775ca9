"""Plain FP64 CPU oracle for the EbV solver (arXiv 1907.05767).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this package; the library
``paper_1907_05767_gb300`` never imports it and shares no code with it.

The arithmetic lives in ``ebv_oracle.c`` (plain C, binary64, no FMA
contraction); this module only builds it with gcc and marshals numpy arrays.
Each function states the passage of the paper it follows:

* ``lu``           -- Doolittle factorisation without pivoting, Eq. 6a and 6c.
* ``forward`` / ``backward`` / ``solve`` -- LY = B then UX = Y, Eq. 1.
* ``band_lu`` / ``band_solve`` -- the same restricted to a band (the paper's
  sparse experiment, Table 1, read as banded storage).
* ``adjoint``      -- transposed solves for gradients (no counterpart in the
  paper; project addition).
* ``inverse``      -- the product-form inverse of Eq. 4c: A^{-1} = U^{-1} L^{-1}
  as the product of the elementary transformations of the elimination.
* ``residual``     -- B - A X by the compensated dot product Dot2.

Every function is pinned by ``tests/test_oracle_pins.py`` against hand-worked
cases, closed forms, brute force and library routines.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ebv_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

_lib = None


def build(force: bool = False, extra_flags: tuple = (), out: str | None = None) -> str:
    """Compile ebv_oracle.c with gcc into a shared library; returns its path."""
    out = out or _LIB_PATH
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]
    tmp = out + f".tmp{os.getpid()}"
    for omp in (["-fopenmp"], []):
        cmd = base + omp + list(extra_flags) + [_SRC, "-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, out)
            return out
    raise RuntimeError("oracle build failed:\n" + r.stderr)


def load(path: str | None = None):
    """Load (building if needed) the oracle library."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _bind(lib):
    i64, dp, vp = ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p
    lib.oracle_set_threads.argtypes = [ctypes.c_int]
    lib.oracle_set_threads.restype = ctypes.c_int
    lib.oracle_lu.argtypes = [i64, dp, i64, i64]
    lib.oracle_lu.restype = i64
    lib.oracle_forward.argtypes = [i64, dp, i64, dp, i64, i64]
    lib.oracle_backward.argtypes = [i64, dp, i64, dp, i64, i64]
    lib.oracle_band_lu.argtypes = [i64, i64, i64, dp, i64]
    lib.oracle_band_lu.restype = i64
    lib.oracle_band_solve.argtypes = [i64, i64, i64, dp, i64, dp, i64, i64]
    lib.oracle_adjoint.argtypes = [i64, i64, dp, i64, dp, dp, i64, dp, vp, i64]
    lib.oracle_residual.argtypes = [i64, dp, i64, dp, i64, dp, i64, i64, vp, i64, dp, i64]
    lib.oracle_band_residual.argtypes = [i64, i64, i64, dp, i64, dp, i64, dp, i64, i64, dp, i64]
    lib.oracle_inverse.argtypes = [i64, dp, i64, dp, i64]
    return lib


def _f64(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.float64)


def _p(x: np.ndarray):
    return x.ctypes.data_as(ctypes.c_void_p)


def set_threads(t: int) -> int:
    """Set the OpenMP thread count of the oracle (0 keeps it); returns the count in use."""
    return load().oracle_set_threads(int(t))


def lu(a, kstop: int = -1, lib=None):
    """Doolittle LU without pivoting (Eq. 6a, 6c).  Returns (packed L\\U, info)."""
    lib = lib or load()
    f = _f64(a).copy()
    n = f.shape[0]
    info = lib.oracle_lu(n, _p(f), n, int(kstop))
    return f, int(info)


def forward(lu_, b, lib=None):
    """LY = B with L unit lower (Eq. 1)."""
    lib = lib or load()
    lu_ = _f64(lu_)
    y = _f64(b).copy()
    y2 = y.reshape(y.shape[0], -1)
    lib.oracle_forward(lu_.shape[0], _p(lu_), lu_.shape[0], _p(y2), y2.shape[1], y2.shape[1])
    return y


def backward(lu_, y, lib=None):
    """UX = Y with U upper (Eq. 1)."""
    lib = lib or load()
    lu_ = _f64(lu_)
    x = _f64(y).copy()
    x2 = x.reshape(x.shape[0], -1)
    lib.oracle_backward(lu_.shape[0], _p(lu_), lu_.shape[0], _p(x2), x2.shape[1], x2.shape[1])
    return x


def solve(lu_, b, lib=None):
    """X from the packed factors: forward then backward substitution (Eq. 1)."""
    return backward(lu_, forward(lu_, b, lib=lib), lib=lib)


def band_lu(ab, kl: int, ku: int, lib=None):
    """Banded Doolittle LU on row-band storage; returns (band factors, info)."""
    lib = lib or load()
    f = _f64(ab).copy()
    info = lib.oracle_band_lu(f.shape[0], kl, ku, _p(f), f.shape[1])
    return f, int(info)


def band_solve(fab, kl: int, ku: int, b, lib=None):
    lib = lib or load()
    fab = _f64(fab)
    x = _f64(b).copy()
    x2 = x.reshape(x.shape[0], -1)
    lib.oracle_band_solve(fab.shape[0], kl, ku, _p(fab), fab.shape[1], _p(x2), x2.shape[1], x2.shape[1])
    return x


def adjoint(lu_, x, g, want_grad_a: bool = True, lib=None):
    """(grad_B, grad_A) for dL/dX = G: grad_B = A^{-T} G, grad_A = -grad_B X^T."""
    lib = lib or load()
    lu_ = _f64(lu_)
    n = lu_.shape[0]
    x2 = _f64(x).reshape(n, -1)
    g2 = _f64(g).reshape(n, -1)
    nrhs = x2.shape[1]
    gb = np.zeros_like(g2)
    ga = np.zeros((n, n)) if want_grad_a else None
    lib.oracle_adjoint(n, nrhs, _p(lu_), n, _p(x2), _p(g2), nrhs, _p(gb),
                       _p(ga) if ga is not None else None, n)
    return gb, ga


def residual(a, x, b, rows=None, lib=None):
    """R = B - A X by Dot2; ``rows`` restricts it to the listed rows."""
    lib = lib or load()
    a = _f64(a)
    n = a.shape[0]
    x2 = _f64(x).reshape(n, -1)
    b2 = _f64(b).reshape(n, -1)
    nrhs = x2.shape[1]
    if rows is None:
        r = np.zeros((n, nrhs))
        lib.oracle_residual(n, _p(a), a.shape[1], _p(x2), nrhs, _p(b2), nrhs, nrhs, None, 0, _p(r), nrhs)
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        r = np.zeros((rows.size, nrhs))
        lib.oracle_residual(n, _p(a), a.shape[1], _p(x2), nrhs, _p(b2), nrhs, nrhs, _p(rows), rows.size,
                            _p(r), nrhs)
    return r


def band_residual(ab, kl: int, ku: int, x, b, lib=None):
    lib = lib or load()
    ab = _f64(ab)
    n = ab.shape[0]
    x2 = _f64(x).reshape(n, -1)
    b2 = _f64(b).reshape(n, -1)
    nrhs = x2.shape[1]
    r = np.zeros((n, nrhs))
    lib.oracle_band_residual(n, kl, ku, _p(ab), ab.shape[1], _p(x2), nrhs, _p(b2), nrhs, nrhs, _p(r), nrhs)
    return r


def inverse(lu_, lib=None):
    """A^{-1} from the packed factors in the product form of Eq. 4c."""
    lib = lib or load()
    lu_ = _f64(lu_)
    n = lu_.shape[0]
    x = np.zeros((n, n))
    lib.oracle_inverse(n, _p(lu_), n, _p(x), n)
    return x


def unpack(lu_):
    """Split packed factors into (L with unit diagonal, U)."""
    lu_ = _f64(lu_)
    lower = np.tril(lu_, -1) + np.eye(lu_.shape[0])
    upper = np.triu(lu_)
    return lower, upper
