"""C ABI: the library loads without a GPU, exports every declared entry point,
and rejects invalid arguments on the host before touching the device."""
import ctypes
import glob
import os
import re

import pytest

import paper_1907_05767_gb300 as ebv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1907_05767_gb300 import _build
    _build.build()
    return ebv.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(ebv_\w+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "ebv_factor" in names and "ebv_solve" in names
    assert "ebv_factor_solve_batched" in names and "ebv_solve_adjoint" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) <= set(ebv.EXPORTED)


def test_version_and_status_strings(lib):
    assert lib.ebv_version() >= 100
    for s in range(9):
        assert lib.ebv_status_string(s)
    assert lib.ebv_status_string(99) == b"unknown status"


def _d(n, ld, kl=0, ku=0, storage=ebv.DENSE):
    return ebv.Desc(n, ld, kl, ku, storage, 0)


FAKE = ctypes.c_void_p(0x100000)  # never dereferenced: every call below fails its host checks


def test_factor_argument_errors(lib):
    info = FAKE
    cases = [
        (None, ebv.FP64),                                  # null descriptor
        (_d(-1, 4), ebv.FP64),                             # negative order
        (_d(8, 7), ebv.FP64),                              # ld < n
        (_d(8, 8), 9),                                     # unknown precision
        (_d(8, 8, 8, 1, ebv.BAND), ebv.FP64),              # kl >= n
        (_d(8, 3, 1, 2, ebv.BAND), ebv.FP64),              # ld < kl+ku+1
        (_d(8, 8, 0, 0, 7), ebv.FP64),                     # unknown storage
        (_d(8, 4, 1, 2, ebv.BAND_SYM), ebv.FP64),          # symmetric band with kl != ku
    ]
    for d, p in cases:
        st = lib.ebv_factor(ctypes.byref(d) if d is not None else None, p, FAKE, None, info, None, 0, None)
        assert st == ebv.ERR_ARG, (d and (d.n, d.ld, d.kl, d.ku, d.storage), p, st)
    d = _d(8, 8)
    assert lib.ebv_factor(ctypes.byref(d), ebv.FP64, FAKE, None, None, None, 0, None) == ebv.ERR_ARG  # null info
    assert lib.ebv_factor(ctypes.byref(d), ebv.FP64, None, None, info, None, 0, None) == ebv.ERR_ARG  # null a
    # mixed precision needs the FP32 output buffer and the workspace
    assert lib.ebv_factor(ctypes.byref(d), ebv.MIXED_BF16, FAKE, None, info, None, 0, None) == ebv.ERR_ARG
    assert lib.ebv_factor(ctypes.byref(d), ebv.MIXED_BF16, FAKE, FAKE, info, None, 0, None) == ebv.ERR_WORKSPACE
    # band storage in mixed precision: FP32 factors into lowp (same band layout), workspace required
    db = _d(8, 3, 1, 1, ebv.BAND)
    assert lib.ebv_factor(ctypes.byref(db), ebv.MIXED_FP16, FAKE, None, info, None, 0, None) == ebv.ERR_ARG
    assert lib.ebv_factor(ctypes.byref(db), ebv.MIXED_FP16, FAKE, FAKE, info, None, 0, None) == ebv.ERR_WORKSPACE


def test_solve_argument_errors(lib):
    d = _d(8, 8)
    ws = ctypes.c_void_p(0x200000)
    ok_ref = ebv.Refine(1e-12, 5, 0)
    bad_ref = ebv.Refine(-1.0, 5, 0)
    call = lambda **k: lib.ebv_solve(ctypes.byref(k.get("d", d)), k.get("p", ebv.FP64), k.get("lu", FAKE),
                                     k.get("a", None), k.get("b", FAKE), k.get("nrhs", 2), k.get("ldb", 2),
                                     k.get("ref", None), None, k.get("ws", ws), k.get("wsb", 1 << 30), None)
    assert call(nrhs=-1) == ebv.ERR_ARG
    assert call(ldb=1) == ebv.ERR_ARG
    assert call(lu=None) == ebv.ERR_ARG
    assert call(b=None) == ebv.ERR_ARG
    assert call(ref=ctypes.byref(bad_ref), a=FAKE) == ebv.ERR_ARG
    assert call(ref=ctypes.byref(ok_ref)) == ebv.ERR_ARG          # refinement needs the original A
    assert call(p=ebv.MIXED_BF16, ref=ctypes.byref(ok_ref)) == ebv.ERR_ARG
    assert call(p=ebv.FP32, ref=ctypes.byref(ok_ref), a=FAKE) == ebv.ERR_UNSUPPORTED
    assert call(ws=None) == ebv.ERR_WORKSPACE
    assert call(ws=ctypes.c_void_p(0x200010)) == ebv.ERR_WORKSPACE  # misaligned workspace


def test_workspace_sizes(lib):
    sz = lambda n, p, r: ebv.ebv_workspace_size(n, p, r)
    assert sz(1024, ebv.MIXED_BF16, 0) >= 2 * 2 * 1024 * 1024  # two 16-bit shadows of the factors
    assert sz(1024, ebv.FP64, 32) >= 1024 * 32 * 8 * 2
    assert sz(1024, ebv.FP64, 32) > sz(1024, ebv.FP64, 1)
    d = _d(-3, 1)
    assert lib.ebv_workspace_size(ctypes.byref(d), ebv.FP64, 0) == 0


def test_band_storage_descriptors(lib):
    # general band: ld >= kl + ku + 1; both symmetric storages need kl == ku;
    # the lower half only needs ld >= kl + 1
    def ok(n, ld, kl, ku, storage):
        d = ebv._desc(n, ld, kl, ku, storage)
        return lib.ebv_workspace_size(ctypes.byref(d), ebv.FP64, 1) > 0
    assert ok(100, 9, 3, 5, ebv.BAND) and not ok(100, 8, 3, 5, ebv.BAND)
    assert ok(100, 9, 4, 4, ebv.BAND_SYM) and not ok(100, 9, 3, 5, ebv.BAND_SYM)
    assert ok(100, 5, 4, 4, ebv.BAND_SYM_LOWER) and not ok(100, 4, 4, 4, ebv.BAND_SYM_LOWER)
    assert not ok(100, 9, 3, 5, ebv.BAND_SYM_LOWER)
    assert not ok(100, 9, 100, 100, ebv.BAND_SYM_LOWER)  # kl < n
    assert not ok(100, 100, 0, 0, 6)  # no such storage
    # dense symmetric (lower triangle): ld >= n, kl / ku ignored
    assert ok(100, 100, 0, 0, ebv.DENSE_SYM) and ok(100, 128, 7, 3, ebv.DENSE_SYM)
    assert not ok(100, 99, 0, 0, ebv.DENSE_SYM)


def test_dense_sym_rejects_mixed_and_inverse(lib):
    d = ebv._desc(64, 64, 0, 0, ebv.DENSE_SYM)
    info = ctypes.c_void_p(0x100000)
    a = ctypes.c_void_p(0x200000)
    ws = ctypes.c_void_p(0x300000)
    assert lib.ebv_factor(ctypes.byref(d), ebv.MIXED_BF16, a, a, info, ws, 1 << 20, None) == ebv.ERR_UNSUPPORTED
    assert lib.ebv_inverse(ctypes.byref(d), ebv.FP64, a, ws, 64, ws, 1 << 20, None) == ebv.ERR_UNSUPPORTED


def test_inverse_argument_errors(lib):
    n = 100
    need = lib.ebv_inverse_workspace_size(n, ebv.FP64)
    assert need >= n * n * 8 and need % 256 == 0
    assert lib.ebv_inverse_workspace_size(n, ebv.FP32) >= n * n * 4
    assert lib.ebv_inverse_workspace_size(n, ebv.MIXED_BF16) == 0
    assert lib.ebv_inverse_workspace_size(-1, ebv.FP64) == 0
    lu, x, ws = ctypes.c_void_p(0x100000), ctypes.c_void_p(0x10000000), ctypes.c_void_p(0x40000000)
    d = _d(n, n)
    call = lambda desc, prec, l, xx, ldx, w, wb: lib.ebv_inverse(  # noqa: E731
        ctypes.byref(desc) if desc is not None else None, prec, l, xx, ldx, w, wb, None)
    assert call(None, ebv.FP64, lu, x, n, ws, need) == 1                      # null descriptor
    assert call(_d(n, n, 2, 2, ebv.BAND), ebv.FP64, lu, x, n, ws, need) == 7  # band storage
    assert call(d, ebv.MIXED_BF16, lu, x, n, ws, need) == 7                   # mixed: pass the FP32 factors
    assert call(d, ebv.FP64, lu, x, n - 1, ws, need) == 1                     # ldx < n
    assert call(d, ebv.FP64, None, x, n, ws, need) == 1                       # null factors
    assert call(d, ebv.FP64, lu, ctypes.c_void_p(0x100004), n, ws, need) == 1  # misaligned x
    assert call(d, ebv.FP64, lu, ctypes.c_void_p(0x100000 + 8 * n * 50), n, ws, need) == 1  # x overlaps lu
    assert call(d, ebv.FP64, lu, x, n, None, need) == 8                       # no workspace
    assert call(d, ebv.FP64, lu, x, n, ws, need - 256) == 8                   # workspace too small
    assert call(d, ebv.FP64, lu, x, n, ctypes.c_void_p(0x40000010), need) == 8  # misaligned workspace
    assert call(_d(0, 1), ebv.FP64, None, None, 1, None, 0) == 0              # n = 0: nothing to do
