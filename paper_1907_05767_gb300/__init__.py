"""EbV linear solver for GB300 (sm_103a): Python binding of libebv.so.

The binding only marshals arguments: every step of the factorisation and the
solves runs in the library's CUDA kernels.  PyTorch supplies device memory and
the current CUDA stream.  If libebv.so has not been built the import succeeds
but every call raises ``EbvUnavailable``; there is no CPU fallback.

Method: Hashemi, Lahooti, Shirani, "Equal bi-Vectorized (EbV) method to high
performance on GPU" (arXiv 1907.05767).  AX = B is solved as L(UX) = B (Eq. 1)
after a Doolittle factorisation without pivoting of a diagonally dominant A
(Eq. 2, Eq. 6a-c), with long and short vectors paired for equal work (Eq. 7).

Names follow the C ABI in include/ebv.h: ``ebv_factor``, ``ebv_solve``,
``ebv_gesv_host``, ``ebv_solve_static``, ``ebv_inverse``, ``ebv_solve_adjoint``
take torch tensors.  Convenience wrappers: ``factor``, ``band_factor`` (both
return ``Factors``), ``solve`` (dense or band factors), ``inverse`` (dense),
``Batch`` / ``uniform_batch`` (``ebv_factor_solve_batched``), and the autograd
function ``EbvSolve``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libebv.so")

# ebv_status_t
OK, ERR_ARG, ERR_ZERO_PIVOT, ERR_NONFINITE, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_CUDA, ERR_UNSUPPORTED, \
    ERR_WORKSPACE = range(9)
# ebv_prec_t
FP64, FP32, MIXED_BF16, MIXED_FP16 = range(4)
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16": MIXED_BF16, "fp16": MIXED_FP16}
DENSE, BAND, BAND_SYM, BAND_SYM_LOWER, PROFILE, DENSE_SYM = 0, 1, 2, 3, 4, 5


class EbvError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


class EbvUnavailable(RuntimeError):
    pass


class Desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("ld", ctypes.c_int64), ("kl", ctypes.c_int64), ("ku", ctypes.c_int64),
                ("storage", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Refine(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class RefineReport(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("resid_first", ctypes.c_double),
                ("resid_final", ctypes.c_double)]


_lib = None

# (name, restype, argtypes)
_VP, _I64, _I32, _SZ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t
_SIGNATURES = [
    ("ebv_version", _I32, []),
    ("ebv_status_string", ctypes.c_char_p, [_I32]),
    ("ebv_workspace_size", _SZ, [ctypes.POINTER(Desc), _I32, _I64]),
    ("ebv_factor", _I32, [ctypes.POINTER(Desc), _I32, _VP, _VP, _VP, _VP, _SZ, _VP]),
    ("ebv_solve", _I32, [ctypes.POINTER(Desc), _I32, _VP, _VP, _VP, _I64, _I64, ctypes.POINTER(Refine), _VP, _VP,
                         _SZ, _VP]),
    ("ebv_gesv_host_workspace_size", _SZ, [ctypes.POINTER(Desc), _I32, _I64]),
    ("ebv_gesv_host", _I32, [ctypes.POINTER(Desc), _I32, _VP, _VP, _VP, _I64, _I64, ctypes.POINTER(Refine), _VP,
                             _VP, _VP, _SZ, _VP]),
    ("ebv_solve_static", _I32, [ctypes.POINTER(Desc), _I32, _VP, _VP, _VP, _I64, _I64, ctypes.POINTER(Refine), _VP,
                                _VP]),
    ("ebv_batch_schedule_len", _I64, [_I64]),
    ("ebv_batch_workspace_size", _SZ, [_I64]),
    ("ebv_batch_schedule", _I32, [_I64, _VP, _VP, _VP, _VP]),
    ("ebv_batch_partition", _I32, [_I64, _VP, _VP, _I32, _VP, _VP]),
    ("ebv_profile_from_band", _I32, [_I64, _I64, _I64, _VP, _I64, _I32, _VP, _SZ, _VP, _VP, _VP]),
    ("ebv_factor_solve_batched", _I32, [_I64, _VP, _VP, _VP, _VP, _I32, _VP, _VP, _VP, _SZ, _VP]),
    ("ebv_batch_autotune_scratch", _SZ, [_I32, _I32, _I32]),
    ("ebv_batch_autotune", _I32, [_VP, _I32, _I32, _I32, _VP, _SZ, _VP, _VP, _VP]),
    ("ebv_inverse_workspace_size", _SZ, [_I64, _I32]),
    ("ebv_inverse", _I32, [ctypes.POINTER(Desc), _I32, _VP, _VP, _I64, _VP, _SZ, _VP]),
    ("ebv_solve_adjoint", _I32, [_I64, _I64, _I64, _VP, _I64, _I64, _VP, _VP, _VP, _VP, _VP]),
    ("ebv_debug_set_lowp_gemm", None, [_I32]),
    ("ebv_debug_set_band_envelope", None, [_I32]),
    ("ebv_debug_set_cluster_panel", None, [_I32]),
    ("ebv_debug_set_band_cluster", None, [_I32]),
    ("ebv_debug_set_band_lookahead", None, [_I32]),
    ("ebv_debug_set_diag_lu", None, [_I32]),
    ("ebv_debug_set_small_dense", None, [_I32]),
    ("ebv_debug_residual", _I32, [_I64, _VP, _I64, _VP, _VP, _I64, _VP, _VP, _SZ, _VP]),
    ("ebv_debug_lowp_update", _I32, [_I32, _I32, _VP, _I64, _VP, _VP, _I64, _VP, _I64, _I64, _I64, _I64, _I64, _I64,
                                     _VP, _VP]),
    ("ebv_debug_tc_available", _I32, []),
    ("ebv_debug_wait_probe", _I32, [_I64, _VP, _VP]),
    ("ebv_debug_launch_count", _I64, []),
    ("ebv_debug_profile", None, [_I32]),
    ("ebv_debug_profile_read", _I32, [_VP, _VP, _VP]),
]
PROFILE_CLASSES = ["lowp_gemm", "simt_gemm", "panel", "trsv", "residual", "batched", "adjoint", "other", "trsm",
                   "l21", "leaf_update", "inverse"]


def launch_count() -> int:
    return int(lib().ebv_debug_launch_count())


def profile(enable: bool):
    lib().ebv_debug_profile(1 if enable else 0)


def profile_read() -> dict:
    """{class: (ms, work, launches)} for launches recorded since the last read."""
    import numpy as np
    ms = np.zeros(len(PROFILE_CLASSES))
    work = np.zeros(len(PROFILE_CLASSES))
    cnt = np.zeros(len(PROFILE_CLASSES), dtype=np.int64)
    _check(lib().ebv_debug_profile_read(ms.ctypes.data, work.ctypes.data, cnt.ctypes.data), "profile_read")
    return {c: (float(ms[i]), float(work[i]), int(cnt[i])) for i, c in enumerate(PROFILE_CLASSES)}
EXPORTED = [s[0] for s in _SIGNATURES]


def lib():
    """The loaded libebv.so (raises EbvUnavailable when it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise EbvUnavailable(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
        handle = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES:
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def build(**kw) -> str:
    from ._build import build as _b
    return _b(**kw)


def status_string(status: int) -> str:
    try:
        return lib().ebv_status_string(status).decode()
    except EbvUnavailable:
        return "unknown"


def _check(status: int, where: str):
    if status != OK:
        raise EbvError(status, where)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(device=None):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _desc(n, ld, kl=0, ku=0, storage=DENSE):
    return Desc(int(n), int(ld), int(kl), int(ku), int(storage), 0)


def _prec(p) -> int:
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def _need_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("tensors must live on a CUDA device")


# ----------------------------------------------------------------------------
# C-ABI names, torch arguments
# ----------------------------------------------------------------------------

def ebv_workspace_size(n, prec, nrhs=0, ld=None, kl=0, ku=0, storage=DENSE) -> int:
    d = _desc(n, ld if ld is not None else (max(1, n) if storage in (DENSE, DENSE_SYM) else kl + ku + 1), kl, ku,
              storage)
    return int(lib().ebv_workspace_size(ctypes.byref(d), _prec(prec), int(nrhs)))


def workspace(n, prec, nrhs=0, device="cuda", **kw) -> torch.Tensor:
    """A device workspace tensor large enough for factor and solve."""
    nbytes = max(256, ebv_workspace_size(n, prec, nrhs, **kw))
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def ebv_factor(a: torch.Tensor, prec="fp64", lowp: torch.Tensor | None = None, info: torch.Tensor | None = None,
               ws: torch.Tensor | None = None, kl=0, ku=0, storage=DENSE, n: int | None = None) -> torch.Tensor:
    """Factor in place (FP64/FP32) or into ``lowp`` (mixed).  Returns ``info``.
    Profile storage: ``a`` is the byte buffer and ``n`` the order."""
    p = _prec(prec)
    _need_cuda(a, lowp, info, ws)
    if storage == PROFILE and n is None:
        raise ValueError("profile storage: pass the order n")
    n = a.shape[0] if n is None else int(n)
    ld = a.stride(0) if storage != PROFILE else 0
    if info is None:
        info = torch.zeros(1, dtype=torch.int32, device=a.device)
    if ws is None:
        ws = workspace(n, p, 0, a.device, ld=ld, kl=kl, ku=ku, storage=storage)
    d = _desc(n, ld, kl, ku, storage)
    _check(lib().ebv_factor(ctypes.byref(d), p, _ptr(a), _ptr(lowp), _ptr(info), _ptr(ws), ws.numel(),
                            _stream(a.device)), "ebv_factor")
    return info


def ebv_solve(lu: torch.Tensor, b: torch.Tensor, prec="fp64", a_orig: torch.Tensor | None = None,
              refine: tuple | None = None, report: torch.Tensor | None = None, ws: torch.Tensor | None = None,
              kl=0, ku=0, storage=DENSE, ld=None) -> torch.Tensor:
    """Overwrite ``b`` (n x nrhs) with X.  ``refine`` = (tol, max_iter) or None."""
    p = _prec(prec)
    _need_cuda(lu, b, a_orig, report, ws)
    n = b.shape[0]
    b2 = b if b.dim() == 2 else b.view(n, 1)
    nrhs = b2.shape[1]
    if ld is None:
        ld = lu.stride(0) if storage != PROFILE else 0
    if ws is None:
        ws = workspace(n, p, nrhs, b.device, ld=ld, kl=kl, ku=ku, storage=storage)
    d = _desc(n, ld, kl, ku, storage)
    ref = Refine(float(refine[0]), int(refine[1]), 0) if refine is not None else None
    if refine is not None and report is None:
        report = torch.zeros(3, dtype=torch.float64, device=b.device)
    _check(lib().ebv_solve(ctypes.byref(d), p, _ptr(lu), _ptr(a_orig), _ptr(b2), nrhs, b2.stride(0),
                           ctypes.byref(ref) if ref is not None else None, _ptr(report), _ptr(ws), ws.numel(),
                           _stream(b.device)), "ebv_solve")
    return b


def ebv_inverse(lu: torch.Tensor, x: torch.Tensor | None = None, prec="fp64", ws: torch.Tensor | None = None,
                ld=None) -> torch.Tensor:
    """A^{-1} (n x n) from packed dense factors, product form of Eq. 4c.
    ``prec``: fp64 or fp32 (the binary32 factors of a mixed factorisation too)."""
    p = _prec(prec)
    _need_cuda(lu, x, ws)
    n = lu.shape[0]
    if ld is None:
        ld = lu.stride(0)
    if x is None:
        x = torch.empty((n, n), dtype=lu.dtype, device=lu.device)
    if ws is None:
        nbytes = int(lib().ebv_inverse_workspace_size(n, p))
        ws = torch.empty(max(256, nbytes), dtype=torch.uint8, device=lu.device)
    d = _desc(n, ld)
    _check(lib().ebv_inverse(ctypes.byref(d), p, _ptr(lu), _ptr(x), x.stride(0), _ptr(ws), ws.numel(),
                             _stream(lu.device)), "ebv_inverse")
    return x


def gesv_host_workspace(n, nrhs, prec="bf16", device="cuda") -> torch.Tensor:
    d = _desc(n, n)
    size = lib().ebv_gesv_host_workspace_size(ctypes.byref(d), _prec(prec), nrhs)
    if size == 0:
        raise ValueError("ebv_gesv_host supports dense mixed precisions only")
    return torch.empty(size, dtype=torch.uint8, device=device)


def ebv_gesv_host(a_host: torch.Tensor, b_host: torch.Tensor, x_host: torch.Tensor | None = None, prec="bf16",
                  refine: tuple | None = (1e-12, 10), report_host: torch.Tensor | None = None,
                  info_host: torch.Tensor | None = None, ws: torch.Tensor | None = None, device="cuda") -> torch.Tensor:
    """Solve A X = B with A, B in (page-locked) host memory; X lands in
    ``x_host`` (default: ``b_host``) once the current stream of ``device``
    completes.  The copy of A overlaps the factorisation.  ``report_host``
    (uint8, >= 24 bytes) and ``info_host`` (int32) are optional host outputs."""
    if x_host is None:
        x_host = b_host
    for t in (a_host, b_host, x_host):
        if t.is_cuda or t.dtype != torch.float64:
            raise ValueError("float64 host tensors expected")
    n = a_host.shape[0]
    b2 = b_host if b_host.dim() == 2 else b_host.view(n, 1)
    x2 = x_host if x_host.dim() == 2 else x_host.view(n, 1)
    nrhs = b2.shape[1]
    if x2.shape != b2.shape or x2.stride(0) != b2.stride(0):
        raise ValueError("x_host must have the shape and row stride of b_host")
    if ws is None:
        ws = gesv_host_workspace(n, nrhs, prec, device)
    d = _desc(n, a_host.stride(0))
    ref = Refine(float(refine[0]), int(refine[1]), 0) if refine is not None else None
    _check(lib().ebv_gesv_host(ctypes.byref(d), _prec(prec), ctypes.c_void_p(a_host.data_ptr()),
                               ctypes.c_void_p(b2.data_ptr()), ctypes.c_void_p(x2.data_ptr()), nrhs, b2.stride(0),
                               ctypes.byref(ref) if ref is not None else None,
                               ctypes.c_void_p(report_host.data_ptr()) if report_host is not None else None,
                               ctypes.c_void_p(info_host.data_ptr()) if info_host is not None else None,
                               _ptr(ws), ws.numel(), _stream(torch.device(device))), "ebv_gesv_host")
    return x_host


# Limits of ebv_solve_static (its workspace is a fixed device array).
STATIC_SCRATCH_BYTES = 20 << 20
STATIC_MAX_N = 4096
STATIC_MAX_NRHS = 32


def ebv_solve_static(lu: torch.Tensor, b: torch.Tensor, prec="fp64", a_orig: torch.Tensor | None = None,
                     refine: tuple | None = None, report: torch.Tensor | None = None, kl=0, ku=0, storage=DENSE,
                     ld=None) -> torch.Tensor:
    """``ebv_solve`` for callers that cannot allocate device memory: the
    workspace is the library's fixed device array (n <= STATIC_MAX_N,
    nrhs <= STATIC_MAX_NRHS).  Overwrites ``b`` with X.  ``report`` must be
    passed in (already allocated) when ``refine`` is given."""
    p = _prec(prec)
    _need_cuda(lu, b, a_orig, report)
    n = b.shape[0]
    b2 = b if b.dim() == 2 else b.view(n, 1)
    nrhs = b2.shape[1]
    if ld is None:
        ld = lu.stride(0)
    d = _desc(n, ld, kl, ku, storage)
    ref = Refine(float(refine[0]), int(refine[1]), 0) if refine is not None else None
    _check(lib().ebv_solve_static(ctypes.byref(d), p, _ptr(lu), _ptr(a_orig), _ptr(b2), nrhs, b2.stride(0),
                                  ctypes.byref(ref) if ref is not None else None, _ptr(report),
                                  _stream(b.device)), "ebv_solve_static")
    return b


def read_report(report: torch.Tensor) -> dict:
    raw = report.detach().cpu().numpy().tobytes()[:ctypes.sizeof(RefineReport)]
    r = RefineReport.from_buffer_copy(raw)
    return {"iters": r.iters, "status": r.status, "resid_first": r.resid_first, "resid_final": r.resid_final}


def read_device_status(ws: torch.Tensor) -> tuple[int, int]:
    """(code, where) of the device status block at the start of a workspace."""
    v = ws[:8].cpu().view(torch.int32)
    return int(v[0]), int(v[1])


# ----------------------------------------------------------------------------
# Convenience API
# ----------------------------------------------------------------------------

@dataclass
class Factors:
    lu: torch.Tensor          # packed L\U (FP64 / FP32)
    info: torch.Tensor        # device int32
    prec: int
    a: torch.Tensor | None    # original FP64 A (mixed precisions, refinement)
    kl: int = 0
    ku: int = 0
    storage: int = DENSE


def factor(a: torch.Tensor, prec="fp64", keep_a: bool = True, sym: bool = False) -> Factors:
    """Factor a dense matrix.  FP64/FP32: a copy of ``a`` is factored.  Mixed:
    ``a`` (FP64) is kept and the FP32 factors go to a new tensor.  sym=True
    (FP64/FP32): A symmetric, only its lower triangle read; the factors keep
    L below the diagonal and the pivots on it (EBV_DENSE_SYM)."""
    p = _prec(prec)
    n = a.shape[0]
    if sym:
        dt = torch.float64 if p == FP64 else torch.float32
        lu = a.to(dt).clone().contiguous()
        info = ebv_factor(lu, p, storage=DENSE_SYM)
        return Factors(lu, info, p, a.to(torch.float64).contiguous() if keep_a else None, storage=DENSE_SYM)
    if p in (MIXED_BF16, MIXED_FP16):
        a64 = a.to(torch.float64).contiguous()
        lowp = torch.empty((n, n), dtype=torch.float32, device=a.device)
        info = ebv_factor(a64, p, lowp=lowp)
        return Factors(lowp, info, p, a64)
    dt = torch.float64 if p == FP64 else torch.float32
    lu = a.to(dt).clone().contiguous()
    info = ebv_factor(lu, p)
    return Factors(lu, info, p, a.to(torch.float64).contiguous() if keep_a else None)


def solve(f: Factors, b: torch.Tensor, refine: tuple | None = None, report: torch.Tensor | None = None):
    dt = torch.float32 if f.prec == FP32 else torch.float64
    x = b.to(dt).clone().contiguous()
    if x.dim() == 1:
        x = x.view(-1, 1)
    ebv_solve(f.lu, x, f.prec, a_orig=f.a, refine=refine, report=report, kl=f.kl, ku=f.ku, storage=f.storage)
    return x.view(b.shape) if b.dim() == 1 else x


def inverse(f: Factors) -> torch.Tensor:
    """Explicit A^{-1} from dense factors (FP64 factors: FP64; FP32 or mixed: FP32)."""
    if f.storage != DENSE:
        raise ValueError("the explicit inverse takes dense factors")
    return ebv_inverse(f.lu, prec=FP64 if f.prec == FP64 else FP32)


def band_factor(ab: torch.Tensor, kl: int, ku: int, prec="fp64", sym=False) -> Factors:
    """Factor a row-band matrix.  sym=False: A general, ab is n x (kl+ku+1).
    sym=True: A symmetric (kl == ku, both halves stored); U is formed from L
    and the pivots (EBV_BAND_SYM).  sym="lower": A symmetric with only the
    lower half stored, ab n x (kl+1) (EBV_BAND_SYM_LOWER); the factors keep
    that storage (L below the diagonal, the pivots on it).  Mixed precisions:
    FP32 factors of the FP64 band in a new tensor, for refined solves to FP64
    accuracy."""
    p = _prec(prec)
    lower = isinstance(sym, str) and sym == "lower"
    storage = BAND_SYM_LOWER if lower else (BAND_SYM if sym else BAND)
    solve_storage = BAND_SYM_LOWER if lower else BAND
    if p in (MIXED_BF16, MIXED_FP16):
        a64 = ab.to(torch.float64).contiguous()
        lowp = torch.empty(a64.shape, dtype=torch.float32, device=a64.device)
        info = ebv_factor(a64, p, lowp=lowp, kl=kl, ku=ku, storage=storage)
        return Factors(lowp, info, p, a64, kl, ku, solve_storage)
    dt = torch.float64 if p == FP64 else torch.float32
    lu = ab.to(dt).clone().contiguous()
    info = ebv_factor(lu, p, kl=kl, ku=ku, storage=storage)
    return Factors(lu, info, p, ab.to(torch.float64).contiguous(), kl, ku, solve_storage)


def ebv_profile_from_band(ab, kl: int, ku: int, prec="fp64"):
    """Profile (skyline) storage of a row-band matrix (host numpy array,
    n x (kl+ku+1)): returns (uint8 numpy buffer to copy to the device as is,
    kl, ku bounds of the profile for the descriptor)."""
    import numpy as np
    ab = np.ascontiguousarray(ab, dtype=np.float64)
    n = ab.shape[0]
    p = _prec(prec)
    need, klo, kuo = ctypes.c_size_t(0), ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib().ebv_profile_from_band(n, kl, ku, ab.ctypes.data, ab.shape[1], p, None, 0, ctypes.byref(need),
                                       ctypes.byref(klo), ctypes.byref(kuo)), "ebv_profile_from_band")
    buf = np.zeros(need.value + 256, dtype=np.uint8)
    off = (-buf.ctypes.data) % 256  # 256-byte aligned start
    out = buf[off:off + need.value]
    _check(lib().ebv_profile_from_band(n, kl, ku, ab.ctypes.data, ab.shape[1], p, out.ctypes.data, out.nbytes, None,
                                       None, None), "ebv_profile_from_band")
    return out, int(klo.value), int(kuo.value)


def profile_factor(ab, kl: int, ku: int, prec="fp64", device="cuda") -> Factors:
    """Factor a row-band matrix (host numpy) held in profile storage on the
    device; the factors stay in that storage (Factors.lu is the buffer)."""
    p = _prec(prec)
    buf, klp, kup = ebv_profile_from_band(ab, kl, ku, p)
    dev = torch.from_numpy(buf).to(device)
    orig = dev.clone() if p == FP64 else None  # the A of FP64 refinement
    info = ebv_factor(dev, p, kl=klp, ku=kup, storage=PROFILE, n=ab.shape[0])
    return Factors(dev, info, p, orig, klp, kup, PROFILE)


def profile_to_band(buf, n: int, kl: int, ku: int, prec="fp64"):
    """Row band (n x (kl+ku+1), float64 numpy) of a profile buffer (host
    numpy uint8), entries outside the profile 0 -- for checks."""
    import numpy as np
    buf = np.asarray(buf)
    nb = (n + 63) // 64
    lo = buf[0:4 * nb].view(np.int32)
    up = buf[4 * nb:8 * nb].view(np.int32)
    offl = buf[8 * nb:16 * nb].view(np.int64)
    offu = buf[16 * nb:24 * nb].view(np.int64)
    h = (24 * nb + 255) // 256 * 256
    vals = buf[h:].view(np.float64 if _prec(prec) == FP64 else np.float32).astype(np.float64)
    ab = np.zeros((n, kl + ku + 1))
    for b in range(nb):
        w = (b + 1) * 64 - lo[b]
        blk = vals[offl[b]:offl[b] + 64 * w].reshape(64, w)
        for r in range(min(64, n - 64 * b)):
            i = 64 * b + r
            for j in range(lo[b], min(n, 64 * (b + 1))):
                if -kl <= j - i <= ku:
                    ab[i, j - i + kl] = blk[r, j - lo[b]]
    for c in range(nb):
        hgt = 64 * c - up[c]
        blk = vals[offu[c]:offu[c] + 64 * hgt].reshape(hgt, 64)
        for i in range(up[c], 64 * c):
            for j in range(64 * c, min(n, 64 * (c + 1))):
                if j - i <= ku:
                    ab[i, j - i + kl] = blk[i - up[c], j - 64 * c]
    return ab


def debug_residual(a: torch.Tensor, x: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """R = B - A X through the refinement's residual kernel (testing hook)."""
    n = a.shape[0]
    x2 = x.reshape(n, -1).contiguous()
    b2 = b.reshape(n, -1).contiguous()
    nrhs = x2.shape[1]
    r = torch.empty_like(x2)
    ws = workspace(n, FP64, nrhs, a.device)
    _check(lib().ebv_debug_residual(n, _ptr(a), a.stride(0), _ptr(x2), _ptr(b2), nrhs, _ptr(r), _ptr(ws), ws.numel(),
                                    _stream(a.device)), "ebv_debug_residual")
    return r


# Batched kernel variants: block width NB x trailing-update tile edge TM.
BATCH_VARIANTS = {0: "nb16_tm64", 1: "nb32_tm64", 2: "nb64_tm64", 3: "nb16_tm32", 4: "nb32_tm32",
                  5: "nb64_tm32"}
MAX_BATCH_ORDER = 4096


def ebv_batch_schedule(n_list, nrhs_list, variant_of_n=None):
    """Host schedule (int32 numpy array) for ebv_factor_solve_batched."""
    import numpy as np
    n_arr = np.ascontiguousarray(n_list, dtype=np.int32)
    r_arr = np.ascontiguousarray(nrhs_list, dtype=np.int32)
    batch = n_arr.size
    sched = np.zeros(int(lib().ebv_batch_schedule_len(batch)), dtype=np.int32)
    vmap = None
    if variant_of_n is not None:
        vmap = np.ascontiguousarray(variant_of_n, dtype=np.int8)
        assert vmap.size >= MAX_BATCH_ORDER
    _check(lib().ebv_batch_schedule(batch, n_arr.ctypes.data, r_arr.ctypes.data,
                                    vmap.ctypes.data if vmap is not None else None, sched.ctypes.data),
           "ebv_batch_schedule")
    return sched


def ebv_batch_partition(n_list, nrhs_list, nranks):
    """Split a batch across ``nranks`` GPUs (host): returns (rank of each
    system as an int32 numpy array, summed cost of each rank in flops)."""
    import numpy as np
    n_arr = np.ascontiguousarray(n_list, dtype=np.int32)
    r_arr = np.ascontiguousarray(nrhs_list, dtype=np.int32)
    rank_of = np.zeros(n_arr.size, dtype=np.int32)
    cost = np.zeros(int(nranks), dtype=np.float64)
    _check(lib().ebv_batch_partition(n_arr.size, n_arr.ctypes.data, r_arr.ctypes.data, int(nranks),
                                     rank_of.ctypes.data, cost.ctypes.data), "ebv_batch_partition")
    return rank_of, cost


class Batch:
    """Many independent dense systems in one device buffer each for A and B.

    System s: A_s (n_s x n_s, row-major) at a_buf[a_off[s]:], B_s (n_s x
    nrhs_s) at b_buf[b_off[s]:].  ``run()`` factors every A_s in place and
    overwrites every B_s with X_s in one persistent launch.
    """

    def __init__(self, n_list, nrhs_list, prec="fp64", device="cuda", variant_of_n=None):
        import numpy as np
        self.prec = _prec(prec)
        if self.prec not in (FP64, FP32):
            raise ValueError("batched path supports fp64 and fp32")
        self.dtype = torch.float64 if self.prec == FP64 else torch.float32
        self.n = np.asarray(n_list, dtype=np.int64)
        self.nrhs = np.asarray(nrhs_list, dtype=np.int64)
        self.batch = int(self.n.size)
        esz = 8 if self.prec == FP64 else 4
        align = 16 // esz  # every system starts on a 16-byte boundary
        a_sz = ((self.n * self.n + align - 1) // align) * align
        b_sz = ((self.n * self.nrhs + align - 1) // align) * align
        self.a_off = np.concatenate([[0], np.cumsum(a_sz)[:-1]]).astype(np.int64)
        self.b_off = np.concatenate([[0], np.cumsum(b_sz)[:-1]]).astype(np.int64)
        self.a_buf = torch.zeros(int(a_sz.sum()), dtype=self.dtype, device=device)
        self.b_buf = torch.zeros(max(1, int(b_sz.sum())), dtype=self.dtype, device=device)
        a_ptrs = self.a_buf.data_ptr() + self.a_off * esz
        b_ptrs = self.b_buf.data_ptr() + self.b_off * esz
        self.ptrs = torch.from_numpy(np.concatenate([a_ptrs, b_ptrs]).astype(np.int64)).to(device)
        self.dims = torch.from_numpy(np.concatenate([self.n, self.nrhs]).astype(np.int32)).to(device)
        self.sched = torch.from_numpy(ebv_batch_schedule(self.n, self.nrhs, variant_of_n)).to(device)
        self.info = torch.zeros(max(1, self.batch), dtype=torch.int32, device=device)
        self.ws = torch.zeros(int(lib().ebv_batch_workspace_size(self.batch)), dtype=torch.uint8, device=device)

    def a_view(self, s):
        o, n = int(self.a_off[s]), int(self.n[s])
        return self.a_buf[o:o + n * n].view(n, n)

    def b_view(self, s):
        o, n, r = int(self.b_off[s]), int(self.n[s]), int(self.nrhs[s])
        return self.b_buf[o:o + n * r].view(n, r)

    def run(self):
        b = self.batch
        dp = self.ptrs.data_ptr()
        dd = self.dims.data_ptr()
        _check(lib().ebv_factor_solve_batched(b, ctypes.c_void_p(dd), ctypes.c_void_p(dd + 4 * b),
                                              ctypes.c_void_p(dp), ctypes.c_void_p(dp + 8 * b), self.prec,
                                              _ptr(self.sched), _ptr(self.info), _ptr(self.ws), self.ws.numel(),
                                              _stream(self.a_buf.device)), "ebv_factor_solve_batched")


def batch_autotune(orders, prec="fp64", reps=16, device="cuda", cache_path=None):
    """Fastest batched variant per order (times each variant on `reps`
    synthetic systems of that order).  Returns (variant_of_n array for every
    order 1..4096 filled by nearest tuned order, {order: [ms per variant]}).
    With cache_path, results are read from / written to that JSON file."""
    import json
    import numpy as np
    p = _prec(prec)
    cap = torch.cuda.get_device_capability(device)
    key = f"{torch.cuda.get_device_name(device)}|sm_{cap[0]}{cap[1]}|{p}|{reps}"
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as fh:
            cache = json.load(fh)
    entry = cache.get(key, {})
    todo = [int(o) for o in orders if str(int(o)) not in entry]
    if todo:
        arr = np.asarray(todo, dtype=np.int32)
        best = np.zeros(arr.size, dtype=np.int8)
        ms = np.zeros(arr.size * len(BATCH_VARIANTS), dtype=np.float32)
        scratch = torch.empty(int(lib().ebv_batch_autotune_scratch(int(arr.max()), reps, p)), dtype=torch.uint8,
                              device=device)
        _check(lib().ebv_batch_autotune(arr.ctypes.data, arr.size, reps, p, _ptr(scratch), scratch.numel(),
                                        best.ctypes.data, ms.ctypes.data, _stream(scratch.device)),
               "ebv_batch_autotune")
        nv = len(BATCH_VARIANTS)
        for i, o in enumerate(todo):
            entry[str(o)] = {"best": int(best[i]), "ms": [float(v) for v in ms[i * nv:(i + 1) * nv]]}
        cache[key] = entry
        if cache_path:
            os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
            with open(cache_path, "w") as fh:
                json.dump(cache, fh, indent=1, sort_keys=True)
    tuned = sorted((int(k), v["best"]) for k, v in entry.items())
    vmap = np.zeros(MAX_BATCH_ORDER, dtype=np.int8)
    keys = np.array([k for k, _ in tuned])
    vals = np.array([v for _, v in tuned], dtype=np.int8)
    for n in range(1, MAX_BATCH_ORDER + 1):
        vmap[n - 1] = vals[np.abs(keys - n).argmin()]
    return vmap, {k: entry[str(k)]["ms"] for k, _ in tuned}


BATCH_BUCKET = 32  # orders per autotuner size bucket


def batch_autotune_buckets(prec="fp64", nmin=16, nmax=512, reps=304, device="cuda", cache_path=None):
    """The autotuner over size buckets: orders nmin..nmax in buckets of
    BATCH_BUCKET, each tuned at its middle order on `reps` systems (304 = two
    resident CTAs on each of 152 SMs, so a launch is timed at full occupancy).
    Returns (variant_of_n for every order 1..4096, {bucket middle order:
    {"best": variant name, "ms": [ms per variant, -1 where not offered]}}).
    With cache_path the per-order results are kept in that JSON file, keyed
    by device name, compute capability, precision and reps."""
    mids = sorted({min(nmax, lo + BATCH_BUCKET // 2) for lo in range(nmin, nmax + 1, BATCH_BUCKET)})
    vmap, ms = batch_autotune(mids, prec, reps=reps, device=device, cache_path=cache_path)
    table = {m: {"best": BATCH_VARIANTS[int(vmap[m - 1])], "ms": [round(v, 4) for v in ms[m]]} for m in mids}
    return vmap, table


def uniform_batch(a: torch.Tensor, b: torch.Tensor, variant_of_n=None) -> "Batch":
    """A Batch over existing contiguous (batch, n, n) / (batch, n, nrhs) FP64 or
    FP32 tensors, factored and solved in place by ``run()``."""
    import numpy as np
    bsz, n, _ = a.shape
    nrhs = b.shape[2]
    self = Batch.__new__(Batch)
    self.prec = FP64 if a.dtype == torch.float64 else FP32
    self.dtype = a.dtype
    self.n = np.full(bsz, n, dtype=np.int64)
    self.nrhs = np.full(bsz, nrhs, dtype=np.int64)
    self.batch = bsz
    self.a_buf = a.view(-1)
    self.b_buf = b.view(-1)
    self.a_off = np.arange(bsz, dtype=np.int64) * n * n
    self.b_off = np.arange(bsz, dtype=np.int64) * n * nrhs
    esz = a.element_size()
    ptrs = np.concatenate([a.data_ptr() + self.a_off * esz, b.data_ptr() + self.b_off * esz]).astype(np.int64)
    self.ptrs = torch.from_numpy(ptrs).to(a.device)
    self.dims = torch.from_numpy(np.concatenate([self.n, self.nrhs]).astype(np.int32)).to(a.device)
    self.sched = torch.from_numpy(ebv_batch_schedule(self.n, self.nrhs, variant_of_n)).to(a.device)
    self.info = torch.zeros(bsz, dtype=torch.int32, device=a.device)
    self.ws = torch.zeros(int(lib().ebv_batch_workspace_size(bsz)), dtype=torch.uint8, device=a.device)
    return self


def ebv_solve_adjoint(lu: torch.Tensor, x: torch.Tensor, grad_x: torch.Tensor, want_grad_a: bool = True):
    """(grad_B, grad_A) for a batch of FP64 systems from their packed factors
    lu (batch, n, n), solutions x and dLoss/dX grad_x (batch, n, nrhs):
    grad_B = A^{-T} grad_X, grad_A = -grad_B X^T."""
    bsz, n, _ = lu.shape
    nrhs = x.shape[2]
    lu = lu.contiguous()
    x = x.contiguous()
    g = grad_x.contiguous().to(torch.float64)
    gb = torch.empty_like(g)
    ga = torch.empty((bsz, n, n), dtype=torch.float64, device=lu.device) if want_grad_a else None
    _check(lib().ebv_solve_adjoint(bsz, n, nrhs, _ptr(lu), n, n * n, _ptr(x), _ptr(g), _ptr(gb), _ptr(ga),
                                   _stream(lu.device)), "ebv_solve_adjoint")
    return gb, ga


class EbvSolve(torch.autograd.Function):
    """X = A^{-1} B for a batch of FP64 systems, A (batch, n, n), B (batch, n,
    nrhs).  Forward: batched EbV factor + solve (one persistent launch); the
    packed factors are kept.  Backward: the adjoint kernels reuse them."""

    @staticmethod
    def forward(ctx, a, b):
        lu = a.detach().to(torch.float64).contiguous().clone()
        x = b.detach().to(torch.float64).contiguous().clone()
        bt = uniform_batch(lu, x)
        bt.run()
        ctx.save_for_backward(lu, x)
        ctx.info = bt.info
        return x.clone()

    @staticmethod
    def backward(ctx, grad_x):
        lu, x = ctx.saved_tensors
        gb, ga = ebv_solve_adjoint(lu, x, grad_x, want_grad_a=ctx.needs_input_grad[0])
        return ga, gb


def tc_available() -> bool:
    return bool(lib().ebv_debug_tc_available())


def debug_lowp_update(c: torch.Tensor, lb: torch.Tensor, ut: torch.Tensor, scale: torch.Tensor, m0: int, n0: int,
                      k0: int, M: int, N: int, K: int, engine: str = "tc", ws: torch.Tensor | None = None,
                      check: bool = True) -> torch.Tensor:
    """C(m0.., n0..) -= scale[2] * lb(m0.., k0..) @ ut(n0.., k0..)^T in place (testing hook).
    check=True synchronises and raises if the device status reports a failure."""
    op = 0 if lb.dtype == torch.bfloat16 else 1
    if ws is None:
        ws = torch.empty(256, dtype=torch.uint8, device=c.device)
    _check(lib().ebv_debug_lowp_update(op, 2 if engine == "tc" else 1, _ptr(c), c.stride(0), _ptr(lb), _ptr(ut),
                                       lb.stride(0), _ptr(scale), m0, n0, k0, M, N, K, _ptr(ws), _stream(c.device)),
           "ebv_debug_lowp_update")
    if check:
        code, where = read_device_status(ws)
        if code != OK:
            raise EbvError(code, f"device status (where={where})")
    return c
