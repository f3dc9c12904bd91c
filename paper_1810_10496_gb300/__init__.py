"""Feature-similarity phase-order suggestion on GB300: thin binding of libfs.so.

The method (Nobre, Reis and Cardoso, Sec. 4): score a new kernel's code
features against a database of explored kernels with the cosine distance of
Sec. 4.2, keep the K most similar and suggest their best phase orders
(Table 1). Every step runs in the CUDA library; this module only marshals
arguments (torch tensors for device memory, the current torch stream) into
the C-ABI declared in ``include/fs.h``. Names follow that header.

The library must be built (``paper_1810_10496_gb300.build.build()``); there
is no CPU path, and every call raises if the library is missing.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfs.so")

FS_OK, FS_EINVAL, FS_ENOMEM, FS_ECUDA, FS_ETIMEOUT, FS_EUNSUPPORTED = range(6)
PRECISIONS = {"fp32": 0, "bf16": 1, "fp8": 2, "fp8_e4m3": 2}
METRICS = {"cosine": 0, "euclidean": 1, "manhattan": 2}
FS_MAX_K = 16
FS_NOALLOC_SCRATCH_BYTES = 32 << 20
STATUS_NAMES = {0: "FS_OK", 1: "FS_EINVAL", 2: "FS_ENOMEM", 3: "FS_ECUDA",
                4: "FS_ETIMEOUT", 5: "FS_EUNSUPPORTED"}
STAT_FIELDS = ("queries", "certified", "fallback", "fp64_evals", "near_ties", "rerank_evals",
               "band_rows")
STAGES = ("prepare", "scan", "select", "fallback", "gather")


class FsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class _Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in STAT_FIELDS]


class _Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * len(STAGES)), ("calls", ctypes.c_uint64 * len(STAGES)),
                ("launches", ctypes.c_uint64)]


TUNING_FIELDS = ("items_per_block", "list_len", "l2_share_pct", "scan_pairs")


class _Tuning(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in TUNING_FIELDS]


_lib = None
P = ctypes.c_void_p
I32, I64, SZ = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t

_SIGNATURES = {
    "fs_normalize": [P, I64, I32, I64, P, P, P],
    "fs_build_db": [P, I64, I32, P, P, P, I32, ctypes.c_int, P, ctypes.POINTER(P)],
    "fs_workspace_size": [P, I32, P, ctypes.POINTER(SZ)],
    "fs_knn": [P, P, I32, P, P, P, P, SZ, P, P, P],
    "fs_recommend": [P, P, I32, P, P, P, P, SZ, P, P, P, P, I32, P, P],
    "fs_knn_noalloc": [P, P, I32, P, P, P, P, P, P],
    "fs_db_destroy": [P],
    "fs_db_check": [P, P],
    "fs_db_stats": [P, P, I32, ctypes.POINTER(_Stats)],
    "fs_db_set_tuning": [P, ctypes.POINTER(_Tuning)],
    "fs_db_set_metric": [P, ctypes.c_int, P],
    "fs_db_get_tuning": [P, ctypes.POINTER(_Tuning)],
    "fs_db_set_wait_test": [P, I32, ctypes.c_uint32],
    "fs_profile_enable": [I32],
    "fs_profile_read": [I32, ctypes.POINTER(_Profile)],
}


def lib() -> ctypes.CDLL:
    """The loaded C library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is not built; run paper_1810_10496_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.fs_last_error.argtypes = []
        L.fs_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def fs_last_error() -> str:
    return lib().fs_last_error().decode()


def _check(status: int):
    if status != FS_OK:
        raise FsError(status, fs_last_error())


def _torch():
    import torch
    return torch


def _stream(stream):
    torch = _torch()
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t):
    return None if t is None else t.data_ptr()


def _dev_tensor(t, dtype, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _host_i32(vals):
    if vals is None:
        return None
    a = np.ascontiguousarray(np.asarray(vals, dtype=np.int32))
    return a


def _host_i64(vals):
    if vals is None:
        return None
    return np.ascontiguousarray(np.asarray(vals, dtype=np.int64))


def _np_ptr(a):
    return None if a is None else a.ctypes.data


def fs_normalize(x, x_unit=None, inv_norm=None, stream=None):
    """Unit rows of ``x`` (float32 [n, f], rows may be strided)."""
    torch = _torch()
    if not x.is_cuda or x.dtype != torch.float32 or x.dim() != 2 or x.stride(1) != 1:
        raise TypeError("x must be a CUDA float32 [n, f] tensor with unit column stride")
    n, f = x.shape
    if x_unit is None:
        x_unit = torch.empty((n, f), device=x.device, dtype=torch.float32)
    if inv_norm is None:
        inv_norm = torch.empty((n,), device=x.device, dtype=torch.float32)
    _check(lib().fs_normalize(_ptr(x), n, f, x.stride(0), _ptr(x_unit), _ptr(inv_norm),
                              _stream(stream)))
    return x_unit, inv_norm


class Database:
    """Owner of an ``fs_db`` handle (freed with :meth:`close` or on deletion)."""

    def __init__(self, handle, n, f, n_seg, prec, device):
        self.handle = handle
        self.n, self.f, self.n_seg, self.prec, self.device = n, f, n_seg, prec, device
        self.metric = "cosine"

    def close(self):
        if self.handle:
            _check(lib().fs_db_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fs_build_db(x, seq_off, seq_ids, seg_off=None, prec="fp32", stream=None) -> Database:
    """Copy the reference set to the device (``x`` float32 [n, f], CSR phase
    orders ``seq_off`` int64 [n+1] / ``seq_ids`` int16, optional host segment
    offsets)."""
    torch = _torch()
    x = _dev_tensor(x, torch.float32, "x")
    seq_off = _dev_tensor(seq_off, torch.int64, "seq_off")
    seq_ids = _dev_tensor(seq_ids, torch.int16, "seq_ids")
    n, f = x.shape
    segs = _host_i64(seg_off)
    n_seg = 1 if segs is None else len(segs) - 1
    h = P()
    _check(lib().fs_build_db(_ptr(x), n, f, _ptr(seq_off), _ptr(seq_ids) if seq_ids.numel() else None,
                             _np_ptr(segs), n_seg, PRECISIONS[prec], _stream(stream),
                             ctypes.byref(h)))
    return Database(h, n, f, n_seg, prec, x.device)


def fs_workspace_size(db: Database, nq: int, q_seg_off=None) -> int:
    qs = _host_i32(q_seg_off)
    out = SZ(0)
    _check(lib().fs_workspace_size(db.handle, nq, _np_ptr(qs), ctypes.byref(out)))
    return out.value


def _k_array(db, k):
    if isinstance(k, (int, np.integer)):
        return np.full(db.n_seg, int(k), dtype=np.int32)
    return _host_i32(k)


def _search_args(db, q, k, q_seg_off, exclude, workspace, idx, dist):
    torch = _torch()
    q = _dev_tensor(q, torch.float32, "q")
    nq = q.shape[0]
    ks = _k_array(db, k)
    qs = _host_i32(q_seg_off)
    k_max = int(ks.max()) if len(ks) else 1
    if workspace is None:
        workspace = torch.empty(max(fs_workspace_size(db, nq, qs), 1), device=q.device,
                                dtype=torch.uint8)
    if idx is None:
        idx = torch.empty((nq, k_max), device=q.device, dtype=torch.int32)
    if dist is None:
        dist = torch.empty((nq, k_max), device=q.device, dtype=torch.float32)
    if exclude is not None:
        exclude = _dev_tensor(exclude, torch.int32, "exclude")
    return q, nq, ks, qs, k_max, workspace, idx, dist, exclude


def fs_knn(db: Database, q, k, q_seg_off=None, exclude=None, workspace=None, idx=None,
           dist=None, stream=None):
    """k nearest rows per query: ``(idx int32 [nq, k_max], dist float32)``."""
    q, nq, ks, qs, k_max, ws, idx, dist, exclude = _search_args(db, q, k, q_seg_off, exclude,
                                                                workspace, idx, dist)
    _check(lib().fs_knn(db.handle, _ptr(q), nq, _np_ptr(qs), _np_ptr(ks), _ptr(exclude),
                        _ptr(ws), ws.numel() * ws.element_size(), _ptr(idx), _ptr(dist),
                        _stream(stream)))
    return idx, dist


def fs_knn_noalloc(db: Database, q, k, q_seg_off=None, exclude=None, idx=None, dist=None,
                   stream=None):
    """fs_knn without a workspace: the scratch is the library's fixed static
    array (FS_NOALLOC_SCRATCH_BYTES), so nothing is allocated on the device
    for scratch. Calls that overlap on the GPU race on that array."""
    torch = _torch()
    q = _dev_tensor(q, torch.float32, "q")
    nq = q.shape[0]
    ks = _k_array(db, k)
    qs = _host_i32(q_seg_off)
    k_max = int(ks.max()) if len(ks) else 1
    if idx is None:
        idx = torch.empty((nq, k_max), device=q.device, dtype=torch.int32)
    if dist is None:
        dist = torch.empty((nq, k_max), device=q.device, dtype=torch.float32)
    if exclude is not None:
        exclude = _dev_tensor(exclude, torch.int32, "exclude")
    _check(lib().fs_knn_noalloc(db.handle, _ptr(q), nq, _np_ptr(qs), _np_ptr(ks), _ptr(exclude),
                                _ptr(idx), _ptr(dist), _stream(stream)))
    return idx, dist


def fs_recommend(db: Database, q, k, q_seg_off=None, exclude=None, l_max=128, workspace=None,
                 idx=None, dist=None, seq_out=None, seq_len=None, dup_of=None, want_dup=False,
                 stream=None):
    """k nearest rows and their phase orders:
    ``(idx, dist, seq_out int16 [nq, k_max, l_max], seq_len int32, dup_of | None)``."""
    torch = _torch()
    q, nq, ks, qs, k_max, ws, idx, dist, exclude = _search_args(db, q, k, q_seg_off, exclude,
                                                                workspace, idx, dist)
    if seq_out is None:
        seq_out = torch.empty((nq, k_max, l_max), device=q.device, dtype=torch.int16)
    if seq_len is None:
        seq_len = torch.empty((nq, k_max), device=q.device, dtype=torch.int32)
    if want_dup and dup_of is None:
        dup_of = torch.empty((nq, k_max), device=q.device, dtype=torch.int32)
    _check(lib().fs_recommend(db.handle, _ptr(q), nq, _np_ptr(qs), _np_ptr(ks), _ptr(exclude),
                              _ptr(ws), ws.numel() * ws.element_size(), _ptr(idx), _ptr(dist),
                              _ptr(seq_out), _ptr(seq_len), l_max, _ptr(dup_of), _stream(stream)))
    return idx, dist, seq_out, seq_len, dup_of


def fs_db_check(db: Database, stream=None):
    _check(lib().fs_db_check(db.handle, _stream(stream)))


def fs_db_stats(db: Database, reset: bool = False, stream=None) -> dict:
    st = _Stats()
    _check(lib().fs_db_stats(db.handle, _stream(stream), 1 if reset else 0, ctypes.byref(st)))
    return {n: int(getattr(st, n)) for n in STAT_FIELDS}


def fs_db_set_metric(db: Database, metric: str = "cosine", stream=None):
    """The similarity of later searches: "cosine" (Sec. 4.2), or "euclidean" /
    "manhattan" on features standardised per segment (FP32 databases)."""
    _check(lib().fs_db_set_metric(db.handle, METRICS[metric], _stream(stream)))
    db.metric = metric


def fs_db_set_tuning(db: Database, tuning: dict | None):
    """Scan planning parameters (``TUNING_FIELDS``; missing or 0 = default;
    None restores every default). Size workspaces after this call."""
    if tuning is None:
        _check(lib().fs_db_set_tuning(db.handle, None))
        return
    bad = set(tuning) - set(TUNING_FIELDS)
    if bad:
        raise ValueError(f"unknown tuning fields {sorted(bad)}")
    t = _Tuning(*(int(tuning.get(n, 0)) for n in TUNING_FIELDS))
    _check(lib().fs_db_set_tuning(db.handle, ctypes.byref(t)))


def fs_db_get_tuning(db: Database) -> dict:
    t = _Tuning()
    _check(lib().fs_db_get_tuning(db.handle, ctypes.byref(t)))
    return {n: int(getattr(t, n)) for n in TUNING_FIELDS}


def fs_db_set_wait_test(db: Database, withhold_first_load: bool, wait_limit_us: int = 0):
    """Test aid: later tensor-core scans on `db` skip their first tile copy
    so their bounded waits run out after `wait_limit_us` (0: the default 2 s);
    fs_db_check then reports FS_ETIMEOUT."""
    _check(lib().fs_db_set_wait_test(db.handle, 1 if withhold_first_load else 0,
                                     int(wait_limit_us)))


def fs_db_destroy(db: Database):
    """Free the database's device memory (same as ``db.close()``)."""
    db.close()


def fs_profile_enable(on: bool = True):
    """Record CUDA events around each stage of every search call."""
    _check(lib().fs_profile_enable(1 if on else 0))


def fs_profile_read(reset: bool = False) -> dict:
    """Per-stage summed milliseconds and call counts, and kernel launches."""
    pr = _Profile()
    _check(lib().fs_profile_read(1 if reset else 0, ctypes.byref(pr)))
    return {"ms": {s: pr.ms[i] for i, s in enumerate(STAGES)},
            "calls": {s: int(pr.calls[i]) for i, s in enumerate(STAGES)},
            "launches": int(pr.launches)}
