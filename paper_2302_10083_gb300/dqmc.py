"""ctypes binding of libdqmc.so (C ABI in include/dqmc.h, include/dqmc_plan.h,
include/dqmc_batch.h and include/dqmc_server.h).

Argument marshalling only: every step of the sweep runs in the library's CUDA
kernels.  The functions named ``dqmc_*`` mirror the C entry points one to one;
the short helpers below them (``primes``, ``count``, ``pairs``, ``*_tensor``)
just allocate outputs for convenience.  There is no CPU fallback: if the
library is missing, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import json
import os
import threading

import numpy as np

from . import build as _build

DQMC_OK = 0
DQMC_EINVAL = -1
DQMC_ENOMEM = -2
DQMC_ETRUNC = -3
DQMC_ECUDA = -4
DQMC_ETIMEOUT = -5
DQMC_MAX_N = 25
DQMC_COMPLEMENT = 1   # flag of the *_ex entry points: the primes of not-f

_lock = threading.Lock()
_lib = None

c_u8p = ctypes.POINTER(ctypes.c_uint8)
c_u32p = ctypes.POINTER(ctypes.c_uint32)
c_u64p = ctypes.POINTER(ctypes.c_uint64)
c_vp = ctypes.c_void_p


class DqmcError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})" if what else strerror(status))


_SIGS = {
    "dqmc_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "dqmc_version": (ctypes.c_int, []),
    "dqmc_bitmap_bytes": (ctypes.c_uint64, [ctypes.c_uint32]),
    "dqmc_bitmap_alloc_bytes": (ctypes.c_uint64, [ctypes.c_uint32]),
    "dqmc_workspace_bytes": (ctypes.c_uint64, [ctypes.c_uint32]),
    "dqmc_primes": (ctypes.c_int, [ctypes.c_uint32, c_u8p, c_u8p, c_u8p]),
    "dqmc_count": (ctypes.c_int, [ctypes.c_uint32, c_u8p, c_u8p, c_u64p]),
    "dqmc_list": (ctypes.c_int, [ctypes.c_uint32, c_u8p, c_u8p, c_u32p, ctypes.c_uint64, c_u64p]),
    "dqmc_primes_ex": (ctypes.c_int, [ctypes.c_uint32, c_u8p, c_u8p, ctypes.c_uint32, c_u8p, c_u64p]),
    "dqmc_list_ex": (ctypes.c_int, [ctypes.c_uint32, c_u8p, c_u8p, ctypes.c_uint32, c_u32p, ctypes.c_uint64,
                                    c_u64p]),
    "dqmc_primes_dev_ex": (ctypes.c_int, [ctypes.c_uint32, c_vp, c_vp, ctypes.c_uint32, c_vp, c_vp, c_vp,
                                          ctypes.c_uint64, c_vp]),
    "dqmc_list_dev_ex": (ctypes.c_int, [ctypes.c_uint32, c_vp, c_vp, ctypes.c_uint32, c_vp, c_vp, ctypes.c_uint64,
                                        c_vp, c_vp, ctypes.c_uint64, c_vp]),
    "dqmc_sparse_list": (ctypes.c_int, [ctypes.c_uint32, c_u8p, c_u8p, ctypes.c_uint32, c_u32p, ctypes.c_uint64,
                                        c_u64p]),
    "dqmc_cover": (ctypes.c_int, [ctypes.c_uint32, c_u8p, c_u8p, c_u32p, ctypes.c_uint64, c_u32p, c_u64p]),
    "dqmc_release": (None, []),
    "dqmc_primes_dev": (ctypes.c_int, [ctypes.c_uint32, c_vp, c_vp, c_vp, c_vp, c_vp, ctypes.c_uint64, c_vp]),
    "dqmc_list_dev": (ctypes.c_int, [ctypes.c_uint32, c_vp, c_vp, c_vp, c_vp, ctypes.c_uint64, c_vp, c_vp,
                                     ctypes.c_uint64, c_vp]),
    "dqmc_compact_dev": (ctypes.c_int, [ctypes.c_uint32, c_vp, c_vp, ctypes.c_uint64, c_vp, c_vp,
                                        ctypes.c_uint64, c_vp]),
    "dqmc_plan_json": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_char_p, ctypes.c_uint64]),
    "dqmc_plan_passes": (ctypes.c_int, [ctypes.c_uint32]),
    "dqmc_dev_status": (ctypes.c_int, [ctypes.c_uint32, c_vp, ctypes.c_uint64, c_vp]),
    "dqmc_pass_bytes": (ctypes.c_uint64, [ctypes.c_uint32, ctypes.c_int, ctypes.c_int]),
    "dqmc_sweep_pass_dev": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_int, c_vp, c_vp, c_vp, c_vp,
                                           ctypes.c_uint64, c_vp, c_vp, ctypes.c_uint64, c_vp]),
    "dqmc_sweep_passes_dev": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_int, ctypes.c_int, c_vp, c_vp, c_vp, c_vp,
                                             ctypes.c_uint64, c_vp, c_vp, ctypes.c_uint64, c_vp]),
    "dqmc_selftest_timeout": (ctypes.c_int, [ctypes.c_uint32, c_vp, ctypes.c_uint64, ctypes.c_uint64, c_vp]),
    "dqmc_primes_dev_static": (ctypes.c_int, [ctypes.c_uint32, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "dqmc_dev_status_static": (ctypes.c_int, [ctypes.c_uint32, c_vp]),
    "dqmc_batch_run": (ctypes.c_int, [ctypes.c_uint32, c_u32p, c_u64p, c_vp, c_u64p, c_vp, c_vp, c_u64p, c_vp]),
    "dqmc_batch_run_one_launch": (ctypes.c_int, [ctypes.c_uint32, c_u32p, c_u64p, c_vp, c_u64p, c_vp, c_vp, c_u64p,
                                                 c_vp]),
    "dqmc_batch_workspace_bytes": (ctypes.c_uint64, [ctypes.c_uint32, c_u32p]),
    "dqmc_batch_release": (ctypes.c_int, []),
    "dqmc_batch_get_config": (ctypes.c_int, [ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32 * 5)]),
    "dqmc_batch_set_config": (ctypes.c_int, [ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32 * 5)]),
    "dqmc_batch_autotune": (ctypes.c_int, [ctypes.c_uint32, c_u32p, c_u64p, c_vp, c_u64p, c_vp, c_vp, c_u64p,
                                           ctypes.c_uint32, c_vp, ctypes.POINTER(ctypes.c_float)]),
    "dqmc_server_create": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.POINTER(c_vp)]),
    "dqmc_server_destroy": (ctypes.c_int, [c_vp]),
    "dqmc_server_job_bytes": (ctypes.c_uint64, [ctypes.c_uint32, ctypes.c_int]),
    "dqmc_server_submit": (ctypes.c_int, [c_vp, ctypes.c_uint32, c_u8p, c_u8p, ctypes.c_uint32, c_u64p]),
    "dqmc_server_query": (ctypes.c_int, [c_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), c_u64p,
                                         ctypes.POINTER(c_vp), c_u64p, c_u64p]),
    "dqmc_server_copy_bitmap": (ctypes.c_int, [c_vp, ctypes.c_uint64, c_u8p, ctypes.c_uint64]),
    "dqmc_server_wait": (ctypes.c_int, [c_vp, ctypes.c_uint64, ctypes.c_uint32]),
    "dqmc_server_free_job": (ctypes.c_int, [c_vp, ctypes.c_uint64]),
    "dqmc_server_stats": (ctypes.c_int, [c_vp, c_u64p]),
    "dqmc_server_replay": (ctypes.c_int, [c_vp, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double), c_u32p, c_vp,
                                          c_vp, c_u64p, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]),
}


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libdqmc.so (building it with nvcc first if needed and allowed)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing and not _build.up_to_date():
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libdqmc.so not found at {path}; run __graft_entry__.build()")
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().dqmc_strerror(status).decode()


def _check(status: int, what: str, ok=(DQMC_OK,)):
    if status not in ok:
        raise DqmcError(status, what)
    return status


def _host_tt(buf, n):
    if buf is None:
        return None
    a = np.ascontiguousarray(np.frombuffer(bytes(buf), dtype=np.uint8) if not isinstance(buf, np.ndarray)
                             else buf.view(np.uint8).reshape(-1))
    if a.size < ((1 << n) + 7) >> 3:
        raise ValueError("truth table too short")
    return a


def _p8(a):
    return None if a is None else a.ctypes.data_as(c_u8p)


# --------------------------------------------------------------- sizes, plan

def dqmc_bitmap_bytes(n: int) -> int:
    return int(lib().dqmc_bitmap_bytes(n))


def dqmc_bitmap_alloc_bytes(n: int) -> int:
    return int(lib().dqmc_bitmap_alloc_bytes(n))


def dqmc_workspace_bytes(n: int) -> int:
    return int(lib().dqmc_workspace_bytes(n))


def dqmc_plan_json(n: int) -> dict:
    L = lib()
    need = L.dqmc_plan_json(n, None, 0)
    _check(min(need, 0), "dqmc_plan_json")
    buf = ctypes.create_string_buffer(need + 1)
    L.dqmc_plan_json(n, buf, need + 1)
    return json.loads(buf.value.decode())


def dqmc_plan_passes(n: int) -> int:
    return _check(lib().dqmc_plan_passes(n), "dqmc_plan_passes", ok=tuple(range(0, 1000)))


def dqmc_pass_bytes(n: int, pass_index: int, with_dc: bool = False) -> int:
    return int(lib().dqmc_pass_bytes(n, pass_index, int(with_dc)))


# ----------------------------------------------------------------- host API

def dqmc_primes(n: int, on_bits, dc_bits=None) -> np.ndarray:
    """Prime bitmap (uint8, dqmc_bitmap_bytes(n)) through the host entry point."""
    on = _host_tt(on_bits, n)
    dc = _host_tt(dc_bits, n)
    out = np.empty(max(dqmc_bitmap_bytes(n), 1), dtype=np.uint8)
    _check(lib().dqmc_primes(n, _p8(on), _p8(dc), _p8(out)), "dqmc_primes")
    return out[: dqmc_bitmap_bytes(n)]


def dqmc_count(n: int, on_bits, dc_bits=None) -> int:
    on = _host_tt(on_bits, n)
    dc = _host_tt(dc_bits, n)
    c = ctypes.c_uint64()
    _check(lib().dqmc_count(n, _p8(on), _p8(dc), ctypes.byref(c)), "dqmc_count")
    return int(c.value)


def _list_cap_guess(n: int, on, dc) -> int:
    """A first list size for dqmc_list(cap=None): the expected prime count of a
    function whose support has the same density with independent minterms,
    with headroom.  Only sizes a host buffer; a function with more primes is
    swept a second time with the exact count."""
    from math import comb
    m = 1 << n
    sup = np.unpackbits(on[: (m + 7) >> 3], bitorder="little")[:m]
    if dc is not None:
        sup = sup | np.unpackbits(dc[: (m + 7) >> 3], bitorder="little")[:m]
    p = float(sup.mean()) if m else 0.0
    e = sum(comb(n, w) * 2.0 ** (n - w) * p ** (2 ** w) * (1.0 - p ** (2 ** w)) ** (n - w) for w in range(n + 1))
    return int(1.1 * e) + 4096


def dqmc_list(n: int, on_bits, dc_bits=None, cap: int | None = None):
    """(pairs (count, 2) uint32, count).  With cap=None the buffer is first
    sized by the expected count of a random function of the same density; if
    the true count is larger, the list is taken again at that size."""
    on = _host_tt(on_bits, n)
    dc = _host_tt(dc_bits, n)
    auto = cap is None
    if auto:
        cap = _list_cap_guess(n, on, dc)
    while True:
        out = np.empty(2 * max(cap, 1), dtype=np.uint32)
        c = ctypes.c_uint64()
        st = lib().dqmc_list(n, _p8(on), _p8(dc), out.ctypes.data_as(c_u32p), cap, ctypes.byref(c))
        _check(st, "dqmc_list", ok=(DQMC_OK, DQMC_ETRUNC))
        if not (auto and st == DQMC_ETRUNC):
            break
        cap = int(c.value)
    k = min(int(c.value), cap)
    return out[: 2 * k].reshape(k, 2), int(c.value)


def dqmc_primes_ex(n: int, on_bits, dc_bits=None, flags: int = 0):
    """(prime bitmap, count) through dqmc_primes_ex (flags: 0 or DQMC_COMPLEMENT)."""
    on = _host_tt(on_bits, n)
    dc = _host_tt(dc_bits, n)
    out = np.empty(max(dqmc_bitmap_bytes(n), 1), dtype=np.uint8)
    c = ctypes.c_uint64()
    _check(lib().dqmc_primes_ex(n, _p8(on), _p8(dc), flags, _p8(out), ctypes.byref(c)), "dqmc_primes_ex")
    return out[: dqmc_bitmap_bytes(n)], int(c.value)


def dqmc_list_ex(n: int, on_bits, dc_bits=None, flags: int = 0, cap: int = 0):
    """(pairs (k, 2) uint32, count) through dqmc_list_ex; k = min(count, cap)."""
    on = _host_tt(on_bits, n)
    dc = _host_tt(dc_bits, n)
    out = np.empty(2 * max(cap, 1), dtype=np.uint32)
    c = ctypes.c_uint64()
    st = lib().dqmc_list_ex(n, _p8(on), _p8(dc), flags, out.ctypes.data_as(c_u32p), cap, ctypes.byref(c))
    _check(st, "dqmc_list_ex", ok=(DQMC_OK, DQMC_ETRUNC))
    k = min(int(c.value), cap)
    return out[: 2 * k].reshape(k, 2), int(c.value)


DQMC_SPARSE_MAX_N = 30


def dqmc_sparse_list(n: int, on_bits, dc_bits=None, flags: int = 0, cap: int | None = None):
    """(pairs (k, 2) uint32 in ascending rho, count) through dqmc_sparse_list
    (SparseQMC on the GPU); cap=None sizes the buffer as dqmc_list does."""
    on = _host_tt(on_bits, n)
    dc = _host_tt(dc_bits, n)
    auto = cap is None
    if auto:
        cap = _list_cap_guess(n, on, dc)
    while True:
        out = np.empty(2 * max(cap, 1), dtype=np.uint32)
        c = ctypes.c_uint64()
        st = lib().dqmc_sparse_list(n, _p8(on), _p8(dc), flags, out.ctypes.data_as(c_u32p), cap, ctypes.byref(c))
        _check(st, "dqmc_sparse_list", ok=(DQMC_OK, DQMC_ETRUNC))
        if not (auto and st == DQMC_ETRUNC):
            break
        cap = int(c.value)
    k = min(int(c.value), cap)
    return out[: 2 * k].reshape(k, 2), int(c.value)


def dqmc_cover(n: int, on_bits, dc_bits, pairs) -> np.ndarray:
    """Indexes (ascending) of the primes dqmc_cover selects: essentials, then
    greedy by uncovered ON minterms (ties: lowest index)."""
    on = _host_tt(on_bits, n)
    dc = _host_tt(dc_bits, n)
    pr = np.ascontiguousarray(pairs, dtype=np.uint32).reshape(-1, 2)
    out = np.empty(max(len(pr), 1), dtype=np.uint32)
    k = ctypes.c_uint64()
    _check(lib().dqmc_cover(n, _p8(on), _p8(dc), pr.ctypes.data_as(c_u32p), len(pr), out.ctypes.data_as(c_u32p),
                            ctypes.byref(k)), "dqmc_cover")
    return out[: k.value].copy()


def dqmc_release() -> None:
    lib().dqmc_release()


# --------------------------------------------------------------- device API
# Arguments are raw device addresses (ints, e.g. torch.Tensor.data_ptr()) and a
# cudaStream_t handle as int (torch.cuda.Stream.cuda_stream).

def dqmc_primes_dev(n, d_on, d_dc, d_bitmap, d_count, d_work, work_bytes, stream) -> int:
    return _check(lib().dqmc_primes_dev(n, d_on, d_dc or None, d_bitmap, d_count or None, d_work, work_bytes,
                                        stream or None), "dqmc_primes_dev")


def dqmc_sweep_pass_dev(n, pass_index, d_on, d_dc, d_bitmap, d_pairs, cap, d_count, d_work, work_bytes,
                        stream) -> int:
    return _check(lib().dqmc_sweep_pass_dev(n, pass_index, d_on, d_dc or None, d_bitmap, d_pairs or None, cap,
                                            d_count or None, d_work, work_bytes, stream or None),
                  "dqmc_sweep_pass_dev")


def dqmc_selftest_timeout(n, d_work, work_bytes, wait_ns, stream) -> int:
    return _check(lib().dqmc_selftest_timeout(n, d_work, work_bytes, wait_ns, stream or None),
                  "dqmc_selftest_timeout")


def dqmc_list_dev(n, d_on, d_dc, d_bitmap, d_pairs, cap, d_count, d_work, work_bytes, stream) -> int:
    return _check(lib().dqmc_list_dev(n, d_on, d_dc or None, d_bitmap, d_pairs or None, cap, d_count, d_work,
                                      work_bytes, stream or None), "dqmc_list_dev")


def dqmc_dev_status(n, d_work, work_bytes, stream) -> int:
    return _check(lib().dqmc_dev_status(n, d_work, work_bytes, stream or None), "dqmc_dev_status")


def dqmc_primes_dev_static(n, d_on, d_dc, d_bitmap, d_count, stream) -> int:
    """dqmc_primes_dev with the library's static 2 MiB workspace (n <= 15, allocates nothing)."""
    return _check(lib().dqmc_primes_dev_static(n, d_on, d_dc or None, d_bitmap, d_count or None, stream or None),
                  "dqmc_primes_dev_static")


def dqmc_dev_status_static(n, stream) -> int:
    """How the last dqmc_primes_dev_static sweep on the current device ended."""
    return _check(lib().dqmc_dev_status_static(n, stream or None), "dqmc_dev_status_static")


def dqmc_compact_dev(n, d_bitmap, d_pairs, cap, d_count, d_work, work_bytes, stream) -> int:
    return _check(lib().dqmc_compact_dev(n, d_bitmap, d_pairs or None, cap, d_count, d_work, work_bytes,
                                         stream or None), "dqmc_compact_dev")


# ------------------------------------------------------- torch conveniences

class DeviceBuffers:
    """Device tensors for one n: inputs, bitmap, count, workspace (torch-owned).
    With inplace=True (n >= 13) the bitmap is the start of the workspace: the
    sweep writes it over its state (one array instead of two)."""

    def __init__(self, n: int, device="cuda", with_dc: bool = False, cap: int = 0, inplace: bool = False):
        import torch
        self.n = n
        tt = max(((1 << n) + 7) >> 3, 1)
        tt_alloc = (tt + 15) // 16 * 16
        self.on = torch.zeros(tt_alloc, dtype=torch.uint8, device=device)
        self.dc = torch.zeros(tt_alloc, dtype=torch.uint8, device=device) if with_dc else None
        self.count = torch.zeros(1, dtype=torch.int64, device=device)
        wb = dqmc_workspace_bytes(n)
        self.work = torch.empty(max(wb, 256), dtype=torch.uint8, device=device)
        self.work_bytes = self.work.numel()
        if inplace:
            if n < 13:
                raise ValueError("the bitmap can share the workspace only for n >= 13")
            self.bitmap = self.work[: dqmc_bitmap_alloc_bytes(n)]
        else:
            self.bitmap = torch.empty(dqmc_bitmap_alloc_bytes(n), dtype=torch.uint8, device=device)
        self.cap = cap
        self.pairs = torch.empty(2 * max(cap, 1), dtype=torch.int32, device=device)

    def primes(self, stream=None):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        return dqmc_primes_dev(self.n, self.on.data_ptr(), self.dc.data_ptr() if self.dc is not None else None,
                               self.bitmap.data_ptr(), self.count.data_ptr(), self.work.data_ptr(),
                               self.work_bytes, s.cuda_stream)

    def status(self, stream=None):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        return dqmc_dev_status(self.n, self.work.data_ptr(), self.work_bytes, s.cuda_stream)

    def list(self, stream=None):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        return dqmc_list_dev(self.n, self.on.data_ptr(), self.dc.data_ptr() if self.dc is not None else None,
                             self.bitmap.data_ptr(), self.pairs.data_ptr() if self.cap else None, self.cap,
                             self.count.data_ptr(), self.work.data_ptr(), self.work_bytes, s.cuda_stream)


# ------------------------------------------------------------------ batch

DQMC_BATCH_MAX_N = 14


def _host_u32(a):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return a, a.ctypes.data_as(c_u32p)


def _host_u64(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a, a.ctypes.data_as(c_u64p)


def batch_bitmap_layout(ns):
    """Bitmap slots for a batch: byte offset of each function's bitmap
    (dqmc_bitmap_alloc_bytes(n) bytes each, 16-aligned) and the total bytes."""
    sizes = np.array([dqmc_bitmap_alloc_bytes(int(n)) for n in ns], dtype=np.uint64)
    off = np.zeros(len(sizes), dtype=np.uint64)
    if len(sizes):
        off[1:] = np.cumsum(sizes)[:-1]
    return off, int(sizes.sum())


def dqmc_batch_workspace_bytes(ns) -> int:
    a, p = _host_u32(ns)
    return int(lib().dqmc_batch_workspace_bytes(len(a), p))


def dqmc_batch_run(ns, tt_off, d_arena, dc_off, d_counts, d_bitmaps, bm_off, stream, one_launch=False) -> int:
    """dqmc_batch_run (one_launch: dqmc_batch_run_one_launch): ns / tt_off /
    dc_off / bm_off are host arrays (dc_off may be None), the d_* arguments
    device pointers (ints), stream a cudaStream_t (int or None).  Returns the
    status."""
    n_a, n_p = _host_u32(ns)
    tt_a, tt_p = _host_u64(tt_off)
    bm_a, bm_p = _host_u64(bm_off)
    if dc_off is None:
        dc_a, dc_p = None, None
    else:
        dc_a, dc_p = _host_u64(dc_off)
    fn = lib().dqmc_batch_run_one_launch if one_launch else lib().dqmc_batch_run
    return fn(len(n_a), n_p, tt_p, d_arena, dc_p, d_counts, d_bitmaps, bm_p, stream)


def dqmc_batch_release() -> int:
    return lib().dqmc_batch_release()


DQMC_BATCH_PATH_SMEM = 0
DQMC_BATCH_PATH_TILES = 1
_CFG_KEYS = ("path", "threads_per_fn", "fns_per_cta", "digits_per_step", "ctas_per_fn")


def dqmc_batch_get_config(n: int) -> dict:
    """The launch configuration (dqmc_batch_config) used for functions of n variables."""
    buf = (ctypes.c_uint32 * 5)()
    st = lib().dqmc_batch_get_config(n, ctypes.byref(buf))
    if st != DQMC_OK:
        raise DqmcError(st, "dqmc_batch_get_config")
    return dict(zip(_CFG_KEYS, (int(x) for x in buf)))


def dqmc_batch_set_config(n: int, cfg: dict) -> int:
    """Set one n's configuration (keys of dqmc_batch_get_config); returns the status."""
    buf = (ctypes.c_uint32 * 5)(*(int(cfg.get(k, 1)) for k in _CFG_KEYS))
    return lib().dqmc_batch_set_config(n, ctypes.byref(buf))


def dqmc_batch_autotune(ns, tt_off, d_arena, dc_off, d_counts, d_bitmaps, bm_off, stream, reps=3):
    """dqmc_batch_autotune on a batch (arguments as dqmc_batch_run).  Returns
    {n: best ms} for the n's present; raises DqmcError on failure."""
    n_a, n_p = _host_u32(ns)
    tt_a, tt_p = _host_u64(tt_off)
    bm_a, bm_p = _host_u64(bm_off)
    if dc_off is None:
        dc_a, dc_p = None, None
    else:
        dc_a, dc_p = _host_u64(dc_off)
    out = (ctypes.c_float * (DQMC_BATCH_MAX_N + 1))()
    st = lib().dqmc_batch_autotune(len(n_a), n_p, tt_p, d_arena, dc_p, d_counts, d_bitmaps, bm_p, reps, stream, out)
    if st != DQMC_OK:
        raise DqmcError(st, "dqmc_batch_autotune")
    return {n: float(out[n]) for n in range(DQMC_BATCH_MAX_N + 1) if out[n] >= 0}


def batch_tuning_table() -> dict:
    """Every n's configuration, keyed by n as a string (the JSON form)."""
    return {str(n): dqmc_batch_get_config(n) for n in range(DQMC_BATCH_MAX_N + 1)}


def load_batch_tuning(table: dict) -> None:
    """Apply a table from batch_tuning_table (for instance read back from JSON)."""
    for k, cfg in table.items():
        st = dqmc_batch_set_config(int(k), cfg)
        if st != DQMC_OK:
            raise DqmcError(st, f"dqmc_batch_set_config({k})")


# ------------------------------------------------------------------ serving

DQMC_SERVER_CONCURRENT = 0
DQMC_SERVER_SERIAL = 1
DQMC_JOB_DISCARD_BITMAP = 1
DQMC_JOB_QUEUED, DQMC_JOB_RUNNING, DQMC_JOB_DONE = 0, 1, 2


def dqmc_server_job_bytes(n: int, with_dc: bool = False) -> int:
    return int(lib().dqmc_server_job_bytes(n, 1 if with_dc else 0))


class Server:
    """The library's serving loop (dqmc_server_*): jobs admitted by device-memory
    footprint, small jobs batched on arrival, results device-resident."""

    def __init__(self, hbm_bytes: int, streams: int = 8, mode: int = DQMC_SERVER_CONCURRENT):
        h = c_vp()
        _check(lib().dqmc_server_create(hbm_bytes, streams, mode, ctypes.byref(h)), "dqmc_server_create")
        self.h = h

    def close(self):
        if self.h:
            st = lib().dqmc_server_destroy(self.h)
            self.h = None
            _check(st, "dqmc_server_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, n: int, on_bits, dc_bits=None, flags: int = 0) -> int:
        on = _host_tt(on_bits, n)
        dc = None if dc_bits is None else _host_tt(dc_bits, n)
        job = ctypes.c_uint64()
        _check(lib().dqmc_server_submit(self.h, n, _p8(on), None if dc is None else _p8(dc), flags,
                                        ctypes.byref(job)), "dqmc_server_submit")
        return job.value

    def wait(self, job: int, timeout_ms: int = 600000) -> None:
        _check(lib().dqmc_server_wait(self.h, job, timeout_ms), "dqmc_server_wait")

    def query(self, job: int):
        state, cnt, ptr = ctypes.c_int(), ctypes.c_uint64(), c_vp()
        ts, td = ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().dqmc_server_query(self.h, job, ctypes.byref(state), ctypes.byref(cnt), ctypes.byref(ptr),
                                       ctypes.byref(ts), ctypes.byref(td)), "dqmc_server_query")
        return {"state": state.value, "count": cnt.value, "d_bitmap": ptr.value, "t_submit_ns": ts.value,
                "t_done_ns": td.value}

    def bitmap(self, job: int, n: int) -> np.ndarray:
        out = np.zeros(dqmc_bitmap_bytes(n), dtype=np.uint8)
        _check(lib().dqmc_server_copy_bitmap(self.h, job, _p8(out), out.size), "dqmc_server_copy_bitmap")
        return out

    def free(self, job: int) -> None:
        _check(lib().dqmc_server_free_job(self.h, job), "dqmc_server_free_job")

    def stats(self) -> dict:
        out = (ctypes.c_uint64 * 8)()
        _check(lib().dqmc_server_stats(self.h, ctypes.cast(out, c_u64p)), "dqmc_server_stats")
        keys = ("submitted", "done", "batches", "batched_jobs", "bytes_in_use", "peak_bytes", "peak_running",
                "budget")
        return dict(zip(keys, (int(v) for v in out)))

    def replay(self, t_arrive, ns, on_list, dc_list=None):
        """Submit job j at t_arrive[j] s (ascending) after the call starts, wait
        for all; returns (counts, latencies_s, span_s)."""
        m = len(ns)
        t = np.ascontiguousarray(t_arrive, dtype=np.float64)
        n_a = np.ascontiguousarray(ns, dtype=np.uint32)
        keep = [_host_tt(on_list[j], int(n_a[j])) for j in range(m)]
        on_ptrs = (c_vp * m)(*[k.ctypes.data for k in keep])
        dc_ptrs = None
        if dc_list is not None:
            dkeep = [None if d is None else _host_tt(d, int(n_a[j])) for j, d in enumerate(dc_list)]
            keep += [d for d in dkeep if d is not None]
            dc_ptrs = (c_vp * m)(*[None if d is None else d.ctypes.data for d in dkeep])
        counts = np.zeros(m, dtype=np.uint64)
        lat = np.zeros(m, dtype=np.float64)
        span = ctypes.c_double()
        st = lib().dqmc_server_replay(self.h, m, t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      n_a.ctypes.data_as(c_u32p), ctypes.cast(on_ptrs, c_vp),
                                      None if dc_ptrs is None else ctypes.cast(dc_ptrs, c_vp),
                                      counts.ctypes.data_as(c_u64p),
                                      lat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(span))
        _check(st, "dqmc_server_replay")
        return counts, lat, span.value
