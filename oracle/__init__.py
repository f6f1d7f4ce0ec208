"""CPU oracle for the dense ternary prime-implicant sweep (arXiv 2302.10083).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` may import this package; the CUDA library and its
Python binding never do.  The oracle shares no code with the CUDA path.

The arithmetic is in ``dqmc_oracle.c`` (plain scalar C, OpenMP over the
independent triples of one digit).  This module compiles it with gcc on first
use and wraps it with ctypes:

* :func:`sweep` -- Algorithm 3 (Section 4.1), one byte per cube, returns the
  final state (nonzero = prime implicant).
* :func:`sweep_packed`, :func:`packed_bitmap`, :func:`packed_pairs` -- the
  same passes with one bit per cube, for n whose byte state does not fit in
  host memory, and its outputs.
* :func:`bitmap`, :func:`count`, :func:`pairs` -- the three outputs: dense
  LSB-first bitmap indexed by rho, the number of primes, the (mask, value) list
  in ascending rho.
* :func:`is_implicant`, :func:`is_prime` -- the plain definitions (Section 2),
  one cube at a time.

Pins (tests/test_oracle_pins.py): brute force for n <= 10 and every function of
n <= 3 (n = 4 on request), the 3-bit majority (Section 1), the Merge example
(Section 3), constant 0 and 1, parity, single minterm, OR of all variables,
symmetric, monotone and unate functions in closed form (unate also with
don't-cares), invariants, metamorphic relations, the
triple counts of the Boolean-circuit theorem (Section 4.1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dqmc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libdqmc_oracle.so")
_lock = threading.Lock()
_lib = None

u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP).  Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-Wall",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.oracle_pow3.restype = ctypes.c_uint64
            L.oracle_pow3.argtypes = [ctypes.c_int]
            L.oracle_max_threads.restype = ctypes.c_int
            L.oracle_sweep.restype = None
            L.oracle_sweep.argtypes = [ctypes.c_int, u8p, u8p, u8p, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_uint64)]
            L.oracle_bitmap.restype = None
            L.oracle_bitmap.argtypes = [ctypes.c_int, u8p, u8p]
            L.oracle_count.restype = ctypes.c_uint64
            L.oracle_count.argtypes = [ctypes.c_int, u8p]
            L.oracle_list.restype = ctypes.c_uint64
            L.oracle_list.argtypes = [ctypes.c_int, u8p, ctypes.POINTER(ctypes.c_uint32),
                                      ctypes.c_uint64]
            L.oracle_encode.restype = None
            L.oracle_encode.argtypes = [ctypes.c_int, ctypes.c_uint64,
                                        ctypes.POINTER(ctypes.c_uint32),
                                        ctypes.POINTER(ctypes.c_uint32)]
            L.oracle_is_implicant.restype = ctypes.c_int
            L.oracle_is_implicant.argtypes = [ctypes.c_int, u8p, u8p, ctypes.c_uint64]
            L.oracle_is_prime.restype = ctypes.c_int
            L.oracle_is_prime.argtypes = [ctypes.c_int, u8p, u8p, ctypes.c_uint64]
            L.oracle_sweep_packed.restype = None
            L.oracle_sweep_packed.argtypes = [ctypes.c_int, u8p, u8p, ctypes.POINTER(ctypes.c_uint64),
                                              ctypes.c_int]
            L.oracle_packed_bitmap.restype = None
            L.oracle_packed_bitmap.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), u8p]
            L.oracle_packed_list.restype = ctypes.c_uint64
            L.oracle_packed_list.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_uint64),
                                             ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint64]
            L.oracle_is_prime_many.restype = None
            L.oracle_is_prime_many.argtypes = [ctypes.c_int, u8p, u8p,
                                               ctypes.POINTER(ctypes.c_uint64),
                                               ctypes.c_uint64, u8p, ctypes.c_int]
            _lib = L
    return _lib


def _tt(buf, n):
    """Contiguous uint8 copy of a truth table (at least ceil(2^n/8) bytes)."""
    if buf is None:
        return None
    a = np.ascontiguousarray(np.frombuffer(bytes(buf), dtype=np.uint8)
                             if not isinstance(buf, np.ndarray) else buf, dtype=np.uint8)
    need = ((1 << n) + 7) >> 3
    if a.size < need:
        raise ValueError(f"truth table has {a.size} bytes, needs {need}")
    return a


def _p(a):
    return None if a is None else a.ctypes.data_as(u8p)


def pow3(n: int) -> int:
    return 3 ** n


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def sweep(n: int, on, dc=None, threads: int = 0, return_counts: bool = False):
    """Algorithm 3 on one byte per cube; returns the uint8 state of 3^n bytes."""
    on = _tt(on, n)
    dc = _tt(dc, n)
    S = np.empty(3 ** n, dtype=np.uint8)
    counts = (ctypes.c_uint64 * 2)()
    lib().oracle_sweep(n, _p(on), _p(dc), _p(S), int(threads), counts)
    if return_counts:
        return S, (int(counts[0]), int(counts[1]))
    return S


def sweep_packed(n: int, on, dc=None, threads: int = 0) -> np.ndarray:
    """Algorithm 3 with one bit per cube (ceil(3^n/64) uint64 words, cube rho
    at bit rho % 64 of word rho // 64): the same passes as :func:`sweep` in a
    ninth of the host memory, for the sizes whose byte state does not fit."""
    on = _tt(on, n)
    dc = _tt(dc, n)
    S = np.empty((3 ** n + 63) // 64, dtype=np.uint64)
    lib().oracle_sweep_packed(n, _p(on), _p(dc), S.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                              int(threads))
    return S


def packed_bitmap(n: int, S: np.ndarray) -> np.ndarray:
    """The dense LSB-first bitmap (ceil(3^n/8) bytes) of a packed state."""
    out = np.empty((3 ** n + 7) // 8, dtype=np.uint8)
    lib().oracle_packed_bitmap(n, S.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _p(out))
    return out


def packed_pairs(n: int, S: np.ndarray) -> np.ndarray:
    """(mask, value) uint32 pairs of a packed state in ascending rho, shape (count, 2)."""
    sp = S.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    c = int(lib().oracle_packed_list(n, sp, None, 0))
    out = np.empty(2 * max(c, 1), dtype=np.uint32)
    lib().oracle_packed_list(n, sp, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), c)
    return out[: 2 * c].reshape(c, 2)


def bitmap(n: int, S: np.ndarray) -> np.ndarray:
    out = np.empty((3 ** n + 7) // 8, dtype=np.uint8)
    lib().oracle_bitmap(n, _p(S), _p(out))
    return out


def count(n: int, S: np.ndarray) -> int:
    return int(lib().oracle_count(n, _p(S)))


def pairs(n: int, S: np.ndarray) -> np.ndarray:
    """(mask, value) uint32 pairs in ascending rho, shape (count, 2)."""
    c = count(n, S)
    out = np.empty(2 * max(c, 1), dtype=np.uint32)
    lib().oracle_list(n, _p(S), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), c)
    return out[: 2 * c].reshape(c, 2)


def encode(n: int, rho: int):
    m = ctypes.c_uint32()
    v = ctypes.c_uint32()
    lib().oracle_encode(n, rho, ctypes.byref(m), ctypes.byref(v))
    return int(m.value), int(v.value)


def is_implicant(n: int, on, dc, rho: int) -> bool:
    on = _tt(on, n)
    dc = _tt(dc, n)
    return bool(lib().oracle_is_implicant(n, _p(on), _p(dc), rho))


def is_prime(n: int, on, dc, rho: int) -> bool:
    on = _tt(on, n)
    dc = _tt(dc, n)
    return bool(lib().oracle_is_prime(n, _p(on), _p(dc), rho))


def is_prime_many(n: int, on, dc, rhos, threads: int = 0) -> np.ndarray:
    on = _tt(on, n)
    dc = _tt(dc, n)
    r = np.ascontiguousarray(rhos, dtype=np.uint64)
    out = np.empty(r.size, dtype=np.uint8)
    lib().oracle_is_prime_many(n, _p(on), _p(dc),
                               r.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                               r.size, _p(out), int(threads))
    return out.astype(bool)


def primes_bitmap(n: int, on, dc=None, threads: int = 0) -> np.ndarray:
    """Convenience: sweep then dense bitmap."""
    return bitmap(n, sweep(n, on, dc, threads))
