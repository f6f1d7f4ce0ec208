"""Seeded synthetic truth tables: the only code shared by the oracle side and the CUDA side.

Nothing here touches cubes, ternary indexes, Merge or Reduce; it only draws bits.

Random numbers
--------------
Every draw is ``u(seed, stream, x)``, a counter-based 64-bit value built from
SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; the finaliser is the one published with Vigna's
``splitmix64.c``)::

    mix(z)  = SplitMix64 output for state z (increment 0x9E3779B97F4A7C15, then
              the two xor-shift-multiply rounds and a final xor-shift)
    key     = mix(seed XOR (stream * 0x9E3779B97F4A7C15))
    u(x)    = mix(key + x)                      (all arithmetic mod 2^64)

A Bernoulli(p) draw is ``u(x) < floor(p * 2^64)`` (p >= 1 gives 1, p <= 0 gives 0).

Streams: 0 = ON set, 1 = don't-care set (drawn only where ON is 0),
2 = per-function parameters of a batch, 3 = serving arrivals.

Bit packing
-----------
A truth table of an n-variable function is ``ceil(2^n / 8)`` bytes, least
significant bit first: minterm t = sum_i 2^(i-1) x_i sits in byte t >> 3 at bit
t & 7.  Bits at t >= 2^n in the last byte are zero.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_ON = 0
STREAM_DC = 1
STREAM_PARAMS = 2
STREAM_ARRIVALS = 3


def _mix(z):
    """SplitMix64 output function applied to state ``z`` (uint64 scalar or array)."""
    with np.errstate(over="ignore"):
        z = np.asarray(z, dtype=np.uint64) + GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def draws(seed: int, stream: int, x) -> np.ndarray:
    """u(seed, stream, x) for an integer array (or scalar) of counters ``x``."""
    with np.errstate(over="ignore"):
        key = _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
                   ^ (np.uint64(stream) * GOLDEN))
        return _mix(key + np.asarray(x, dtype=np.uint64))


def threshold(p: float) -> int | None:
    """floor(p * 2^64) as a Python int; None means 'always true' (p >= 1)."""
    if p >= 1.0:
        return None
    if p <= 0.0:
        return 0
    return int(p * 2.0 ** 64)


def bernoulli(seed: int, stream: int, count: int, p: float) -> np.ndarray:
    """Bool array of ``count`` Bernoulli(p) draws on counters 0..count-1."""
    thr = threshold(p)
    if thr is None:
        return np.ones(count, dtype=bool)
    if thr == 0:
        return np.zeros(count, dtype=bool)
    u = draws(seed, stream, np.arange(count, dtype=np.uint64))
    return u < np.uint64(thr)


def tt_bytes(n: int) -> int:
    """Bytes of an n-variable truth table: ceil(2^n / 8)."""
    return ((1 << n) + 7) >> 3


def pack(bits: np.ndarray) -> np.ndarray:
    """Pack a bool array (index = minterm) into LSB-first bytes."""
    return np.packbits(np.asarray(bits, dtype=bool), bitorder="little")


def unpack(data, n: int) -> np.ndarray:
    """Inverse of :func:`pack` for an n-variable table (bool array of 2^n)."""
    b = np.frombuffer(bytes(data), dtype=np.uint8) if not isinstance(data, np.ndarray) else data
    return np.unpackbits(b.astype(np.uint8), bitorder="little")[: 1 << n].astype(bool)


def random_function(n: int, seed: int, p_on: float, p_dc: float = 0.0):
    """ON ~ Bernoulli(p_on); DC ~ Bernoulli(p_dc) on the minterms where ON is 0.

    Returns ``(on_bytes, dc_bytes_or_None)`` as uint8 arrays of ceil(2^n/8) bytes.
    """
    m = 1 << n
    on = bernoulli(seed, STREAM_ON, m, p_on)
    if p_dc <= 0.0:
        return pack(on), None
    dc = bernoulli(seed, STREAM_DC, m, p_dc) & ~on
    return pack(on), pack(dc)


# --------------------------------------------------------------------------
# The workloads: one function each at n = 10, 20, 24, a batch of small
# functions and a stream of serving requests.
# --------------------------------------------------------------------------

def single_n10(seed: int = 1):
    """n=10, ON ~ Bernoulli(0.5), no don't-cares."""
    return random_function(10, seed, 0.5)


def single_n20(seed: int = 1):
    """n=20, ON ~ Bernoulli(0.7), DC ~ Bernoulli(0.1) on the OFF minterms."""
    return random_function(20, seed, 0.7, 0.1)


def single_n24(seed: int = 1):
    """n=24, ON ~ Bernoulli(0.85), no don't-cares."""
    return random_function(24, seed, 0.85)


def batch_params(count: int, seed: int, n_lo: int = 4, n_hi: int = 14):
    """Per-function parameters of a batch, drawn on stream 2 with counters 4f..4f+3.

    n = n_lo + u0 mod (n_hi - n_lo + 1); ON density = 0.3 + 0.6 * u1 / 2^64;
    a don't-care set ~ Bernoulli(0.05) iff u2 < 0.1 * 2^64; the function's own
    seed is u3.
    """
    f = np.arange(count, dtype=np.uint64) * np.uint64(4)
    u0 = draws(seed, STREAM_PARAMS, f)
    u1 = draws(seed, STREAM_PARAMS, f + np.uint64(1))
    u2 = draws(seed, STREAM_PARAMS, f + np.uint64(2))
    u3 = draws(seed, STREAM_PARAMS, f + np.uint64(3))
    span = np.uint64(n_hi - n_lo + 1)
    ns = (np.uint64(n_lo) + u0 % span).astype(np.int64)
    dens = 0.3 + 0.6 * (u1.astype(np.float64) / 2.0 ** 64)
    has_dc = u2 < np.uint64(threshold(0.1))
    return ns, dens, has_dc, u3


def batch_functions(count: int = 65536, seed: int = 1, n_lo: int = 4, n_hi: int = 14):
    """The batched workload as an arena.

    Returns a dict with ``n`` (int64[count]), ``tt_off`` (uint64[count], byte
    offsets of each ON table in ``arena``), ``dc_off`` (uint64[count], offset of
    the DC table or 2^64-1 for none) and ``arena`` (uint8).  Every table starts
    on a 16-byte boundary.
    """
    ns, dens, has_dc, fseeds = batch_params(count, seed, n_lo, n_hi)
    parts = []
    tt_off = np.zeros(count, dtype=np.uint64)
    dc_off = np.full(count, np.iinfo(np.uint64).max, dtype=np.uint64)
    pos = 0

    def put(buf):
        nonlocal pos
        off = pos
        size = (len(buf) + 15) & ~15
        pad = np.zeros(size, dtype=np.uint8)
        pad[: len(buf)] = buf
        parts.append(pad)
        pos += size
        return off

    for f in range(count):
        n = int(ns[f])
        on, dc = random_function(n, int(fseeds[f]), float(dens[f]),
                                 0.05 if has_dc[f] else 0.0)
        tt_off[f] = put(on)
        if dc is not None:
            dc_off[f] = put(dc)
    arena = np.concatenate(parts) if parts else np.zeros(0, dtype=np.uint8)
    return {"n": ns, "tt_off": tt_off, "dc_off": dc_off, "arena": arena,
            "density": dens, "has_dc": has_dc}


def serving_requests(count: int, seed: int, rate: float, n_lo: int = 6, n_hi: int = 22):
    """Poisson arrivals at ``rate`` jobs/s; n log-uniform in [n_lo, n_hi]; ON density U[0.2, 0.95].

    Uses stream 3 with counters 4j..4j+3: exponential gap from u0, n =
    floor(exp(U(ln n_lo, ln(n_hi+1)))) clipped to [n_lo, n_hi] from u1,
    density from u2, the job's own seed u3.  Returns arrays ``t_arrive`` (s),
    ``n``, ``density``, ``seed``.
    """
    j = np.arange(count, dtype=np.uint64) * np.uint64(4)
    u0 = draws(seed, STREAM_ARRIVALS, j).astype(np.float64) / 2.0 ** 64
    u1 = draws(seed, STREAM_ARRIVALS, j + np.uint64(1)).astype(np.float64) / 2.0 ** 64
    u2 = draws(seed, STREAM_ARRIVALS, j + np.uint64(2)).astype(np.float64) / 2.0 ** 64
    u3 = draws(seed, STREAM_ARRIVALS, j + np.uint64(3))
    gaps = -np.log1p(-u0) / rate
    t = np.cumsum(gaps)
    lo, hi = np.log(n_lo), np.log(n_hi + 1)
    ns = np.clip(np.floor(np.exp(lo + (hi - lo) * u1)), n_lo, n_hi).astype(np.int64)
    dens = 0.2 + 0.75 * u2
    return {"t_arrive": t, "n": ns, "density": dens, "seed": u3}
