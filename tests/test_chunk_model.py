"""Host model of the register arithmetic on one 256-bit row (no GPU).

A row holds the 3^5 = 243 cells of the five low ("chunk") digits, cell q at bit
q % 32 of word q // 32 (Section 4.2's idea of a block of h digits; here h = 5
and the block is one 32-byte sector).  The kernels merge those digits while
spreading a row's 32 truth-table bits, and reduce them later with funnel
shifts and constant masks; with no wildcard anywhere above, the row is an
n = 5 function on its own, so the result must be the oracle's (Algorithm 3,
Section 4.1) for that function.

The model repeats the kernels' steps: word w of v << S and v >> S built from
two neighbouring words with a funnel shift, the digit masks from their
definition (digit i of q equals v), the Merge of digit i as
v |= (v << 3^i) & (v << 2*3^i) & (digit i is '*'), and the Reduce of a set of
digits as one snapshot: acc collects (y >> 3^i) | (y >> 2*3^i) with y the '*'
cells of digit i, then v &= ~acc.  The plan reduces chunk digits {0, 1, 2} in
one pass and {3, 4} in a later one; both splits are checked.
"""
import numpy as np
import pytest

import oracle

M32 = 0xFFFFFFFF
WORDS = 8
C = 5


def funnel_l(lo, hi, sh):
    return ((((hi << 32) | lo) << sh) >> 32) & M32


def funnel_r(lo, hi, sh):
    return ((((hi << 32) | lo) >> sh)) & M32


def shl_word(v, S, w):
    """Word w of (v << S) over eight words, as the kernels build it."""
    ws, bs = S >> 5, S & 31
    src = w - ws
    hi = v[src] if src >= 0 else 0
    if bs == 0:
        return hi
    lo = v[src - 1] if src - 1 >= 0 else 0
    return funnel_l(lo, hi, bs)


def shr_word(v, S, w):
    ws, bs = S >> 5, S & 31
    src = w + ws
    lo = v[src] if src < WORDS else 0
    if bs == 0:
        return lo
    hi = v[src + 1] if src + 1 < WORDS else 0
    return funnel_r(lo, hi, bs)


def digit(q, i):
    return (q // 3 ** i) % 3


def mask(i, val):
    m = [0] * WORDS
    for q in range(3 ** C):
        if digit(q, i) == val:
            m[q >> 5] |= 1 << (q & 31)
    return m


STAR = [mask(i, 2) for i in range(C)]


def spread_pos(t):
    return sum(3 ** i for i in range(C) if (t >> i) & 1)


def from_minterms(x):
    """The 32 truth-table bits of a row spread to their binary cells, then
    chunk digits 0..4 merged in order."""
    v = [0] * WORDS
    for t in range(32):
        q = spread_pos(t)
        v[q >> 5] |= ((x >> t) & 1) << (q & 31)
    for i in range(C):
        d = 3 ** i
        v = [v[w] | (shl_word(v, d, w) & shl_word(v, 2 * d, w) & STAR[i][w]) for w in range(WORDS)]
    return v


def reduce_digits(v, digits):
    acc = [0] * WORDS
    for i in digits:
        d = 3 ** i
        y = [v[w] & STAR[i][w] for w in range(WORDS)]
        for w in range(WORDS):
            acc[w] |= shr_word(y, d, w) | shr_word(y, 2 * d, w)
    return [v[w] & ~acc[w] & M32 for w in range(WORDS)]


def as_int(v):
    return sum(x << (32 * w) for w, x in enumerate(v))


def from_int(z):
    return [(z >> (32 * w)) & M32 for w in range(WORDS)]


def test_word_shifts_equal_wide_shifts():
    rng = np.random.default_rng(1)
    for _ in range(200):
        z = int(rng.integers(0, 1 << 62)) | (int(rng.integers(0, 1 << 62)) << 62) | \
            (int(rng.integers(0, 1 << 62)) << 124) | (int(rng.integers(0, 1 << 62)) << 186)
        z &= (1 << 256) - 1
        v = from_int(z)
        for S in (1, 2, 3, 6, 9, 18, 27, 32, 54, 64, 81, 162, 200):
            assert [shl_word(v, S, w) for w in range(WORDS)] == from_int((z << S) & ((1 << 256) - 1))
            assert [shr_word(v, S, w) for w in range(WORDS)] == from_int(z >> S)


def test_masks_partition_the_cells():
    """For each digit the three masks split cells 0 .. 242; bits 243.. are in none."""
    cells = (1 << 243) - 1
    for i in range(C):
        a, b, s = as_int(mask(i, 0)), as_int(mask(i, 1)), as_int(mask(i, 2))
        assert a & b == 0 and a & s == 0 and b & s == 0
        assert a | b | s == cells


def oracle_row(x):
    S = oracle.sweep(C, np.array([x & 0xFF, (x >> 8) & 0xFF, (x >> 16) & 0xFF, x >> 24], dtype=np.uint8))
    return sum(1 << int(q) for q in np.nonzero(S)[0])


def sample_functions():
    rng = np.random.default_rng(7)
    fixed = [0, M32, 0x96696996, 0xFFFEFFFF, 0x00010000, 0xE8808000, 0x7FFFFFFF, 0xAAAAAAAA]
    return fixed + [int(v) for v in rng.integers(0, 1 << 32, 600, dtype=np.uint64)] + \
        [int(v) | int(w) for v, w in zip(rng.integers(0, 1 << 32, 300, dtype=np.uint64),
                                         rng.integers(0, 1 << 32, 300, dtype=np.uint64))]


@pytest.mark.parametrize("groups", [[range(5)], [range(3), range(3, 5)], [[0], [1, 2, 3, 4]], [[4], [3], [2], [1], [0]]])
def test_row_merge_and_grouped_reduce_equal_oracle(groups):
    for x in sample_functions():
        v = from_minterms(x)
        for g in groups:
            v = reduce_digits(v, g)
        assert as_int(v) == oracle_row(x), hex(x)


def test_merged_row_is_the_implicant_set():
    """After the Merge alone, cell q is set iff every minterm it covers is on."""
    for x in sample_functions()[:200]:
        v = as_int(from_minterms(x))
        for q in range(3 ** C):
            ds = [digit(q, i) for i in range(C)]
            stars = [i for i in range(C) if ds[i] == 2]
            base = sum(1 << i for i in range(C) if ds[i] == 1)
            imp = all((x >> (base | sum(1 << stars[k] for k in range(len(stars)) if (a >> k) & 1))) & 1
                      for a in range(1 << len(stars)))
            assert ((v >> q) & 1) == int(imp), (hex(x), q)
