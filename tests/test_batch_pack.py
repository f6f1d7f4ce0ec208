"""Host model of how the whole-function kernels write a function's bitmap (no GPU).

A function with n <= 14 sits in shared memory as R rows of 243 cells (the five
chunk digits; row r holds cells 243 r .. 243 r + 242 of the dense bitmap,
Section 4.2 order), or as one part of `parts` such ranges when a cluster of
3 or 9 CTAs (or one CTA, a third at a time) holds it.
* Pack: a warp takes 32 rows at a time (32 * 243 bits are exactly 243 words)
  and writes them, shifted to their bit offsets, over the start of the same
  1 KB of shared memory.  Lane l's row starts at bit 243 l; the word it shares
  with the next row is finished by the next lane, which ORs in the tail it
  gets by shuffle; a row whose next row is absent writes its tail itself.
* Store: the part's packed stream, which starts at bit part * R * 243 of the
  bitmap, is shifted to that offset; the words shared with the neighbouring
  parts are merged under a mask; the last part also zeroes the rest of the
  slot.  With one part the packed regions are copied to the bitmap as they are.

The model repeats the arithmetic and compares with placing every bit directly,
for the row counts and splits the kernels use, checking that no lane writes a
word another lane writes and that every packed word is written.
"""
import numpy as np
import pytest

M32 = 0xFFFFFFFF
C3 = 243


def funnel_l(lo, hi, sh):
    return ((((hi << 32) | lo) << sh) >> 32) & M32


def row_words(bits):
    w = [0] * 8
    for c in np.nonzero(bits)[0]:
        w[c >> 5] |= 1 << (c & 31)
    return w


def pack(rows):
    """The packed words of R rows, as {region g: {word k: value}} (k < 256)."""
    R = len(rows)
    regions = {}
    for g in range((R + 31) // 32):
        o_all, tail = {}, {}
        for lane in range(32):
            r = 32 * g + lane
            v = rows[r] if r < R else [0] * 8
            sh, w0 = (C3 * lane) & 31, (C3 * lane) >> 5
            k8 = sh + C3 > 256
            o = [funnel_l(0, v[0], sh)] + [funnel_l(v[k - 1], v[k], sh) for k in range(1, 8)] + \
                [funnel_l(v[7], 0, sh)]
            tail[lane] = o[8] if k8 else o[7]
            o_all[lane] = (o, sh, w0, k8)
        words, owner = {}, {}
        for lane in range(32):
            r = 32 * g + lane
            o, sh, w0, k8 = o_all[lane]
            if lane > 0 and sh != 0:
                o[0] |= tail[lane - 1]                 # shuffle from the previous lane
            if r >= R:
                continue
            shares = ((sh + C3) & 31) != 0
            own_last = (not shares) or lane == 31 or r + 1 >= R
            put = list(range(7)) + ([7] if (k8 or own_last) else []) + ([8] if (k8 and own_last) else [])
            for k in put:
                assert w0 + k not in owner, f"region {g} word {w0 + k}: lanes {owner[w0 + k]} and {lane}"
                owner[w0 + k] = lane
                words[w0 + k] = o[k]
        regions[g] = words
    NP = (R * C3 + 31) // 32
    for j in range(NP):
        assert j % C3 in regions[j // C3], f"packed word {j} never written"
    return regions


def stream_out(glob, regions, R, part, parts, out_words, alloc_words):
    NP = (R * C3 + 31) // 32

    def packed(j):
        if j < 0 or j >= NP:
            return 0
        return regions[j // C3][j % C3]

    bit0 = part * R * C3
    o, W0 = bit0 & 31, bit0 >> 5
    L = R * C3
    nw = (o + L + 31) >> 5
    last = part == parts - 1
    tail = (o + L) & 31
    for i in range(nw):
        val = funnel_l(packed(i - 1), packed(i), o) if o else packed(i)
        shared_prev = i == 0 and o != 0
        shared_next = i == nw - 1 and not last and tail != 0
        if not shared_prev and not shared_next:
            glob[W0 + i] = val
        else:
            m = M32
            if shared_prev:
                m &= (M32 << o) & M32
            if shared_next:
                m &= (1 << tail) - 1
            glob[W0 + i] = (glob[W0 + i] & (val | ~m)) | (val & m)
    if last:
        for w in range(out_words, alloc_words):
            glob[w] = 0


@pytest.mark.parametrize("n,parts,first_direct", [(5, 1, False), (6, 1, False), (8, 1, False), (10, 1, False),
                                                  (11, 1, False), (13, 1, False), (13, 3, False), (14, 3, False),
                                                  (14, 9, False), (14, 3, True)])
def test_function_bitmap_written_exactly(n, parts, first_direct):
    """first_direct: one CTA doing the thirds in turn writes third 0 as a
    stream that starts at bit 0 (whole words, its last one with the upper bits
    0), before the masked stores of thirds 1 and 2."""
    rng = np.random.default_rng(n * 10 + parts)
    total_rows = 3 ** (n - 5)
    R = total_rows // parts
    cells = rng.random(total_rows * C3) < 0.4
    out_words = (3 ** n + 31) // 32
    alloc_words = ((3 ** n + 7) // 8 + 15) // 16 * 4     # the slot: bitmap bytes rounded to 16
    glob = [int(x) for x in rng.integers(0, 1 << 32, alloc_words, dtype=np.uint64)]
    for part in range(parts):
        rows = [row_words(cells[(part * R + r) * C3:(part * R + r + 1) * C3]) for r in range(R)]
        regions = pack(rows)
        if parts == 1 or (first_direct and part == 0):   # DIRECT: packed regions straight to the bitmap
            NP = (R * C3 + 31) // 32
            for j in range(NP):
                glob[j] = regions[j // C3][j % C3]
            if parts == 1:
                for w in range(out_words, alloc_words):
                    glob[w] = 0
        else:
            stream_out(glob, regions, R, part, parts, out_words, alloc_words)
    want = np.packbits(cells, bitorder="little")
    want = np.concatenate([want, np.zeros(4 * alloc_words - want.size, dtype=np.uint8)])
    got = np.array(glob, dtype=np.uint32).view(np.uint8)
    assert np.array_equal(got, want)
