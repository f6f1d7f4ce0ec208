"""Host model of how the bitmap pass writes a tile's dense bits (no GPU).

A tile of 2187 reduced rows (243 cells each, the five chunk digits) is 729
units of three rows; its cells are bits bit0 .. bit0 + 2187 * 243 - 1 of the
dense bitmap (bit rho, Section 4.2 order), and bit0 starts at bit o = bit0 % 32
of word W0.  One warp takes a region of 32 units (the last region has 25):
lane L places unit U0 + L's three rows, at bit o + 729 L of the region's
staging words, as nine funnel-shifted words per row, carrying a row's last
partial word into the next row and a unit's last partial word to the next lane
by shuffle.  Then the staged words go to the bitmap: words wholly inside the
region are stored, the two it shares with the regions before and after it are
merged under a mask (an AND then an OR, so that concurrent merges of the other
bits of the word stay intact), and the last tile also writes the bits past 3^n
as zeros.

The model repeats that arithmetic step by step and checks it against placing
every bit directly, for every bit offset o, full and partial regions, and the
last tile: every bit lands once, no lane writes a staging word another lane
writes, every word read was written, and bits of other tiles stay untouched.
"""
import numpy as np
import pytest

M32 = 0xFFFFFFFF
ROW_BITS = 243
UNIT_BITS = 3 * ROW_BITS            # 729
TILE_UNITS = 729
REGIONS = [(32 * r, min(32, TILE_UNITS - 32 * r)) for r in range((TILE_UNITS + 31) // 32)]


def funnel_l(lo, hi, sh):
    """__funnelshift_l: the high 32 bits of the 64-bit (hi:lo) shifted left by sh (0..31)."""
    return ((((hi << 32) | lo) << sh) >> 32) & M32


def row_words(bits):
    """243 cells -> 8 words, cell c at bit c % 32 of word c // 32 (the padding bits 0)."""
    w = [0] * 8
    for c in np.nonzero(bits)[0]:
        w[c >> 5] |= 1 << (c & 31)
    return w


def stage_region(unit_rows, o, nun):
    """The warp's staging words {index: value} for units 0 .. nun-1 of a region."""
    stg, owner = {}, {}

    def put(lane, i, v):
        assert i not in owner or owner[i] == lane, f"word {i} written by lanes {owner[i]} and {lane}"
        owner[i] = lane
        stg[i] = v

    carry, first, base = [0] * 32, [0] * 32, [0] * 32
    for lane in range(nun):
        lb0 = o + UNIT_BITS * lane
        s0 = lb0 & 31
        base[lane] = lb0 >> 5
        c = 0
        for k in range(3):
            x = unit_rows[lane][k]
            sb = s0 + ROW_BITS * k           # row k's first bit, from the lane's first word
            sh = sb & 31
            rw = base[lane] + (sb >> 5)
            w9 = [((x[0] << sh) & M32) | c] + [funnel_l(x[j - 1], x[j], sh) for j in range(1, 8)] \
                + [funnel_l(x[7], 0, sh)]
            nine = sh >= 13                  # the row fills word 7 (and may reach word 8)
            if k == 0:
                first[lane] = w9[0]
            else:
                put(lane, rw, w9[0])
            for j in range(1, 7):
                put(lane, rw + j, w9[j])
            if nine:
                put(lane, rw + 7, w9[7])
            c = w9[8] if nine else w9[7]
        carry[lane] = c
    for lane in range(nun):                   # after the shuffle of the carries
        cin = carry[lane - 1] if lane > 0 else 0
        put(lane, base[lane], first[lane] | cin)
        if lane == nun - 1:
            s0 = (o + UNIT_BITS * lane) & 31
            put(lane, base[lane] + ((s0 + UNIT_BITS) >> 5), carry[lane])
    return stg


def masked(dst, val, m):
    dst &= (val | ~m) & M32                   # atomicAnd
    dst |= val & m                            # atomicOr
    return dst


def store_region(glob, stg, o, nun, S0, last_word):
    """The region's staged words into the bitmap words glob (a dict)."""
    hi_bit = o + UNIT_BITS * nun
    if nun == 32:
        for j in range(1, 729):
            glob[S0 + j] = stg[j]
        if o == 0:
            glob[S0] = stg[0]
        else:
            glob[S0] = masked(glob[S0], stg[0], (M32 << o) & M32)
            glob[S0 + 729] = masked(glob[S0 + 729], stg[729], (1 << o) - 1)
        return
    nw = (hi_bit + 31) >> 5
    for j in range(nw):
        lo = o if j == 0 else 0
        hi = min(hi_bit - 32 * j, 32)
        hi2 = 32 if S0 + j == last_word else hi    # bits past 3^n are written as 0
        if hi2 <= lo:
            continue
        val = stg[j]
        if lo == 0 and hi2 == 32:
            glob[S0 + j] = val
        else:
            m = (M32 if hi2 == 32 else (1 << hi2) - 1) & ((M32 << lo) & M32)
            glob[S0 + j] = masked(glob[S0 + j], val, m)


def run_tile(cells, o, last_tile, rng):
    """Place a tile's cells (bool, 2187*243) at bit offset o; returns (got, want) word arrays."""
    W0 = 5
    nbits = TILE_UNITS * UNIT_BITS
    nwords = W0 + (o + nbits + 31) // 32 + 3
    fill = [int(v) for v in rng.integers(0, 1 << 32, nwords, dtype=np.uint64)]
    want = list(fill)
    for b in range(nbits):                    # direct placement
        g = 32 * W0 + o + b
        want[g >> 5] = (want[g >> 5] & ~(1 << (g & 31))) | (int(cells[b]) << (g & 31))
    last_word = W0 + (o + nbits - 1) // 32 if last_tile else -1
    if last_tile:                             # bits past 3^n in the last word are 0
        end = 32 * W0 + o + nbits
        want[last_word] &= (1 << (end & 31)) - 1 if end & 31 else M32
    glob = dict(enumerate(fill))
    for U0, nun in REGIONS:
        unit_rows = []
        for lane in range(nun):
            u = U0 + lane
            unit_rows.append([row_words(cells[(3 * u + k) * ROW_BITS:(3 * u + k + 1) * ROW_BITS])
                              for k in range(3)])
        stg = stage_region(unit_rows, o, nun)
        top = (o + UNIT_BITS * nun - 1) >> 5
        assert all(j in stg for j in range(top + 1)), "a staged word that is read was never written"
        store_region(glob, stg, o, nun, W0 + UNIT_BITS * (U0 >> 5), last_word)
    return [glob[i] for i in range(nwords)], want


@pytest.mark.parametrize("o", list(range(32)))
def test_tile_bits_placed_exactly(o):
    rng = np.random.default_rng(100 + o)
    cells = rng.random(TILE_UNITS * UNIT_BITS) < 0.3
    got, want = run_tile(cells, o, last_tile=False, rng=rng)
    assert got == want


@pytest.mark.parametrize("o", [0, 1, 13, 19, 31])
def test_last_tile_zero_tail(o):
    rng = np.random.default_rng(200 + o)
    cells = rng.random(TILE_UNITS * UNIT_BITS) < 0.9
    got, want = run_tile(cells, o, last_tile=True, rng=rng)
    assert got == want


def test_tile_offsets_reachable():
    """Tile t starts at bit 2187 * 243 * t; its offset mod 32 takes all 32 values
    over t = 0 .. 31, so the cases above are the ones the tiles meet."""
    assert sorted({(2187 * 243 * t) % 32 for t in range(32)}) == list(range(32))


def test_staging_fits_region_slots():
    """A region's staged words stay inside its own 16-byte slots (6 per unit):
    the full region's 730 words in 768, the 25-unit tail's in 600."""
    for U0, nun in REGIONS:
        for o in range(32):
            top = (o + UNIT_BITS * nun - 1) >> 5
            extra = 1 if nun == 32 and o else 0
            assert max(top, 728 + extra if nun == 32 else top) < 4 * 6 * nun
