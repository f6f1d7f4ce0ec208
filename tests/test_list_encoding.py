"""Host model of how the bitmap pass encodes a listed prime (no GPU).

A prime s is listed as (mask, value): mask bit i-1 set iff s_i is 0 or 1,
value bit i-1 = s_i there (the cube's literals, Section 2).  The bitmap pass
builds the pair from three parts instead of decoding rho digit by digit:
* the digits fixed per tile (high digits 7 .. n-6), taken from the tile's
  index with the plan's radices in ascending digit order, as literal and value
  bits at their variable positions;
* the tile's unit u (tile digits 1..6) from a table of u's base-3 digits, and
  the row k in the unit (tile digit 0);
* the chunk cell q (the five low digits) from a table of q's base-3 digits;
and masks both words with 2^n - 1.

The model takes the plan from the library (the same table the kernels get),
repeats those steps, and checks every sampled cell against the oracle's
encoding of rho, for tiles at the start, middle and end of the bitmap.
"""
import numpy as np
import pytest

import oracle
from paper_2302_10083_gb300 import dqmc

C = 5
TILE_DIGITS = 7


def base3_code(x, digits):
    """bit d: digit d of x is 0/1; bit 8+d: it is 1."""
    m = v = 0
    for d in range(digits):
        dg = x % 3
        x //= 3
        if dg != 2:
            m |= 1 << d
        if dg == 1:
            v |= 1 << d
    return m | (v << 8)


CODE = [base3_code(u, 6) for u in range(729)]
C5 = [base3_code(q, 5) for q in range(243)]


def decode_tile(fixed, t):
    """Tile index -> (first row, literal bits, value bits) of its fixed digits."""
    base = m = v = 0
    for j, radix in fixed:
        d = t & 1 if radix == 2 else t % 3
        t = t >> 1 if radix == 2 else t // 3
        base += d * 3 ** j
        if d != 2:
            m |= 1 << (C + j)
        if d == 1:
            v |= 1 << (C + j)
    return base, m, v


def encode_cell(n, tile_m, tile_v, u, k, q):
    code = CODE[u]
    um = tile_m | ((code & 0x3F) << (C + 1))
    uv = tile_v | (((code >> 8) & 0x3F) << (C + 1))
    rm = um | ((1 << C) if k != 2 else 0)
    rv = uv | ((1 << C) if k == 1 else 0)
    c5 = C5[q]
    nmask = (1 << n) - 1
    return (rm | (c5 & 0x1F)) & nmask, (rv | (c5 >> 8)) & nmask


@pytest.mark.parametrize("n", [13, 16, 20, 24, 25])
def test_pairs_match_oracle_encoding(n):
    plan = dqmc.dqmc_plan_json(n)
    out = plan["passes"][-1]
    assert out["phases"][0]["out"] == 1 and out["phases"][0]["K"] == TILE_DIGITS
    fixed = out["sb"]
    assert [j for j, _ in fixed] == list(range(TILE_DIGITS, n - C))
    assert all(r == 3 for _, r in fixed)    # every digit merged before the bitmap pass
    tiles = out["n_sb"]
    assert tiles == plan["out_tiles"] == 3 ** (n - C - TILE_DIGITS)
    rng = np.random.default_rng(n)
    picks = sorted({0, 1, tiles // 2, tiles - 1} | {int(x) for x in rng.integers(0, tiles, 3)})
    for t in picks:
        base, tm, tv = decode_tile(fixed, t)
        assert base == t * 3 ** TILE_DIGITS     # tiles in rho order, contiguous rows
        rows = rng.integers(0, 3 ** TILE_DIGITS, 300)
        cells = rng.integers(0, 243, 300)
        for r, q in zip(rows.tolist() + [0, 2186], cells.tolist() + [0, 242]):
            u, k = divmod(r, 3)
            rho = (base + r) * 243 + q
            assert encode_cell(n, tm, tv, u, k, q) == oracle.encode(n, rho), (n, t, r, q)
