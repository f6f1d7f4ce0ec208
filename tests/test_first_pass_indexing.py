"""Host check of the first pass's indexing (no GPU).

The first pass reads the truth table in 32-bit words: word w holds minterms
32 w .. 32 w + 31, whose five low variables are the chunk digits and whose
other bits are the high digits, all 0/1 (Section 4.2 embeds the minterms as
the binary cubes).  A tile fixes the high digits 7 .. n-6 (radix 2: none is
merged yet) and takes the 128 words gb of high digits 0..6; word ttb + gb
goes to row base + sp3(gb) (sp3 spreads the bits of gb to base-3 digits), its
bit b to cell spread(b) of that row.  This must put minterm t at
rho(t) = row * 243 + cell, and visit every word once.  The tile's fixed digits
come from the library's plan.
"""
import numpy as np
import pytest

from paper_2302_10083_gb300 import dqmc

C = 5
TILE_DIGITS = 7


def spread(x, k):
    return sum(3 ** i for i in range(k) if (x >> i) & 1)


def rho_of_minterm(n, t):
    return spread(t, n)


def decode(fixed, t):
    base = ttb = 0
    for j, radix in fixed:
        d = t & 1 if radix == 2 else t % 3
        t = t >> 1 if radix == 2 else t // 3
        base += d * 3 ** j
        ttb += d * 2 ** j
    return base, ttb


@pytest.mark.parametrize("n", [13, 15, 18, 21, 24, 25])
def test_words_to_rows_and_cells(n):
    first = dqmc.dqmc_plan_json(n)["passes"][0]
    ph = first["phases"][0]
    assert ph["load"] == "tt" and ph["K"] == TILE_DIGITS and ph["B"] == 0
    fixed = first["sb"]
    assert [j for j, _ in fixed] == list(range(TILE_DIGITS, n - C)) and all(r == 2 for _, r in fixed)
    tiles = first["n_sb"]
    assert tiles == 2 ** (n - C - TILE_DIGITS)
    rng = np.random.default_rng(n)
    seen = set()
    picks = range(tiles) if tiles <= 64 else sorted({0, tiles - 1} | {int(x) for x in rng.integers(0, tiles, 40)})
    for tile in picks:
        base, ttb = decode(fixed, tile)
        for gb in range(1 << TILE_DIGITS):
            w = ttb + gb
            assert w not in seen and w < 2 ** (n - C)
            seen.add(w)
            row = base + spread(gb, TILE_DIGITS)
            for b in (0, 1, 17, 31) if n > 15 else range(32):
                t = 32 * w + b
                assert row * 243 + spread(b, C) == rho_of_minterm(n, t), (n, tile, gb, b)
    if tiles <= 64:
        assert seen == set(range(2 ** (n - C)))
