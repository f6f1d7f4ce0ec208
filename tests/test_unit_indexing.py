"""Host check of the sparse Merge pass's unit indexing (no GPU).

A streaming pass's tile holds 7 digits of the row index: B inner digits (the
lowest high digits, contiguous rows) and K = 7 - B group digits a .. a+K-1;
every other high digit is fixed per tile (Algorithm 3's Merge, Section 4.1,
done K digits per pass).  The sparse Merge pass works on units of three rows
(inner digit 0): unit u = eh + RU g with eh < RU = 3^(B-1) the other inner
digits and g < 3^K the group digits, first row base + 3 eh + g 3^a.
* It loads only the units whose group digits are all 0/1: u = eh + RU sp3(gb)
  for gb < 2^K (sp3 spreads bits to base-3 digits).
* Merge of group digit j: one unit per thread, the units whose digit j is '*'
  and whose later group digits are 0/1 (earlier ones any), each the AND of its
  units 2 * 3^j * RU and 3^j * RU below.
* It writes the units with a '*' in some group digit.
The check: the rows of every unit are the rows its digits name, the loaded
units are the binary ones, each Merge step covers its units once (and reads
units with digit j = 0 and 1), and after the K steps every unit is loaded or
computed exactly once.  The (a, K, B) triples come from the library's plans.
"""
import pytest

from paper_2302_10083_gb300 import dqmc

TILE = 7


def spread3(x, k):
    return sum(3 ** i for i in range(k) if (x >> i) & 1)


def digits_of(x, k):
    return [(x // 3 ** i) % 3 for i in range(k)]


def merge_pass_shapes():
    shapes = set()
    for n in (19, 20, 21, 22, 23, 24, 25):
        for p in dqmc.dqmc_plan_json(n)["passes"]:
            ph = p["phases"][0]
            if ph["load"] == "sparse":
                shapes.add((ph["a"], ph["K"], ph["B"]))
    return sorted(shapes)


SHAPES = merge_pass_shapes()


def test_shapes_found():
    assert SHAPES and all(K + B == TILE and B >= 1 for _, K, B in SHAPES)


@pytest.mark.parametrize("a,K,B", SHAPES)
def test_unit_rows_loads_and_merge_items(a, K, B):
    RU = 3 ** (B - 1)
    base = 12345   # any tile base: row offsets are what is checked
    units = 3 ** (TILE - 1)
    assert RU * 3 ** K == units

    def unit_row(u):
        g, eh = divmod(u, RU)
        return base + 3 * eh + g * 3 ** a

    for u in range(units):
        ud = digits_of(u, TILE - 1)               # unit digit d = tile digit d + 1
        inner = [0] + ud[:B - 1]                  # tile digits 0 .. B-1 (digit 0 = row in unit)
        group = ud[B - 1:]
        want = base + sum(d * 3 ** i for i, d in enumerate(inner)) + sum(d * 3 ** (a + i) for i, d in enumerate(group))
        assert unit_row(u) == want

    group_of = lambda u: digits_of(u // RU, K)
    loaded = {eh + RU * spread3(gb, K) for gb in range(1 << K) for eh in range(RU)}
    assert loaded == {u for u in range(units) if 2 not in group_of(u)}

    have = set(loaded)
    for j in range(K):
        Dj = 3 ** j
        items = RU * Dj * (1 << (K - 1 - j))
        assert items <= 384
        made = []
        for tid in range(items):
            eh, rest = tid % RU, tid // RU
            lo, hb = rest % Dj, rest // Dj
            u = eh + RU * (lo + 2 * Dj + 3 * Dj * spread3(hb, K - 1 - j))
            g = group_of(u)
            assert g[j] == 2 and 2 not in g[j + 1:]
            src0, src1 = u - 2 * Dj * RU, u - Dj * RU
            assert group_of(src0)[j] == 0 and group_of(src1)[j] == 1
            assert src0 in have and src1 in have     # both already loaded or merged
            made.append(u)
        assert len(set(made)) == len(made)
        want = {u for u in range(units) if group_of(u)[j] == 2 and 2 not in group_of(u)[j + 1:]}
        assert set(made) == want and not have.intersection(made)
        have.update(made)
    assert have == set(range(units))
    written = {u for u in range(units) if 2 in group_of(u)}
    assert written == set(range(units)) - loaded


def row_pass_shapes():
    shapes = set()
    for n in (13, 16, 19, 21, 24, 25):
        for p in dqmc.dqmc_plan_json(n)["passes"]:
            ph = p["phases"][0]
            if ph["B"] >= 1 and ph["load"] in ("sparse", "full"):
                shapes.add((ph["a"], ph["K"], ph["B"], ph["load"]))
    return sorted(shapes)


@pytest.mark.parametrize("a,K,B,load", row_pass_shapes())
def test_row_pass_rows_and_loads(a, K, B, load):
    """The Merge + Reduce and Reduce passes hold the tile row-major: tile row
    e + 3^B g (e: inner digits, g: group digits) is state row base + e + g 3^a,
    so the tile's base-3 digits are the inner digits, then the group digits, as
    the block steps assume.  The sparse load takes the rows with 0/1 group
    digits, each once."""
    RE = 3 ** B
    base = 777
    seen = set()
    for ri in range(3 ** TILE):
        g, e = divmod(ri, RE)
        row = base + e + g * 3 ** a
        d = digits_of(ri, TILE)
        assert row == base + sum(x * 3 ** i for i, x in enumerate(d[:B])) + \
            sum(x * 3 ** (a + i) for i, x in enumerate(d[B:]))
        assert row not in seen
        seen.add(row)
    if load == "sparse":
        rows = [e + RE * spread3(gb, K) for gb in range(1 << K) for e in range(RE)]
        assert len(set(rows)) == len(rows)
        assert set(rows) == {ri for ri in range(3 ** TILE) if 2 not in digits_of(ri, TILE)[B:]}
