"""CPU-only checks of the C ABI library: it loads, exports every symbol the
headers declare, rejects bad arguments without touching the GPU, and its pass
plan is sound (every digit merged once and reduced once, tiles cover the rows
they must, and the grouped schedule gives the oracle's primes when simulated
on the host)."""
import glob
import os
import re

import numpy as np
import pytest

import oracle
from paper_2302_10083_gb300 import dqmc, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(dqmc_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = dqmc.lib()
    names = declared_functions()
    assert "dqmc_primes" in names and "dqmc_list_dev" in names and "dqmc_plan_json" in names
    for name in names:
        assert hasattr(L, name), name


def test_sizes():
    for n in range(0, 26):
        assert dqmc.dqmc_bitmap_bytes(n) == (3 ** n + 7) // 8
        assert dqmc.dqmc_bitmap_alloc_bytes(n) % 16 == 0
        assert dqmc.dqmc_bitmap_alloc_bytes(n) >= dqmc.dqmc_bitmap_bytes(n)
    assert dqmc.dqmc_bitmap_bytes(26) == 0
    assert dqmc.dqmc_workspace_bytes(26) == 0
    # n=24: padded state (3^19 rows of 32 bytes) dominates the workspace
    assert dqmc.dqmc_workspace_bytes(24) >= 3 ** 19 * 32
    assert dqmc.dqmc_workspace_bytes(12) < 1 << 20   # whole function in one tile


def test_strerror():
    for s in (0, -1, -2, -3, -4, -5):
        assert dqmc.strerror(s)
    assert dqmc.strerror(-99) == "unknown status"


def test_bad_arguments_rejected_without_gpu():
    L = dqmc.lib()
    # n too large / NULL truth table: rejected before any CUDA call
    assert L.dqmc_primes(26, None, None, None) == dqmc.DQMC_EINVAL
    assert L.dqmc_primes(5, None, None, None) == dqmc.DQMC_EINVAL
    assert L.dqmc_count(5, None, None, None) == dqmc.DQMC_EINVAL
    assert L.dqmc_primes_dev(26, 256, None, 256, None, 256, 1 << 30, None) == dqmc.DQMC_EINVAL
    # workspace too small / misaligned
    assert L.dqmc_primes_dev(20, 256, None, 256, None, 256, 16, None) == dqmc.DQMC_EINVAL
    assert L.dqmc_primes_dev(20, 256, None, 256, None, 257, 1 << 40, None) == dqmc.DQMC_EINVAL
    # misaligned truth table for n >= 5
    assert L.dqmc_primes_dev(8, 258, None, 256, None, 256, 1 << 20, None) == dqmc.DQMC_EINVAL
    # list without a count pointer, compaction without a bitmap
    assert L.dqmc_list_dev(8, 256, None, 256, None, 0, None, 256, 1 << 20, None) == dqmc.DQMC_EINVAL
    assert L.dqmc_compact_dev(8, None, None, 0, 256, 256, 1 << 20, None) == dqmc.DQMC_EINVAL
    assert L.dqmc_plan_json(26, None, 0) == dqmc.DQMC_EINVAL


# ------------------------------------------------------------------ plan

def plan(n):
    return dqmc.dqmc_plan_json(n)


@pytest.mark.parametrize("n", list(range(0, 26)))
def test_plan_digit_coverage(n):
    p = plan(n)
    C, H = p["C"], p["H"]
    assert C == min(n, 5) and H == n - C
    merged, reduced, chunk_reduced = [], [], 0
    for q in p["passes"]:
        digits = list(range(q["a"], q["a"] + q["K"]))
        if q["kind"] in ("first", "merge"):
            merged += digits
            if q["fuse_reduce"]:
                reduced += digits
        else:
            reduced += digits
        chunk_reduced += q["chunk_reduce"]
        assert q["K"] + q["B"] <= 7
    assert sorted(merged) == list(range(H))
    assert sorted(reduced) == list(range(H))
    assert chunk_reduced == 1
    # merge groups ascend; the bitmap is written by the last pass only
    assert [q["write_out"] for q in p["passes"]] == [False] * (len(p["passes"]) - 1) + [True]
    assert p["passes"][0]["kind"] == "first"
    if H > 7:
        assert p["state_rows"] == 3 ** H
        out = p["passes"][-1]
        assert out["a"] == 0 and out["B"] == 0  # contiguous rows for the dense write


def spread3(x):
    r, w = 0, 1
    while x:
        if x & 1:
            r += w
        x >>= 1
        w *= 3
    return r


def tile_rows(q, tile, binary_group):
    """Rows a tile touches, with the same formulas as the kernel."""
    RE, K = 3 ** q["B"], q["K"]
    mid = tile % q["n_mid"]
    topi = tile // q["n_mid"]
    top_t = spread3(topi) if q["top_binary"] else topi
    base = mid * RE + top_t * q["w_top"]
    gs = [spread3(b) for b in range(1 << K)] if binary_group else range(3 ** K)
    return [base + e + g * q["w_g"] for g in gs for e in range(RE)]


def row_digits(r, H):
    d = []
    for _ in range(H):
        d.append(r % 3)
        r //= 3
    return d


@pytest.mark.parametrize("n", [13, 14, 16, 17])
def test_plan_tiles_cover_rows(n):
    """Every pass touches exactly the rows it must, each once."""
    p = plan(n)
    H = p["H"]
    done = set()            # digits merged so far
    for q in p["passes"]:
        grp = set(range(q["a"], q["a"] + q["K"]))
        writes = []
        reads = []
        for t in range(q["tiles"]):
            if q["kind"] == "first":
                writes += tile_rows(q, t, False)
            elif q["kind"] == "merge":
                reads += tile_rows(q, t, True)
                writes += tile_rows(q, t, False)
            else:
                reads += tile_rows(q, t, False)
                writes += tile_rows(q, t, False)
        assert len(set(writes)) == len(writes), "tiles overlap"
        assert all(0 <= r < 3 ** H for r in writes)
        if q["kind"] in ("first", "merge"):
            after = done | grp
            # written rows: merged digits any value, the rest binary
            want = [r for r in range(3 ** H)
                    if all(dg != 2 or j in after for j, dg in enumerate(row_digits(r, H)))]
            assert sorted(writes) == want
            if q["kind"] == "merge":
                # read rows: group digits and unmerged digits binary, all previously written
                want_r = [r for r in range(3 ** H)
                          if all(dg != 2 or j in done for j, dg in enumerate(row_digits(r, H)))]
                assert sorted(reads) == want_r
            done = after
        else:
            assert sorted(writes) == list(range(3 ** H))


def grouped_reduce(S, n, digits):
    """Reduce over a set of digits, every read taken from the state as it was before."""
    A = S.reshape((3,) * n) if n else S
    clear = np.zeros_like(A)
    for j in digits:
        ax = n - 1 - j
        star = np.take(A, [2], axis=ax)
        for v in (0, 1):
            idx = [slice(None)] * n
            idx[ax] = slice(v, v + 1)
            clear[tuple(idx)] |= star
    return (A & ~clear).reshape(-1)


def merge_digit(S, n, j):
    A = S.reshape((3,) * n).copy()
    ax = n - 1 - j
    s0 = np.take(A, [0], axis=ax)
    s1 = np.take(A, [1], axis=ax)
    idx = [slice(None)] * n
    idx[ax] = slice(2, 3)
    A[tuple(idx)] |= s0 & s1
    return A.reshape(-1)


@pytest.mark.parametrize("n,seed", [(8, 1), (13, 2), (14, 3), (15, 4)])
def test_plan_schedule_simulated(n, seed):
    """Run the plan's digit schedule on the host (Merge per digit, Reduce grouped
    per pass from the pass's starting state) and compare with the oracle."""
    on, dc = synth.random_function(n, seed, 0.75, 0.1)
    p = plan(n)
    C = p["C"]
    sup = np.unpackbits(on, bitorder="little")[: 1 << n].astype(bool) | \
        np.unpackbits(dc, bitorder="little")[: 1 << n].astype(bool)
    S = np.zeros(3 ** n, dtype=bool)
    t = np.arange(1 << n)
    rho = np.zeros_like(t)
    for i in range(n):
        rho += ((t >> i) & 1) * 3 ** i
    S[rho] = sup
    chunk_digits = list(range(C))
    for q in p["passes"]:
        grp = [C + d for d in range(q["a"], q["a"] + q["K"])]
        if q["kind"] in ("first", "merge"):
            digits = (chunk_digits if q["kind"] == "first" else []) + grp
            for j in digits:
                S = merge_digit(S, n, j)
            if q["fuse_reduce"]:
                S = grouped_reduce(S, n, grp + (chunk_digits if q["chunk_reduce"] else []))
        else:
            S = grouped_reduce(S, n, grp + (chunk_digits if q["chunk_reduce"] else []))
    want = oracle.sweep(n, on, dc) != 0
    assert np.array_equal(S, want)


@pytest.mark.parametrize("n", list(range(13, 26)))
def test_plan_rows_in_bounds(n):
    """The highest row any tile of any pass touches is below 3^H (same index
    formulas as the kernel, evaluated at the last tile, the largest group index
    and the largest inner index); tile counts fit a 1-D grid."""
    p = plan(n)
    H = p["H"]
    for q in p["passes"]:
        assert 0 < q["tiles"] < 2 ** 31
        last = q["tiles"] - 1
        mid = last % q["n_mid"]
        topi = last // q["n_mid"]
        top_t = spread3(topi) if q["top_binary"] else topi
        base = mid * 3 ** q["B"] + top_t * q["w_top"]
        g_max = 3 ** q["K"] - 1
        row_max = base + (3 ** q["B"] - 1) + g_max * q["w_g"]
        assert row_max < 3 ** H
        if q["kind"] == "first" and H > 7:
            # truth-table words read: topi * 2^K + gb < 2^H
            assert (topi + 1) * 2 ** q["K"] <= 2 ** H
        if q["write_out"]:
            # the bitmap pass covers rows 0 .. 3^H-1 contiguously
            assert q["a"] == 0 and q["B"] == 0 and q["tiles"] * 3 ** q["K"] == 3 ** H
