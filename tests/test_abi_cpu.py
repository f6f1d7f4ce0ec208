"""CPU-only checks of the C ABI library: it loads, exports every symbol the
headers declare, rejects bad arguments without touching the GPU, and its pass
plan is sound (every digit merged once and reduced once, tiles cover the rows
they must, and the grouped schedule gives the oracle's primes when simulated
on the host)."""
import ctypes
import glob
import json
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
    # the static-workspace sweep takes n <= 15 only: larger n is refused before any CUDA call
    assert L.dqmc_primes_dev_static(16, 256, None, 256, None, None) == dqmc.DQMC_EINVAL
    assert L.dqmc_primes_dev_static(26, 256, None, 256, None, None) == dqmc.DQMC_EINVAL
    assert L.dqmc_dev_status_static(16, None) == dqmc.DQMC_EINVAL
    # unknown flags of the *_ex entry points are refused before any CUDA call
    on = np.zeros(16, dtype=np.uint8)
    assert L.dqmc_primes_ex(4, on.ctypes.data_as(dqmc.c_u8p), None, 2, None, None) == dqmc.DQMC_EINVAL
    assert L.dqmc_list_ex(4, on.ctypes.data_as(dqmc.c_u8p), None, 6, None, 0, None) == dqmc.DQMC_EINVAL
    assert L.dqmc_primes_dev_ex(14, 256, None, 2, 256, None, 256, 1 << 30, None) == dqmc.DQMC_EINVAL


def test_batch_arguments_rejected_without_gpu():
    L = dqmc.lib()
    n = np.array([4, 14], dtype=np.uint32)
    off = np.array([0, 16], dtype=np.uint64)
    n_p = n.ctypes.data_as(dqmc.c_u32p)
    o_p = off.ctypes.data_as(dqmc.c_u64p)
    assert L.dqmc_batch_run(0, None, None, None, None, None, None, None, None) == dqmc.DQMC_OK
    assert L.dqmc_batch_run(2, None, o_p, 256, None, 256, 256, o_p, None) == dqmc.DQMC_EINVAL
    assert L.dqmc_batch_run(2, n_p, o_p, None, None, 256, 256, o_p, None) == dqmc.DQMC_EINVAL
    too_big = np.array([4, 15], dtype=np.uint32)
    assert L.dqmc_batch_run(2, too_big.ctypes.data_as(dqmc.c_u32p), o_p, 256, None, 256, 256, o_p,
                            None) == dqmc.DQMC_EINVAL
    odd = np.array([0, 2], dtype=np.uint64)      # n = 14 table not 4-aligned; bitmap not 16-aligned
    assert L.dqmc_batch_run(2, n_p, odd.ctypes.data_as(dqmc.c_u64p), 256, None, 256, 256, o_p,
                            None) == dqmc.DQMC_EINVAL
    assert L.dqmc_batch_run(2, n_p, o_p, 256, None, 256, 256, odd.ctypes.data_as(dqmc.c_u64p),
                            None) == dqmc.DQMC_EINVAL
    assert L.dqmc_batch_run(2, n_p, o_p, 256, None, 260, 256, o_p, None) == dqmc.DQMC_EINVAL  # counts


def test_batch_workspace_and_layout():
    # n <= 12 functions need no state; on the tile path n = 13, 14 one padded
    # state each, on the shared-memory path none
    saved = dqmc.batch_tuning_table()
    try:
        assert dqmc.dqmc_batch_workspace_bytes(np.array([4, 12])) < 1 << 16
        for n in (13, 14):
            assert dqmc.dqmc_batch_set_config(n, dict(saved[str(n)], path=dqmc.DQMC_BATCH_PATH_TILES)) == 0
        w = dqmc.dqmc_batch_workspace_bytes(np.array([13, 14, 14]))
        assert w >= (3 ** 8 + 2 * 3 ** 9) * 32
        for n in (13, 14):
            cfg = dict(path=dqmc.DQMC_BATCH_PATH_SMEM, threads_per_fn=256, fns_per_cta=1, digits_per_step=2,
                       ctas_per_fn=3 if n == 14 else 1)
            assert dqmc.dqmc_batch_set_config(n, cfg) == 0
        # no states; n = 14 keeps a scratch third (3^8 rows) per CTA slot of its one-CTA kernel
        assert dqmc.dqmc_batch_workspace_bytes(np.array([13])) < 1 << 16
        w14 = dqmc.dqmc_batch_workspace_bytes(np.array([13, 14, 14]))
        assert w14 % (3 ** 8 * 32) < 1 << 16 and 64 * 3 ** 8 * 32 <= w14 < 1024 * 3 ** 8 * 32
    finally:
        dqmc.load_batch_tuning(saved)
    assert dqmc.dqmc_batch_workspace_bytes(np.array([15])) == 0
    off, total = dqmc.batch_bitmap_layout([0, 4, 5, 14])
    sizes = [dqmc.dqmc_bitmap_alloc_bytes(n) for n in (0, 4, 5, 14)]
    assert list(off) == [0, sizes[0], sizes[0] + sizes[1], sum(sizes[:3])] and total == sum(sizes)
    assert all(o % 16 == 0 for o in off)


def test_server_arguments_rejected_without_gpu():
    import ctypes
    L = dqmc.lib()
    h = dqmc.c_vp()
    assert L.dqmc_server_create(1 << 10, 4, 0, ctypes.byref(h)) == dqmc.DQMC_EINVAL   # budget < 1 MB
    assert L.dqmc_server_create(1 << 30, 0, 0, ctypes.byref(h)) == dqmc.DQMC_EINVAL   # no stream
    assert L.dqmc_server_create(1 << 30, 33, 0, ctypes.byref(h)) == dqmc.DQMC_EINVAL
    assert L.dqmc_server_create(1 << 30, 4, 7, ctypes.byref(h)) == dqmc.DQMC_EINVAL   # mode
    assert L.dqmc_server_create(1 << 30, 4, 0, None) == dqmc.DQMC_EINVAL
    assert L.dqmc_server_destroy(None) == dqmc.DQMC_EINVAL
    assert L.dqmc_server_submit(None, 4, None, None, 0, None) == dqmc.DQMC_EINVAL


def test_server_job_bytes():
    # a job holds its truth table(s), its bitmap slot and (n >= 15, the
    # streaming path) its workspace; n <= 14 keep their state in shared memory
    for n in (0, 5, 12, 13, 14, 15, 18, 22):
        b = dqmc.dqmc_server_job_bytes(n)
        assert b >= dqmc.dqmc_bitmap_alloc_bytes(n) + ((1 << n) + 7) // 8
        if n >= 15:
            assert b >= dqmc.dqmc_workspace_bytes(n)
        else:
            assert b < dqmc.dqmc_bitmap_alloc_bytes(n) + 2 * ((1 << n) + 7) // 8 + 4096
        assert dqmc.dqmc_server_job_bytes(n, True) > b
    assert dqmc.dqmc_server_job_bytes(26) == 0


# ------------------------------------------------------------------ plan

def plan(n):
    return dqmc.dqmc_plan_json(n)


def decode_fixed(fix, x):
    """Mixed-radix decode exactly as the kernel: first entry least significant."""
    row = 0
    for digit, radix in fix:
        d = x % radix
        x //= radix
        row += d * 3 ** digit
    return row


def spread3(x):
    r, w = 0, 1
    while x:
        if x & 1:
            r += w
        x >>= 1
        w *= 3
    return r


def tile_rows(ph, base, binary_group):
    RE, K = 3 ** ph["B"], ph["K"]
    gs = [spread3(b) for b in range(1 << K)] if binary_group else range(3 ** K)
    return [base + e + g * 3 ** ph["a"] for g in gs for e in range(RE)]


def row_digits(r, H):
    d = []
    for _ in range(H):
        d.append(r % 3)
        r //= 3
    return d


@pytest.mark.parametrize("n", list(range(0, 26)))
def test_plan_digit_coverage(n):
    p = plan(n)
    C, H = p["C"], p["H"]
    assert C == min(n, 5) and H == n - C
    merged, reduced, chunk = [], [], 0
    merge_done = False
    for sp in p["passes"]:
        for ph in sp["phases"]:
            digits = list(range(ph["a"], ph["a"] + ph["K"]))
            assert ph["K"] + ph["B"] <= 7
            assert ph["B"] <= ph["a"] or ph["K"] == 0 or ph["a"] == 0
            if ph["merge"]:
                assert not merge_done or ph["reduce"], "a Merge after the first Reduce"
                merged += digits
            if ph["reduce"]:
                # every digit is merged before the first Reduce
                merge_done = True
                reduced += digits
            if ph["nbr_K"]:
                # the neighbour group: only in the bitmap pass, and only the
                # digits just above its tile (the first fixed digits)
                assert ph["out"] and ph["nbr_a"] == 7 and 1 <= ph["nbr_K"] <= 6
                reduced += list(range(ph["nbr_a"], ph["nbr_a"] + ph["nbr_K"]))
            chunk += bin(ph["chunk_mask"]).count("1")
    assert sorted(merged) == list(range(H))
    assert sorted(reduced) == list(range(H))
    assert chunk == C
    last = p["passes"][-1]["phases"][-1]
    assert last["out"] == 1
    outs = [ph["out"] for sp in p["passes"] for ph in sp["phases"]]
    assert sum(outs) == 1
    if H > 7:
        assert p["state_rows"] == 3 ** H
        assert last["a"] == 0 and last["B"] == 0 and last["K"] == 7
        assert p["out_tiles"] == 3 ** H // 2187
        for sp in p["passes"]:
            ph = sp["phases"][0]
            assert ph["K"] + ph["B"] == 7   # 2187-row tiles


@pytest.mark.parametrize("n", [13, 14, 15, 16, 17])
def test_plan_tiles_cover_rows(n):
    """Every phase's tiles touch exactly the rows they must, each once; sparse
    loads read exactly the rows earlier phases wrote."""
    p = plan(n)
    H = p["H"]
    merged = set()
    written = set()
    for sp in p["passes"]:
        sb_digits = sorted(set(range(H)) - {d for d, _ in sp["sb"]})
        for ph in sp["phases"]:
            grp = set(range(ph["a"], ph["a"] + ph["K"]))
            reads, writes = [], []
            for sb in range(sp["n_sb"]):
                b0 = decode_fixed(sp["sb"], sb)
                for t in range(ph["tiles"]):
                    base = b0 + decode_fixed(ph["fix"], t)
                    if ph["load"] == "sparse":
                        reads += tile_rows(ph, base, True)
                    elif ph["load"] == "full":
                        reads += tile_rows(ph, base, False)
                    writes += tile_rows(ph, base, False)
            assert len(set(writes)) == len(writes), "tiles overlap"
            assert all(0 <= r < 3 ** H for r in writes)
            after = merged | (grp if ph["merge"] else set())
            want = {r for r in range(3 ** H)
                    if all(dg != 2 or j in after for j, dg in enumerate(row_digits(r, H)))}
            assert set(writes) == want
            if ph["load"] == "sparse":
                got = set(reads)
                assert got == {r for r in want if all(row_digits(r, H)[j] != 2 for j in grp)}
                assert got <= written
            elif ph["load"] == "full":
                assert set(reads) == want and set(reads) <= written
            written |= set(writes)
            merged = after
        # super-block digit set: group + inner + phase-fixed digits of every phase
        for ph in sp["phases"]:
            inside = set(range(ph["B"])) | set(range(ph["a"], ph["a"] + ph["K"])) | {d for d, _ in ph["fix"]}
            assert inside == set(sb_digits) or sp["kind"] == "whole"


@pytest.mark.parametrize("n", list(range(13, 26)))
def test_plan_rows_in_bounds(n):
    """Extreme tiles stay below 3^H; tile and ticket counts fit the kernel's types."""
    p = plan(n)
    H = p["H"]
    for sp in p["passes"]:
        last_sb = decode_fixed(sp["sb"], sp["n_sb"] - 1)
        tickets = 0
        for ph in sp["phases"]:
            top = last_sb + decode_fixed(ph["fix"], ph["tiles"] - 1)
            row_max = top + 3 ** ph["B"] - 1 + (3 ** ph["K"] - 1) * 3 ** ph["a"]
            assert row_max < 3 ** H
            assert 3 ** (ph["K"] + ph["B"]) <= 2187
            tickets += ph["tiles"] * sp["n_sb"]
            if ph["load"] == "tt":
                # truth-table words: binary value of the fixed digits times 2^K + gb < 2^H
                tt = sum(2 ** d for d, r in sp["sb"]) + 2 ** ph["K"] - 1
                assert tt < 2 ** H
            if ph["out"]:
                assert ph["a"] == 0 and ph["B"] == 0 and ph["K"] == 7
        assert tickets < 2 ** 32


# ------------------------------------------------- ticket order (host replica)

def decode_ticket(sp, ticket):
    """Replica of the device decode: fixed-size pipeline steps; None = empty ticket."""
    step, r = divmod(ticket, sp["step_size"])
    offs, acc = [], 0
    for ph in sp["phases"]:
        offs.append(acc)
        acc += sp["window"] * ph["tiles"]
    p_ = len(sp["phases"]) - 1
    while p_ > 0 and r < offs[p_]:
        p_ -= 1
    r -= offs[p_]
    if step < p_:
        return None
    g = step - p_
    if g >= sp["groups"]:
        return None
    tiles = sp["phases"][p_]["tiles"]
    sbl, t = divmod(r, tiles)
    sb = g * sp["window"] + sbl
    if sb >= sp["n_sb"]:
        return None
    return p_, sb, t


@pytest.mark.parametrize("n", [13, 15, 16, 18, 21, 24])
def test_ticket_order_is_a_valid_schedule(n):
    """The device's ticket -> (phase, super-block, tile) map is a bijection and
    every tile's dependencies (all tiles of the previous phase of its block)
    hold smaller tickets; bitmap tiles come in ascending rho order."""
    p = plan(n)
    for sp in p["passes"]:
        if sp["kind"] == "whole":
            continue
        want = sum(ph["tiles"] for ph in sp["phases"]) * sp["n_sb"]
        assert sp["step_size"] == sp["window"] * sum(ph["tiles"] for ph in sp["phases"])
        assert sp["n_steps"] == sp["groups"] + len(sp["phases"]) - 1
        assert sp["groups"] == -(-sp["n_sb"] // sp["window"])
        if want > 400000:
            # large plans: same window, truncated to a few super-block groups
            nsb = min(sp["n_sb"], 7 * sp["window"] + 3)
            sp = dict(sp, n_sb=nsb, groups=-(-nsb // sp["window"]))
            sp["n_steps"] = sp["groups"] + len(sp["phases"]) - 1
            want = sum(ph["tiles"] for ph in sp["phases"]) * sp["n_sb"]
        total = sp["n_steps"] * sp["step_size"]
        assert total < 2 ** 32
        seen = {}
        last_of = {}
        for tk in range(total):
            key = decode_ticket(sp, tk)
            if key is None:
                continue
            assert key not in seen
            seen[key] = tk
            last_of[(key[0], key[1])] = max(last_of.get((key[0], key[1]), -1), tk)
        assert len(seen) == want
        for (ph, sb, t), tk in seen.items():
            if ph > 0:
                assert last_of[(ph - 1, sb)] < tk
        out_phase = [i for i, ph in enumerate(sp["phases"]) if ph["out"]]
        if out_phase:
            op = out_phase[0]
            bases = sorted((tk, decode_fixed(sp["sb"], sb) + decode_fixed(sp["phases"][op]["fix"], t))
                           for (ph, sb, t), tk in seen.items() if ph == op)
            rows = [b for _, b in bases]
            assert rows == sorted(rows)


# ------------------------------------------------- semantic simulation

def reduce_clear(S, n, digits):
    """Cells whose '*' neighbour in one of the digits is set in S."""
    A = S.reshape((3,) * n) if n else S
    clear = np.zeros_like(A)
    for j in digits:
        ax = n - 1 - j
        star = np.take(A, [2], axis=ax)
        for v in (0, 1):
            idx = [slice(None)] * n
            idx[ax] = slice(v, v + 1)
            clear[tuple(idx)] |= star
    return clear.reshape(-1)


def grouped_reduce(S, n, digits):
    """Reduce over a set of digits, every read taken from the state as it was before."""
    return S & ~reduce_clear(S, n, digits)


def merge_digit(S, n, j):
    A = S.reshape((3,) * n).copy()
    ax = n - 1 - j
    s0 = np.take(A, [0], axis=ax)
    s1 = np.take(A, [1], axis=ax)
    idx = [slice(None)] * n
    idx[ax] = slice(2, 3)
    A[tuple(idx)] |= s0 & s1
    return A.reshape(-1)


@pytest.mark.parametrize("n,seed", [(8, 1), (13, 2), (14, 3), (15, 4), (16, 5), (19, 6)])
def test_plan_schedule_simulated(n, seed):
    """Run the plan's digit schedule on the host (Merge digit by digit, Reduce
    grouped per phase from the phase's starting state) against the oracle."""
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
    for sp in p["passes"]:
        for ph in sp["phases"]:
            grp = [C + d for d in range(ph["a"], ph["a"] + ph["K"])]
            if ph["load"] == "tt":
                for j in range(C):
                    S = merge_digit(S, n, j)
            if ph["merge"]:
                for j in grp:
                    S = merge_digit(S, n, j)
            red = (grp if ph["reduce"] else []) + [i for i in range(C) if (ph["chunk_mask"] >> i) & 1]
            before = S
            if red:
                S = grouped_reduce(S, n, red)
            if ph["nbr_K"]:
                # the neighbour group reads the state as the pass found it
                S = S & ~reduce_clear(before, n, [C + d for d in range(ph["nbr_a"], ph["nbr_a"] + ph["nbr_K"])])
    want = oracle.sweep(n, on, dc) != 0
    assert np.array_equal(S, want)


def _cfg(path, tg, fpc, d, ctas=1):
    return dict(path=path, threads_per_fn=tg, fns_per_cta=fpc, digits_per_step=d, ctas_per_fn=ctas)


def test_batch_config_rules_without_gpu():
    """dqmc_batch_set_config accepts exactly the launchable shapes (host
    logic only: threads, functions per CTA, digits per step, shared memory,
    clusters of 3 for n = 13, 14 and of 9 for n = 14, the shared-memory path
    only for 5 <= n <= 14)."""
    saved = dqmc.batch_tuning_table()
    S, T = dqmc.DQMC_BATCH_PATH_SMEM, dqmc.DQMC_BATCH_PATH_TILES
    try:
        for n in range(dqmc.DQMC_BATCH_MAX_N + 1):
            c = saved[str(n)]
            assert c["path"] in (S, T) and (c["path"] == T or 5 <= n <= 14)
            assert dqmc.dqmc_batch_set_config(n, _cfg(T, 0, 0, 0, 0)) == dqmc.DQMC_OK
        ok = [(5, 32, 15, 2), (5, 32, 8, 3), (12, 512, 1, 3), (12, 64, 3, 2), (13, 1024, 1, 2), (12, 1024, 1, 3),
              (14, 512, 1, 3, 3), (14, 32, 1, 2, 9), (14, 1024, 1, 3, 9), (13, 256, 1, 2, 3), (10, 96, 3, 3),
              (14, 1024, 1, 3, 1)]     # one CTA doing the thirds of the top digit in turn
        bad = [(4, 32, 1, 2),        # below the chunk size
               (15, 32, 1, 2),       # above the batch range
               (8, 48, 1, 2),        # not whole warps
               (8, 0, 1, 2), (8, 32, 0, 2), (8, 32, 16, 2),
               (8, 64, 1, 4), (8, 64, 1, 1),     # digits per step
               (8, 512, 4, 2),       # 2048 threads
               (12, 64, 4, 2),       # 4 x 70 KB of shared memory
               (13, 64, 2, 2),       # 2 x 210 KB
               (14, 64, 2, 2, 3),    # clusters hold one function
               (14, 64, 2, 2, 1),    # 2 x 210 KB
               (13, 64, 1, 2, 9),    # nine CTAs only for n = 14
               (12, 64, 1, 2, 3),    # clusters only for n = 13, 14
               (14, 64, 1, 2, 2),    # 1, 3 or 9 CTAs
               (14, 64, 1, 2, 0)]
        for t in ok:
            assert dqmc.dqmc_batch_set_config(t[0], _cfg(S, *t[1:])) == dqmc.DQMC_OK, t
            assert dqmc.dqmc_batch_get_config(t[0]) == _cfg(S, *t[1:])
        for t in bad:
            assert dqmc.dqmc_batch_set_config(t[0], _cfg(S, *t[1:])) == dqmc.DQMC_EINVAL, t
        assert dqmc.dqmc_batch_set_config(2, _cfg(7, 32, 1, 2)) == dqmc.DQMC_EINVAL   # unknown path
        with pytest.raises(dqmc.DqmcError):
            dqmc.dqmc_batch_get_config(15)
        # the JSON form goes through unchanged
        table = json.loads(json.dumps(dqmc.batch_tuning_table()))
        dqmc.load_batch_tuning(saved)
        dqmc.load_batch_tuning(table)
        assert dqmc.batch_tuning_table() == table
    finally:
        dqmc.load_batch_tuning(saved)


def test_batch_autotune_arguments_without_gpu():
    L = dqmc.lib()
    out = (ctypes.c_float * (dqmc.DQMC_BATCH_MAX_N + 1))()
    assert L.dqmc_batch_autotune(0, None, None, None, None, None, None, None, 3, None, out) == dqmc.DQMC_OK
    assert all(x == -1.0 for x in out)
    n = np.array([5, 6], dtype=np.uint32)
    o = np.zeros(2, dtype=np.uint64)
    n_p, o_p = n.ctypes.data_as(dqmc.c_u32p), o.ctypes.data_as(dqmc.c_u64p)
    assert L.dqmc_batch_autotune(2, n_p, o_p, 256, None, 256, 256, o_p, 0, None, out) == dqmc.DQMC_EINVAL
    assert L.dqmc_batch_autotune(2, n_p, o_p, 256, None, 256, 256, o_p, 1001, None, out) == dqmc.DQMC_EINVAL
    assert L.dqmc_batch_autotune(2, None, o_p, 256, None, 256, 256, o_p, 3, None, out) == dqmc.DQMC_EINVAL


# ---------------------------------------------------------------- Table 1 memory

def test_state_size_matches_table1_ram_column():
    """Table 1 (DenseQMC, density: any): the RAM column is the in-place state
    of 3^(n-5) blocks of 256 bits (h = 5 digits per block), at the printed
    precision, for n = 16 .. 27.  The library's plan keeps exactly that state,
    one 32-byte row per block, up to n = 25 (the largest n it takes); its
    device workspace adds under 1% (a control block and the list's scan
    counters)."""
    unit = {"MiB": 2 ** 20, "GiB": 2 ** 30, "TiB": 2 ** 40}
    rows = []
    for line in open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_dense_ram.txt")):
        if line.strip() and not line.startswith("#"):
            n, val, u = line.split()
            rows.append((int(n), val, u))
    assert [n for n, _, _ in rows] == list(range(16, 28))
    for n, val, u in rows:
        decimals = len(val.split(".")[1]) if "." in val else 0
        state = 3 ** (n - 5) * 32
        assert round(state / unit[u], decimals) == float(val), (n, state / unit[u], val)
        if n <= 25:
            assert dqmc.dqmc_plan_json(n)["state_rows"] * 32 == state
            assert state <= dqmc.dqmc_workspace_bytes(n) <= state * 1.01


@pytest.mark.parametrize("n", [0, 8, 12, 13, 21, 24, 25])
def test_plan_json_fields_as_documented(n):
    """dqmc_plan_json writes exactly the fields include/dqmc_plan.h lists."""
    p = dqmc.dqmc_plan_json(n)
    assert set(p) == {"n", "C", "H", "state_rows", "out_tiles", "passes"}
    assert p["n"] == n and p["C"] == min(n, 5) and p["H"] == n - p["C"]
    assert len(p["passes"]) == dqmc.dqmc_plan_passes(n)
    for q in p["passes"]:
        assert q["kind"] in ("whole", "super")
        want = {"kind", "n_sb", "window", "sb", "phases"} | (
            {"step_size", "n_steps", "groups"} if q["kind"] == "super" else set())
        assert set(q) == want
        assert len(q["phases"]) == 1
        ph = q["phases"][0]
        assert set(ph) == {"load", "K", "B", "a", "merge", "reduce", "chunk_mask", "out", "nbr_a", "nbr_K",
                           "tiles", "fix"}
        assert ph["load"] in ("tt", "sparse", "full") and ph["fix"] == []
        if q["kind"] == "super":
            assert q["window"] == q["step_size"] == q["n_sb"] and q["n_steps"] == q["groups"] == 1
    assert (p["state_rows"] == 0) == (p["passes"][0]["kind"] == "whole")


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: with the library absent (and no build allowed), the
    binding raises instead of computing anything."""
    monkeypatch.setattr(dqmc, "_lib", None)
    monkeypatch.setattr(dqmc._build, "LIB", str(tmp_path / "libdqmc.so"))
    with pytest.raises(RuntimeError, match="libdqmc.so not found"):
        dqmc.lib(build_if_missing=False)
    monkeypatch.setattr(dqmc._build, "up_to_date", lambda: True)
    with pytest.raises(RuntimeError, match="libdqmc.so not found"):
        dqmc.dqmc_primes(4, np.zeros(2, dtype=np.uint8))


def test_oracle_and_cuda_path_share_no_code():
    """The oracle and the CUDA path are independent: no file of the package or
    of include/ names the oracle, and no oracle file names the package, its
    headers or its sources.  Only the seeded input generator (synth.py, no
    method arithmetic) is used by both, and by the tests alone on the oracle
    side."""
    pkg = os.path.join(ROOT, "paper_2302_10083_gb300")
    product = [p for ext in ("py", "cu", "cuh", "h") for p in glob.glob(os.path.join(pkg, "**", "*." + ext),
                                                                         recursive=True)]
    product += glob.glob(os.path.join(ROOT, "include", "*.h"))
    for p in product:
        text = open(p).read()
        if p.endswith("synth.py"):
            text = text.split('"""', 2)[-1]   # its docstring names the oracle as a user
        assert not re.search(r"\boracle\b|dqmc_oracle", text), p
    for p in glob.glob(os.path.join(ROOT, "oracle", "*.py")) + glob.glob(os.path.join(ROOT, "oracle", "*.c")):
        text = open(p).read()
        assert not re.search(r"paper_2302_10083_gb300|libdqmc\.so|dqmc\.h|csrc|#include \"", text), p


def test_static_workspace_tests_collected_last():
    """The static-workspace GPU test sits in the module pytest collects last
    (files in name order), so a run that stops at its first failure has run
    every other test before it."""
    files = sorted(os.path.basename(p) for p in glob.glob(os.path.join(ROOT, "tests", "test_*.py")))
    assert files[-1] == "test_zzz_no_alloc.py", files[-3:]
