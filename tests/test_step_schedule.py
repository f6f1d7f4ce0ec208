"""The schedules the shared-memory kernels follow, run on the host against the
oracle (no GPU): high digits merged D at a time from the lowest digit up,
each block in place (a '*' cell of digit d is the AND of its 0 and 1 cells,
computed in the order of d); Reduce D digits at a time, a block's cells
updated in order of their number of '*' digits in the block (so every cell
reads its neighbours as the step found them); the chunk digits last, all
from one snapshot.  And the split of a function on its top one or two high
digits (clusters of 3 or 9 CTAs, or one CTA doing the three thirds of the
top digit in turn): each part merged from the truth-table slices of its
top-digit values (a '*' value ANDs the slices of 0 and 1), the top digits
reduced one after the other from the parts as they stand, then each part's
own digits.  Algorithm 3 (Section 4.1) fixes the result; these tests pin
that the orders the kernels use reach it."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2302_10083_gb300 import synth

C = 5   # chunk digits


def digits(n):
    """digit i of every cell rho = sum 3^i d_i, shape (n, 3^n)"""
    r = np.arange(3 ** n)
    return np.stack([(r // 3 ** i) % 3 for i in range(n)])


def support(n, on, dc):
    sup = np.unpackbits(on, bitorder="little")[: 1 << n].astype(bool)
    if dc is not None:
        sup |= np.unpackbits(dc, bitorder="little")[: 1 << n].astype(bool)
    return sup


def binary_cells(n, sup, fixed=None):
    """S with the support on the binary cells (Merge not started).  fixed:
    {digit: value} restricts to cells with those digits (a '*' value ANDs the
    minterms with 0 and 1 there, as a '*' part of a split does)."""
    S = np.zeros(3 ** n, dtype=bool)
    dg = digits(n)
    binary = (dg != 2).all(axis=0)
    rho = np.nonzero(binary)[0]
    t = np.zeros(len(rho), dtype=np.int64)
    for i in range(n):
        t |= dg[i, rho].astype(np.int64) << i
    S[rho] = sup[t]
    if fixed:
        # a '*' split digit: the cell holds the AND over both values there (the
        # AND of the truth-table slices); two '*' digits AND all four
        have = rho
        for d, v in sorted(fixed.items()):
            if v == 2:
                lo = have[dg[d, have] == 0]
                S[lo + 2 * 3 ** d] = S[lo] & S[lo + 3 ** d]
                have = np.concatenate([have, lo + 2 * 3 ** d])
    return S


def merge_block(S, n, J, D, hi_end, dg):
    """Merge of digits J..J+D-1: blocks whose digits below J take any value
    and whose digits J+D .. hi_end-1 are 0/1 (the digits from hi_end up are
    fixed per part of a split); in-block order by digit."""
    hi_binary = np.ones(3 ** n, dtype=bool)
    for i in range(J + D, hi_end):
        hi_binary &= dg[i] != 2
    for d in range(J, J + D):
        w = 3 ** d
        sel = hi_binary & (dg[d] == 2)
        for e in range(d + 1, J + D):        # digits above d in the block still 0/1
            sel &= dg[e] != 2
        idx = np.nonzero(sel)[0]
        S[idx] = S[idx - 2 * w] & S[idx - w]
    return S


def reduce_block(S, n, J, D, dg):
    """Reduce of digits J..J+D-1, in place, cells with k '*' digits in the
    block updated at step k (their neighbours have k+1 and are unchanged)."""
    twos = sum((dg[d] == 2).astype(int) for d in range(J, J + D))
    for k in range(D):
        idx = np.nonzero(twos == k)[0]
        acc = np.zeros(len(idx), dtype=bool)
        for d in range(J, J + D):
            w = 3 ** d
            td = dg[d, idx]
            nb = idx + (2 - td) * w
            acc |= np.where(td != 2, S[np.where(td != 2, nb, idx)], False)
        S[idx] &= ~acc
    return S


def reduce_group(S, n, ds, dg):
    """Reduce of the digits ds from one snapshot (a grouped Reduce)."""
    snap = S.copy()
    acc = np.zeros(3 ** n, dtype=bool)
    for d in ds:
        w = 3 ** d
        for v in (0, 1):
            idx = np.nonzero(dg[d] == v)[0]
            acc[idx] |= snap[idx + (2 - v) * w]
    return S & ~acc


def sweep_blocks(n, sup, D, top=0):
    """The whole-function schedule with `top` (0, 1, 2) split digits."""
    dg = digits(n)
    H = n - C
    HL = H - top
    parts = {}
    for vals in itertools.product(range(3), repeat=top):
        fixed = {C + HL + c: v for c, v in enumerate(vals)}
        S = binary_cells(n, sup, fixed)
        # chunk digits merged on load (digit by digit), then the part's high digits
        for j in range(C):
            S = merge_block(S, n, j, 1, C + HL, dg)
        J = C
        while J < C + HL:
            DD = min(D, C + HL - J)
            S = merge_block(S, n, J, DD, C + HL, dg)
            J += DD
        keep = np.ones(3 ** n, dtype=bool)
        for d, v in fixed.items():
            keep &= dg[d] == v
        parts[vals] = (S & keep, keep)
    # top digits: one after the other, each from the parts as they stand
    for c in range(top):
        new = {}
        for vals, (S, keep) in parts.items():
            if vals[c] != 2:
                star = list(vals)
                star[c] = 2
                T, _ = parts[tuple(star)]
                w = 3 ** (C + HL + c)
                idx = np.nonzero(keep)[0]
                S = S.copy()
                S[idx] &= ~T[idx + (2 - vals[c]) * w]
            new[vals] = (S, keep)
        parts = new
    out = np.zeros(3 ** n, dtype=bool)
    for vals, (S, keep) in parts.items():
        J = C
        while J < C + HL:
            DD = min(D, C + HL - J)
            S = reduce_block(S, n, J, DD, dg)
            J += DD
        S = reduce_group(S, n, range(C), dg)
        out |= S & keep
    return out


@pytest.mark.parametrize("n,D,top", [(5, 2, 0), (6, 3, 0), (8, 2, 0), (8, 3, 0), (9, 3, 0), (9, 2, 1),
                                     (8, 3, 1), (9, 2, 2), (9, 3, 2)])
def test_block_schedule_equals_oracle(n, D, top):
    for seed, p_on, p_dc in ((1, 0.75, 0.1), (2, 0.5, 0.0), (3, 0.9, 0.05)):
        on, dc = synth.random_function(n, seed + 10 * n, p_on, p_dc)
        got = sweep_blocks(n, support(n, on, dc), D, top)
        want = oracle.sweep(n, on, dc) != 0
        assert np.array_equal(got, want), (n, D, top, seed)


def test_reversed_in_block_order_is_wrong():
    """The in-block order matters: updating a block's cells starting with the
    most '*' digits (reading neighbours already updated in the same step)
    clears the extensions a cell needs, so for f = 1 the cells with binary
    block digits survive beside the all-'*' prime."""
    n, D = 7, 2
    dg = digits(n)
    on = np.full(synth.tt_bytes(n), 0xFF, dtype=np.uint8)
    sup = support(n, on, None)

    def reduce_block_reversed(S, J):
        twos = sum((dg[d] == 2).astype(int) for d in range(J, J + D))
        for k in reversed(range(D)):
            idx = np.nonzero(twos == k)[0]
            acc = np.zeros(len(idx), dtype=bool)
            for d in range(J, J + D):
                td = dg[d, idx]
                nb = idx + (2 - td) * 3 ** d
                acc |= np.where(td != 2, S[np.where(td != 2, nb, idx)], False)
            S[idx] &= ~acc
        return S

    S = binary_cells(n, sup)
    for j in range(n):
        S = merge_block(S, n, j, 1, n, dg)
    good, bad = S.copy(), S.copy()
    good = reduce_block(good, n, C, D, dg)
    bad = reduce_block_reversed(bad, C)
    for T in (good, bad):
        T[:] = reduce_group(T, n, range(C), dg)
    want = oracle.sweep(n, on, None) != 0
    assert want.sum() == 1 and want[3 ** n - 1]   # f = 1: only the all-'*' cube
    assert np.array_equal(good, want)
    assert not np.array_equal(bad, want)


# ----------------------------------------- the bitmap pass's row-loop digit

def _clear(S, n, digs):
    """Cells whose '*' neighbour in one of the digits (cell digit indices) is
    set in S."""
    A = S.reshape((3,) * n)
    out = np.zeros_like(A)
    for j in digs:
        ax = n - 1 - j
        star = np.take(A, [2], axis=ax)
        for v in (0, 1):
            idx = [slice(None)] * n
            idx[ax] = slice(v, v + 1)
            out[tuple(idx)] |= star
    return out.reshape(-1)


def _implicants(n, sup):
    """Merge of every digit from the support: M(s) = every covered minterm in ON or DC."""
    S = np.zeros(3 ** n, dtype=bool)
    t = np.arange(1 << n)
    rho = np.zeros_like(t)
    for i in range(n):
        rho += ((t >> i) & 1) * 3 ** i
    S[rho] = sup
    A = S.reshape((3,) * n)
    for j in range(n):
        ax = n - 1 - j
        s0 = np.take(A, [0], axis=ax)
        s1 = np.take(A, [1], axis=ax)
        idx = [slice(None)] * n
        idx[ax] = slice(2, 3)
        A[tuple(idx)] = s0 & s1
    return A.reshape(-1)


@pytest.mark.parametrize("n,tile,nbr,seed,p_on,p_dc", [
    (12, 7, 0, 1, 0.8, 0.0), (12, 7, 0, 2, 0.6, 0.1), (12, 4, 2, 3, 0.75, 0.05),
    (11, 3, 2, 4, 0.85, 0.0), (10, 3, 1, 5, 0.5, 0.2), (12, 5, 2, 6, 0.9, 0.0)])
def test_bitmap_pass_row_loop_digit_is_exact(n, tile, nbr, seed, p_on, p_dc):
    """The bitmap pass reduces its tile digits but the top one in steps (each
    step reading what the previous left), then, per row, clears a cell by its
    neighbour group (read from the state the previous pass left, which had
    the groups above reduced), its chunk digits (read from its row as the
    steps left it) and its top tile digit, whose '*' row another thread may
    be writing back at the same time: each bit of it is seen either as the
    steps left it or final.  The result is the prime set for any such mix,
    all-old and all-new included (Algorithm 3's ReduceAll, Section 4.1)."""
    on, dc = synth.random_function(n, seed, p_on, p_dc)
    sup = support(n, on, dc)
    want = oracle.sweep(n, on, dc) != 0
    H = n - C
    tile_d = [C + j for j in range(tile)]              # high digits 0 .. tile-1
    top = tile_d[-1]
    nbr_d = [C + j for j in range(tile, tile + nbr)]   # the neighbour group
    rest = [C + j for j in range(tile + nbr, H)]       # reduced by earlier passes
    M = _implicants(n, sup)
    S1 = M & ~_clear(M, n, rest)                       # the state the bitmap pass reads
    T1 = S1.copy()
    steps = [tile_d[:-1][i:i + 3] for i in range(0, len(tile_d) - 1, 3)]
    for st in steps:
        T1 = T1 & ~_clear(T1, n, st)
    rng = np.random.default_rng(seed)
    for mix in ("old", "new", "random", "random"):
        if mix == "old":
            X = T1
        elif mix == "new":
            X = want
        else:
            X = np.where(rng.random(T1.size) < 0.5, T1, want)
        got = T1 & ~_clear(S1, n, nbr_d) & ~_clear(T1, n, list(range(C))) & ~_clear(X, n, [top])
        assert np.array_equal(got, want), mix


def test_row_loop_digit_model_catches_a_second_racy_digit():
    """Planted mistake: read two tile digits from a mix of old and final
    states (instead of one); some function then keeps a non-prime cell, so
    the model above tells the one-digit argument from a wrong one."""
    found = False
    for seed in range(1, 40):
        n = 9
        on, dc = synth.random_function(n, seed, 0.8, 0.0)
        sup = support(n, on, dc)
        want = oracle.sweep(n, on, dc) != 0
        tile_d = [C + j for j in range(4)]
        M = _implicants(n, sup)
        T1 = M & ~_clear(M, n, tile_d[:2])
        X = want   # both racy digits read entirely final
        got = T1 & ~_clear(T1, n, list(range(C))) & ~_clear(X, n, tile_d[2:])
        if not np.array_equal(got, want):
            found = True
            break
    assert found
