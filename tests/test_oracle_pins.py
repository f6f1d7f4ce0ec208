"""Pins for the CPU oracle: things the paper and the mathematics fix, none of
which re-runs the oracle's own Merge/Reduce loops.

Each test names the passage of arXiv 2302.10083 it rests on.
"""
import os

import numpy as np
import pytest

import bruteforce as bf
import oracle
from paper_2302_10083_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def oracle_cells(n, support_bool, dc_bool=None):
    on = bf.bitmap_from_bool(support_bool)
    dc = None if dc_bool is None else bf.bitmap_from_bool(dc_bool)
    S = oracle.sweep(n, on, dc)
    return S != 0


# ---------------------------------------------------------------- worked examples

def test_majority_golden():
    """Section 1: Maj(x, y, z) = xy + xz + yz, so its primes are 11*, 1*1, *11."""
    meta, rows = bf.load_golden(os.path.join(GOLDEN, "maj3.txt"))
    n = int(meta["n"])
    on = np.zeros(1 << n, dtype=bool)
    for t in meta["on_minterms"].split(","):
        on[int(t)] = True
    S = oracle.sweep(n, bf.bitmap_from_bool(on))
    got = oracle.pairs(n, S)
    assert [tuple(map(int, p)) for p in got] == [(m, v) for _, _, m, v in rows]
    assert sorted(np.nonzero(S)[0].tolist()) == [r for _, r, _, _ in rows]
    for cube, rho, _, _ in rows:
        assert bf.rho_of_string(cube) == rho
        assert oracle.encode(n, rho) == next((m, v) for c, r, m, v in rows if r == rho)


def test_merge_example_golden():
    """Section 3 example: 0011* + 0111* = 0*11* (the merged cube is the only prime)."""
    meta, rows = bf.load_golden(os.path.join(GOLDEN, "merge_example.txt"))
    n = int(meta["n"])
    cubes = meta["cubes"].split(",")
    sup = np.zeros(1 << n, dtype=bool)
    for t in range(1 << n):
        for c in cubes:
            if all(ch == "*" or int(ch) == ((t >> i) & 1) for i, ch in enumerate(c)):
                sup[t] = True
    S = oracle.sweep(n, bf.bitmap_from_bool(sup))
    assert np.nonzero(S)[0].tolist() == [rows[0][1]]
    assert bf.cube_string(n, rows[0][1]) == rows[0][0]
    assert tuple(map(int, oracle.pairs(n, S)[0])) == (rows[0][2], rows[0][3])


def test_example_cube_string():
    """Section 2 example: for n = 5 the product x1 x3' is the string 1*0**."""
    rho = bf.rho_of_string("1*0**")
    m, v = oracle.encode(5, rho)
    assert m == 0b00101 and v == 0b00001


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("n", list(range(0, 9)))
def test_bruteforce_random(n):
    """Definitions (Section 2) evaluated by enumeration, random functions n <= 8."""
    for seed in range(1, 6):
        for p in (0.3, 0.6, 0.9):
            on, _ = synth.random_function(n, seed, p)
            sup = bf.support_of(n, on)
            want = bf.primes(n, sup)
            got = oracle.sweep(n, on) != 0
            assert np.array_equal(got, want), (n, seed, p)


@pytest.mark.parametrize("n", [9, 10])
def test_bruteforce_n9_n10(n):
    on, dc = synth.random_function(n, 7, 0.6, 0.2)
    sup = bf.support_of(n, on, dc)
    want = bf.primes(n, sup)
    got = oracle.sweep(n, on, dc) != 0
    assert np.array_equal(got, want)


def test_bruteforce_n10_config():
    """The n=10 workload: ON ~ Bernoulli(0.5), no don't-cares, seeds 1..3."""
    for seed in (1, 2, 3):
        on, dc = synth.single_n10(seed)
        assert dc is None
        want = bf.primes(10, bf.support_of(10, on))
        got = oracle.sweep(10, on) != 0
        assert np.array_equal(got, want)


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_every_function_small(n):
    """Every Boolean function of n <= 3 variables against brute force."""
    for _, sup in bf.all_functions(n):
        want = bf.primes(n, sup)
        got = oracle_cells(n, sup)
        assert np.array_equal(got, want)


def test_every_function_n4():
    """All 2^16 functions of 4 variables, brute force vectorised over functions."""
    n = 4
    m = 1 << n
    mask, value = bf.mask_value(n)
    covered = np.zeros(3 ** n, dtype=np.int64)  # 16-bit set of covered minterms
    for r in range(3 ** n):
        for t in range(m):
            if (t & mask[r]) == value[r]:
                covered[r] |= 1 << t
    f = np.arange(1 << m, dtype=np.int64)
    imp = (f[:, None] & covered[None, :]) == covered[None, :]
    d = bf.digits(n)
    prime = imp.copy()
    for i in range(n):
        for r in range(3 ** n):
            if d[r, i] != 2:
                ext = r + (2 - int(d[r, i])) * 3 ** i
                prime[:, r] &= ~imp[:, ext]
    for fi in range(1 << m):
        on = np.array([fi & 0xFF, fi >> 8], dtype=np.uint8)
        got = oracle.sweep(n, on) != 0
        assert np.array_equal(got, prime[fi]), fi


def test_dont_care_union():
    """Implicants are taken over ON u DC; overlapping ON and DC bits are a union."""
    n = 7
    for seed in range(1, 4):
        on, _ = synth.random_function(n, seed, 0.5)
        dc_raw, _ = synth.random_function(n, seed + 100, 0.3)  # overlaps ON on purpose
        sup = bf.support_of(n, on) | bf.support_of(n, dc_raw)
        want = bf.primes(n, sup)
        got = oracle.sweep(n, on, dc_raw) != 0
        assert np.array_equal(got, want)


def test_dc_only_prime_kept():
    """A prime whose minterms are all don't-cares is still reported."""
    n = 3
    on = np.zeros(8, dtype=bool)
    on[0] = True
    dc = np.zeros(8, dtype=bool)
    dc[7] = True
    S = oracle.sweep(n, bf.bitmap_from_bool(on), bf.bitmap_from_bool(dc))
    assert set(np.nonzero(S)[0].tolist()) == {bf.rho_of_string("000"), bf.rho_of_string("111")}


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [1, 5, 9, 12])
def test_constant_one(n):
    """Section 3, proof of the Proposition: for f = 1 every cube is an implicant and
    only the all-wildcard cube is prime."""
    S = oracle.sweep(n, np.full(synth.tt_bytes(n), 0xFF, dtype=np.uint8))
    assert np.nonzero(S)[0].tolist() == [3 ** n - 1]


@pytest.mark.parametrize("n", [0, 1, 6, 12])
def test_constant_zero(n):
    S = oracle.sweep(n, np.zeros(synth.tt_bytes(n), dtype=np.uint8))
    assert oracle.count(n, S) == 0


def test_constant_one_n0():
    """n = 0: the empty cube is prime iff f = 1."""
    S = oracle.sweep(0, np.array([1], dtype=np.uint8))
    assert S.tolist() == [1]


@pytest.mark.parametrize("n", [1, 4, 8, 12])
def test_parity(n):
    """n-bit parity: no two ON minterms are adjacent, so the primes are its 2^(n-1) ON minterms."""
    t = np.arange(1 << n)
    sup = np.array([bin(x).count("1") % 2 == 1 for x in t])
    S = oracle.sweep(n, bf.bitmap_from_bool(sup))
    assert oracle.count(n, S) == 2 ** (n - 1)
    d = bf.digits(n)
    cells = np.nonzero(S)[0]
    assert np.all(d[cells] != 2)
    assert np.all((d[cells] == 1).sum(axis=1) % 2 == 1)


@pytest.mark.parametrize("n", [3, 7, 11])
def test_single_minterm(n):
    t0 = (0x5A5A5A >> 1) & ((1 << n) - 1)
    sup = np.zeros(1 << n, dtype=bool)
    sup[t0] = True
    S = oracle.sweep(n, bf.bitmap_from_bool(sup))
    rho = sum(((t0 >> i) & 1) * 3 ** i for i in range(n))
    assert np.nonzero(S)[0].tolist() == [rho]


@pytest.mark.parametrize("n", [2, 6, 11])
def test_or_of_variables(n):
    sup = np.arange(1 << n) != 0
    S = oracle.sweep(n, bf.bitmap_from_bool(sup))
    want = sorted((3 ** n - 1) - 3 ** i for i in range(n))  # digit i = 1, others *
    assert np.nonzero(S)[0].tolist() == want


@pytest.mark.parametrize("n,W", [
    (3, {2, 3}),                    # majority
    (7, {4, 5, 6, 7}),              # threshold
    (9, {5, 6, 7, 8, 9}),           # majority of 9
    (10, {0, 3, 4, 5, 9}),
    (12, {1, 2, 6, 7, 8, 12}),
    (11, set(range(1, 12, 2))),     # parity
])
def test_symmetric_closed_form(n, W):
    """Symmetric functions: cell-by-cell closed form and multinomial count."""
    sup = bf.symmetric_support(n, W)
    S = oracle.sweep(n, bf.bitmap_from_bool(sup))
    want = bf.symmetric_prime_cells(n, W)
    assert np.array_equal(S != 0, want)
    assert oracle.count(n, S) == bf.symmetric_prime_count(n, W)


@pytest.mark.parametrize("n,seed", [(5, 1), (8, 2), (10, 3), (12, 4)])
def test_monotone_closed_form(n, seed):
    """A monotone (positive) function's primes are exactly the positive terms
    of its minimal true points (Section 2's prime definition: a smaller
    positive term would be true below a minimal point, and a literal x_i' can
    be dropped from any implicant since raising x_i keeps f true).  The list
    is pinned too: minimal point m gives the pair (m, m)."""
    sup, mins = bf.monotone_case(n, seed)
    S = oracle.sweep(n, bf.bitmap_from_bool(sup))
    assert np.nonzero(S)[0].tolist() == [bf.rho_positive(n, m) for m in mins]
    assert oracle.pairs(n, S).tolist() == [[m, m] for m in mins]


@pytest.mark.parametrize("n,seed,nu", [(6, 11, 0b101101), (9, 12, 0b110010011), (11, 13, 0b01010101010)])
def test_unate_closed_form(n, seed, nu):
    """A unate function (a monotone function with the inputs in nu negated)
    has the monotone closed form with the literals' polarity flipped where nu
    is set, so its primes mix 0 and 1 digits: pinned cell by cell and in the
    list, byte and bit-per-cube modes."""
    sup, want = bf.unate_case(n, seed, nu)
    on = bf.bitmap_from_bool(sup)
    S = oracle.sweep(n, on)
    assert np.nonzero(S)[0].tolist() == [bf.rho_of_pair(n, m, v) for m, v in want]
    assert oracle.pairs(n, S).tolist() == [[m, v] for m, v in want]
    cells = np.zeros(3 ** n, dtype=bool)
    cells[[bf.rho_of_pair(n, m, v) for m, v in want]] = True
    assert np.array_equal(packed_cells(n, on), cells)


@pytest.mark.parametrize("n,seed,nu", [(6, 11, 0b101101), (10, 16, 0b1001110001)])
def test_unate_dont_care_closed_form(n, seed, nu):
    """Don't-cares in closed form: ON = the unate function's minimal true
    points alone, DC = the rest of its true points.  The implicants are those
    of ON u DC (the don't-care reading of the scope), so the primes are the
    unate closed form again; without the don't-cares they would be the ON
    minterms themselves (an antichain has no two adjacent points)."""
    sup, want = bf.unate_case(n, seed, nu)
    on = np.zeros(1 << n, dtype=bool)
    on[[m ^ nu for m, _ in want]] = True
    dc = sup & ~on
    S = oracle.sweep(n, bf.bitmap_from_bool(on), bf.bitmap_from_bool(dc))
    assert oracle.pairs(n, S).tolist() == [[m, v] for m, v in want]
    S0 = oracle.sweep(n, bf.bitmap_from_bool(on))
    assert oracle.count(n, S0) == len(want) and np.array_equal(oracle.pairs(n, S0)[:, 0], np.full(len(want), (1 << n) - 1))


def test_majority_count():
    """Odd-n majority has C(n, (n+1)/2) primes."""
    from math import comb
    for n in (3, 5, 7, 9, 11):
        W = set(range((n + 1) // 2, n + 1))
        S = oracle.sweep(n, bf.bitmap_from_bool(bf.symmetric_support(n, W)))
        assert oracle.count(n, S) == comb(n, (n + 1) // 2)


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("n", [5, 8, 10])
def test_invariants(n):
    """Primes cover the ON set, cover no OFF minterm, form an antichain, and
    every implicant lies under a prime."""
    on, dc = synth.random_function(n, 11, 0.7, 0.1)
    sup = bf.support_of(n, on, dc)
    onb = bf.support_of(n, on)
    S = oracle.sweep(n, on, dc)
    P = oracle.pairs(n, S).astype(np.int64)
    x = np.arange(1 << n, dtype=np.int64)
    cov = np.zeros(1 << n, dtype=bool)
    for m, v in P:
        c = (x & m) == v
        assert np.all(sup[c])          # no OFF minterm
        cov |= c
    assert np.all(cov[onb])            # ON covered
    # antichain: no prime's minterm set contains another's
    for a in range(len(P)):
        for b in range(len(P)):
            if a != b:
                ma, va = P[a]
                mb, vb = P[b]
                assert not ((ma & mb) == ma and (vb & ma) == va)
    imp = bf.implicants(n, sup)
    mask, value = bf.mask_value(n)
    for r in np.nonzero(imp)[0][:400]:
        assert np.any(((P[:, 0] & mask[r]) == P[:, 0]) & ((value[r] & P[:, 0]) == P[:, 1]))


def test_metamorphic_permutation_and_negation():
    n = 7
    rng = np.random.default_rng(5)
    on, _ = synth.random_function(n, 21, 0.65)
    sup = bf.support_of(n, on)
    base = oracle.sweep(n, on) != 0
    perm = rng.permutation(n)
    t = np.arange(1 << n)
    tp = np.zeros_like(t)
    for i, j in enumerate(perm):
        tp |= ((t >> i) & 1) << j
    sup_p = np.zeros_like(sup)
    sup_p[tp] = sup
    got = oracle.sweep(n, bf.bitmap_from_bool(sup_p)) != 0
    idx = bf.perm_digits(n, perm)
    want = np.zeros_like(base)
    want[idx] = base
    assert np.array_equal(got, want)
    # negating x_k swaps digits 0 and 1 at position k
    k = 3
    sup_n = sup[t ^ (1 << k)]
    got = oracle.sweep(n, bf.bitmap_from_bool(sup_n)) != 0
    d = bf.digits(n).astype(np.int64)
    dk = d[:, k]
    swapped = np.arange(3 ** n) + np.where(dk == 0, 1, np.where(dk == 1, -1, 0)) * 3 ** k
    want = np.zeros_like(base)
    want[swapped] = base
    assert np.array_equal(got, want)


def test_dc_monotone():
    """Adding don't-cares never removes an implicant: each old prime lies under a new one."""
    n = 8
    on, _ = synth.random_function(n, 3, 0.6)
    _, dc = synth.random_function(n, 4, 0.6, 0.3)
    P0 = oracle.pairs(n, oracle.sweep(n, on)).astype(np.int64)
    P1 = oracle.pairs(n, oracle.sweep(n, on, dc)).astype(np.int64)
    for m, v in P0:
        assert np.any(((P1[:, 0] & m) == P1[:, 0]) & ((v & P1[:, 0]) == P1[:, 1]))


# ---------------------------------------------------------------- structure

@pytest.mark.parametrize("n", [1, 4, 9])
def test_triple_counts(n):
    """Boolean-circuit theorem (Section 4.1): n * 3^(n-1) triples per operator."""
    on, _ = synth.random_function(n, 1, 0.5)
    _, (merges, reduces) = oracle.sweep(n, on, return_counts=True)
    assert merges == n * 3 ** (n - 1) and reduces == merges


def test_threads_agree():
    on, dc = synth.random_function(14, 9, 0.8, 0.1)
    cores = oracle.max_threads()
    a = oracle.sweep(14, on, dc, threads=1)
    assert oracle.max_threads() == cores   # the thread count applies to that call only
    b = oracle.sweep(14, on, dc, threads=0)
    assert np.array_equal(a, b)


def test_pointwise_matches_sweep():
    """The pointwise definition agrees with the sweep on every cell (n = 8)
    and on a sample of cells (n = 14)."""
    for n, sample in ((8, None), (14, 20000)):
        on, dc = synth.random_function(n, 5, 0.8, 0.05)
        S = oracle.sweep(n, on, dc) != 0
        rhos = np.arange(3 ** n) if sample is None else \
            np.random.default_rng(0).integers(0, 3 ** n, sample)
        rhos = np.concatenate([rhos, np.nonzero(S)[0][:2000]])
        got = oracle.is_prime_many(n, on, dc, rhos)
        assert np.array_equal(got, S[rhos])


def test_bitmap_layout():
    """Bitmap bit rho sits in byte rho >> 3 at position rho & 7; bits past 3^n are 0."""
    n = 5
    on, _ = synth.random_function(n, 2, 0.7)
    S = oracle.sweep(n, on)
    bm = oracle.bitmap(n, S)
    assert bm.size == (3 ** n + 7) // 8
    bits = np.unpackbits(bm, bitorder="little")
    assert np.array_equal(bits[: 3 ** n].astype(bool), S != 0)
    assert not bits[3 ** n:].any()


# ---------------------------------------------------------------- statistics

def test_expected_counts_formula_small():
    """E[#implicants], E[#primes] for i.i.d. Bernoulli(p) support: exact average over
    all functions of n = 3 weighted by p (the formula is exact, not asymptotic)."""
    n, p = 3, 0.6
    e_imp = e_pr = 0.0
    for f, sup in bf.all_functions(n):
        k = int(sup.sum())
        w = p ** k * (1 - p) ** ((1 << n) - k)
        e_imp += w * bf.implicants(n, sup).sum()
        e_pr += w * (oracle_cells(n, sup)).sum()
    assert abs(e_imp - bf.expected_implicants(n, p)) < 1e-9
    assert abs(e_pr - bf.expected_primes(n, p)) < 1e-9


def test_expected_prime_count_band():
    """n = 14, p = 0.7: mean prime count over seeds within 3% of the expectation."""
    n, p = 14, 0.7
    counts = []
    for seed in range(1, 5):
        on, _ = synth.random_function(n, seed, p)
        counts.append(oracle.count(n, oracle.sweep(n, on)))
    e = bf.expected_primes(n, p)
    assert abs(np.mean(counts) - e) / e < 0.03


# ---------------------------------------------------------------- packed mode

def test_packed_pairs_equal_byte_pairs():
    """The packed mode's list equals the byte mode's (ascending rho, same encoding)."""
    for n, seed, p, q in ((0, 1, 0.9, 0.0), (3, 1, 0.7, 0.0), (9, 2, 0.8, 0.05), (14, 1, 0.85, 0.0),
                          (16, 3, 0.5, 0.2)):
        on, dc = synth.random_function(n, seed, p, q)
        want = oracle.pairs(n, oracle.sweep(n, on, dc))
        assert np.array_equal(oracle.packed_pairs(n, oracle.sweep_packed(n, on, dc)), want), n


def packed_cells(n, on, dc=None, threads=0):
    return bf.bool_from_bitmap(oracle.packed_bitmap(n, oracle.sweep_packed(n, on, dc, threads)), n)


@pytest.mark.parametrize("n", list(range(0, 9)))
def test_packed_bruteforce_random(n):
    """Packed mode against the definitions (Section 2) by enumeration, n <= 8,
    with and without don't-cares."""
    for seed in range(1, 4):
        for p, p_dc in ((0.4, 0.0), (0.7, 0.15), (0.92, 0.0)):
            on, dc = synth.random_function(n, seed, p, p_dc)
            want = bf.primes(n, bf.support_of(n, on, dc))
            assert np.array_equal(packed_cells(n, on, dc), want), (n, seed, p)


@pytest.mark.parametrize("n,W", [(9, {5, 6, 7, 8, 9}), (12, {1, 2, 6, 7, 8, 12}), (13, set(range(1, 14, 2)))])
def test_packed_symmetric_closed_form(n, W):
    """Symmetric functions in closed form at sizes where runs of a digit are
    both shorter and longer than a 64-cube word."""
    cells = packed_cells(n, bf.bitmap_from_bool(bf.symmetric_support(n, W)))
    assert np.array_equal(cells, bf.symmetric_prime_cells(n, W))


@pytest.mark.parametrize("n,seed", [(7, 5), (9, 6)])
def test_packed_monotone_closed_form(n, seed):
    """The monotone closed form (primes = positive terms of the minimal true
    points) in the bit-per-cube mode."""
    sup, mins = bf.monotone_case(n, seed)
    want = np.zeros(3 ** n, dtype=bool)
    want[[bf.rho_positive(n, m) for m in mins]] = True
    assert np.array_equal(packed_cells(n, bf.bitmap_from_bool(sup)), want)


def test_packed_constant_one_and_tail():
    """f = 1 (Section 3): only the all-* cube; the bits past 3^n stay 0."""
    for n in (4, 11):
        bm = oracle.packed_bitmap(n, oracle.sweep_packed(n, np.full(synth.tt_bytes(n), 0xFF, dtype=np.uint8)))
        cells = np.nonzero(np.unpackbits(bm, bitorder="little"))[0].tolist()
        assert cells == [3 ** n - 1]


@pytest.mark.parametrize("n", [10, 13, 15])
def test_packed_equals_byte_sweep(n):
    """The two storage modes give the same primes, on one thread and on all."""
    on, dc = synth.random_function(n, 40 + n, 0.8, 0.1)
    want = oracle.bitmap(n, oracle.sweep(n, on, dc))
    assert np.array_equal(oracle.packed_bitmap(n, oracle.sweep_packed(n, on, dc, threads=1)), want)
    assert np.array_equal(oracle.packed_bitmap(n, oracle.sweep_packed(n, on, dc)), want)


# ---------------------------------------------------------------- stored digests

def _make_digests():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_digests", os.path.join(GOLDEN, "make_digests.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_digest_script_matches_byte_oracle():
    """The script that stores the large-n digests, run at small n, gives the
    SHA-256 and count of the byte oracle's bitmap."""
    import hashlib
    md = _make_digests()
    for n, seed, p, q in ((9, 2, 0.8, 0.05), (14, 1, 0.85, 0.0)):
        h, c, hl = md.digest(n, seed, p, q)
        on, dc = synth.random_function(n, seed, p, q)
        S = oracle.sweep(n, on, dc)
        assert h == hashlib.sha256(oracle.bitmap(n, S).tobytes()).hexdigest()
        assert c == oracle.count(n, S)
        assert hl == hashlib.sha256(oracle.pairs(n, S).astype("<u4").tobytes()).hexdigest()


def test_stored_digest_counts_near_expectation():
    """Each stored count is within 1% of the exact expected prime count for
    i.i.d. support of its density (ON, plus DC on the OFF minterms)."""
    path = os.path.join(GOLDEN, "bitmap_digests.txt")
    if not os.path.exists(path):
        pytest.skip("no stored digests")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert rows
    for n, seed, p_on, p_dc, count, h, hl in rows:
        n, p_on, p_dc, count = int(n), float(p_on), float(p_dc), int(count)
        assert len(h) == len(hl) == 64 and int(h, 16) >= 0 and int(hl, 16) >= 0
        e = bf.expected_primes(n, p_on + (1 - p_on) * p_dc)
        assert abs(count - e) / e < 0.01, (n, count, e)


# ------------------------------------------------------ complement (CNF) mode

@pytest.mark.parametrize("n,W,Wdc", [
    (3, {2, 3}, set()),             # not-majority: primes 00*, 0*0, *00
    (7, {4, 5, 6, 7}, set()),
    (10, {0, 3, 4, 5, 9}, {1, 8}),
    (11, set(range(1, 12, 2)), set()),   # not-parity is even parity
])
def test_complement_symmetric_closed_form(n, W, Wdc):
    """Section 1: the primes of not-f give f's prime CNF (De Morgan).  The
    complement of a symmetric function with ON weights W and don't-care
    weights Wdc is symmetric with support weights ({0..n} - W) | Wdc, so its
    primes have the same closed form.  The complement's tables are built the
    way the library forms them: ON' = not(ON or DC), DC' = DC."""
    on = bf.symmetric_support(n, W)
    dc = bf.symmetric_support(n, Wdc) & ~on
    S = oracle.sweep(n, bf.bitmap_from_bool(~on & ~dc), bf.bitmap_from_bool(dc))
    Wc = (set(range(n + 1)) - W) | Wdc
    assert np.array_equal(S != 0, bf.symmetric_prime_cells(n, Wc))
    if n == 3 and not Wdc:
        got = sorted(bf.cube_string(n, r) for r in np.nonzero(S)[0])
        assert got == sorted(["00*", "0*0", "*00"])


def test_complement_of_constant_zero_is_constant_one():
    """not(0) = 1: the only prime is the all-'*' cube (Section 3)."""
    n = 6
    S = oracle.sweep(n, bf.bitmap_from_bool(np.ones(1 << n, dtype=bool)))
    assert np.nonzero(S)[0].tolist() == [3 ** n - 1]
