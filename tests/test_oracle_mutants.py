"""The pins must catch plausible mistakes in the oracle.

Each case compiles a copy of ``oracle/dqmc_oracle.c`` with one planted mistake
(a dropped term, a wrong index, a wrong operator, a skipped digit, an ignored
don't-care set; in the packed mode a wrong sibling, a digit that does not
wrap, a skipped word, a wrong byte order) and checks that brute force (Section 2 definitions) or a worked
example rejects it.  Everything runs on the CPU.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import bruteforce as bf
from paper_2302_10083_gb300 import synth

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "dqmc_oracle.c")

MUTANTS = {
    "reduce_drops_t": ("S[it] = (uint8_t)(S[it] & !z);", ""),
    "merge_or": ("S[iu] | (S[is] & S[it])", "S[iu] | (S[is] | S[it])"),
    "merge_wrong_operand": ("S[iu] | (S[is] & S[it])", "S[iu] | (S[is] & S[is])"),
    "skip_last_digit": ("for (int i = 1; i <= n; ++i) {\n        const uint64_t dd = d;\n"
                        "        #pragma omp parallel for schedule(static) reduction(+:reduces)",
                        "for (int i = 1; i < n; ++i) {\n        const uint64_t dd = d;\n"
                        "        #pragma omp parallel for schedule(static) reduction(+:reduces)"),
    "ignore_dc": ("(dc ? tt_bit(dc, t) : 0)", "0"),
    "load_bit_order": ("if ((t >> i) & 1) r += w;", "if ((t >> (n - 1 - i)) & 1) r += w;"),
    "reduce_reads_wrong_cell": ("const uint8_t z = S[iu];", "const uint8_t z = S[it];"),
}

# mistakes in the packed (bit per cube) mode
PACKED_MUTANTS = {
    "packed_merge_same_sibling": ("pk_get(S, r - 2 * dd) && pk_get(S, r - dd)",
                                  "pk_get(S, r - 2 * dd) && pk_get(S, r - 2 * dd)"),
    "packed_reduce_wrong_sibling": ("pk_get(S, r + (2u - digit) * dd)", "pk_get(S, r + (1u + digit) * dd)"),
    "packed_digit_no_wrap": ("digit = (digit + 1u) % 3u;", "digit = digit + 1u;"),
    "packed_last_word_skipped": ("for (uint64_t w = 0; w < W; ++w) {", "for (uint64_t w = 0; w < W - 1; ++w) {"),
    "packed_bitmap_byte_order": ("(uint8_t)(S[k >> 3] >> (8 * (k & 7)))",
                                 "(uint8_t)(S[k >> 3] >> (8 * (7 - (k & 7))))"),
}


def build_mutant(tmp_path, name):
    old, new = {**MUTANTS, **PACKED_MUTANTS}[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    src = src.replace(old, new, 1)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O1", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", str(so), str(c)],
                   check=True)
    L = ctypes.CDLL(str(so))
    u8p = ctypes.POINTER(ctypes.c_uint8)
    L.oracle_sweep.argtypes = [ctypes.c_int, u8p, u8p, u8p, ctypes.c_int,
                               ctypes.POINTER(ctypes.c_uint64)]
    L.oracle_sweep.restype = None
    u64p = ctypes.POINTER(ctypes.c_uint64)
    L.oracle_sweep_packed.argtypes = [ctypes.c_int, u8p, u8p, u64p, ctypes.c_int]
    L.oracle_sweep_packed.restype = None
    L.oracle_packed_bitmap.argtypes = [ctypes.c_int, u64p, u8p]
    L.oracle_packed_bitmap.restype = None

    if name in PACKED_MUTANTS:
        def sweep_packed(n, on, dc=None):
            S = np.empty((3 ** n + 63) // 64, dtype=np.uint64)
            bm = np.empty((3 ** n + 7) // 8, dtype=np.uint8)
            on = np.ascontiguousarray(on, dtype=np.uint8)
            dcp = None if dc is None else np.ascontiguousarray(dc, dtype=np.uint8)
            L.oracle_sweep_packed(n, on.ctypes.data_as(u8p), None if dcp is None else dcp.ctypes.data_as(u8p),
                                  S.ctypes.data_as(u64p), 2)
            L.oracle_packed_bitmap(n, S.ctypes.data_as(u64p), bm.ctypes.data_as(u8p))
            return bf.bool_from_bitmap(bm, n)
        return sweep_packed

    def sweep(n, on, dc=None):
        S = np.empty(3 ** n, dtype=np.uint8)
        cnt = (ctypes.c_uint64 * 2)()
        on = np.ascontiguousarray(on, dtype=np.uint8)
        dcp = None if dc is None else np.ascontiguousarray(dc, dtype=np.uint8)
        L.oracle_sweep(n, on.ctypes.data_as(u8p),
                       None if dcp is None else dcp.ctypes.data_as(u8p),
                       S.ctypes.data_as(u8p), 1, cnt)
        return S != 0
    return sweep


def pins_pass(sweep):
    """A subset of the pins: brute force with and without don't-cares, majority."""
    for n in (3, 5, 6):
        for seed in (1, 2):
            on, dc = synth.random_function(n, seed, 0.6, 0.25)
            for d in (None, dc):
                want = bf.primes(n, bf.support_of(n, on, d))
                if not np.array_equal(sweep(n, on, d), want):
                    return False
    on = bf.bitmap_from_bool(bf.symmetric_support(3, {2, 3}))
    got = np.nonzero(sweep(3, on))[0].tolist()
    return got == [14, 16, 22]


def test_unmutated_copy_passes(tmp_path):
    old = MUTANTS["ignore_dc"][0]
    MUTANTS["_identity"] = (old, old)
    try:
        assert pins_pass(build_mutant(tmp_path, "_identity"))
    finally:
        del MUTANTS["_identity"]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    assert not pins_pass(build_mutant(tmp_path, name)), name


def test_unmutated_packed_copy_passes(tmp_path):
    old = PACKED_MUTANTS["packed_digit_no_wrap"][0]
    PACKED_MUTANTS["_packed_identity"] = (old, old)
    try:
        assert pins_pass(build_mutant(tmp_path, "_packed_identity"))
    finally:
        del PACKED_MUTANTS["_packed_identity"]


@pytest.mark.parametrize("name", sorted(PACKED_MUTANTS))
def test_packed_mutant_is_caught(tmp_path, name):
    assert not pins_pass(build_mutant(tmp_path, name)), name


def unate_pin_passes(sweep):
    """The unate closed forms alone (no brute force): the function itself, and
    its minimal true points as ON with the other true points as don't-cares."""
    for n, seed, nu in ((6, 11, 0b101101), (9, 12, 0b110010011), (11, 13, 0b01010101010)):
        sup, want = bf.unate_case(n, seed, nu)
        rho = [bf.rho_of_pair(n, m, v) for m, v in want]
        if np.nonzero(sweep(n, bf.bitmap_from_bool(sup)))[0].tolist() != rho:
            return False
        on = np.zeros(1 << n, dtype=bool)
        on[[m ^ nu for m, _ in want]] = True
        got = sweep(n, bf.bitmap_from_bool(on), bf.bitmap_from_bool(sup & ~on))
        if np.nonzero(got)[0].tolist() != rho:
            return False
    return True


def test_unate_pin_passes_unmutated(tmp_path):
    old = MUTANTS["ignore_dc"][0]
    MUTANTS["_identity"] = (old, old)
    try:
        assert unate_pin_passes(build_mutant(tmp_path, "_identity"))
    finally:
        del MUTANTS["_identity"]


@pytest.mark.parametrize("name", sorted(set(MUTANTS) | set(PACKED_MUTANTS)))
def test_unate_pin_alone_catches(tmp_path, name):
    """An independent second net: the unate closed forms (with and without
    don't-cares) catch every planted mistake on their own."""
    assert not unate_pin_passes(build_mutant(tmp_path, name)), name
