"""Host model of SparseQMC's level procedure (Section 5, "SparseQMC", on
Algorithm 1), the rules the GPU kernels of csrc/dqmc_sparse.cu follow, with
Python sets in place of the hash sets:
  - a cube is a 2n-bit code, 00 = '0', 01 = '1', 10 = '*' per variable;
  - level w: for s in L_{w-1} and a position i with s_i = '0' and no
    wildcard before i, if s with '1' at i is in L_{w-1}, s with '*' at i
    joins L_w (each new implicant is made once: from its first wildcard);
  - then every u in L_w flags both of its merge pairs, at every wildcard
    position, redundant in L_{w-1} (the extra pass the rule needs);
  - the unflagged cubes of each level are the primes.
Checked against the oracle (Algorithm 3) and Section 2's definitions, and a
negative case: without the extra marking pass, non-primes survive."""
import numpy as np
import pytest

import bruteforce as bf
import oracle
from paper_2302_10083_gb300 import synth


def spread2(t, n):
    return sum(((t >> i) & 1) << (2 * i) for i in range(n))


def sparse_primes(n, support, mark_all_pairs=True):
    cur = {spread2(t, n) for t in range(1 << n) if support[t]}
    primes, made = [], 0
    for w in range(1, n + 2):
        if not cur:
            break
        nxt = set()
        if w <= n:
            for s in cur:
                for i in range(n):
                    sym = (s >> (2 * i)) & 3
                    if sym == 2:
                        break
                    if sym == 0 and (s | (1 << (2 * i))) in cur:
                        u = s | (2 << (2 * i))
                        assert u not in nxt   # made once
                        nxt.add(u)
                        made += 1
        red = set()
        for u in nxt:
            for j in range(n):
                if (u >> (2 * j)) & 3 != 2:
                    continue
                if not mark_all_pairs and any((u >> (2 * k)) & 3 == 2 for k in range(j)):
                    continue      # only the pair the cube was made from
                s0 = u & ~(3 << (2 * j))
                red.add(s0)
                red.add(s0 | (1 << (2 * j)))
        primes += [c for c in cur if c not in red]
        cur = nxt
    rho = sorted(sum(((c >> (2 * i)) & 3) * 3 ** i for i in range(n)) for c in primes)
    return rho


def oracle_rho(n, support):
    S = oracle.sweep(n, bf.bitmap_from_bool(support))
    return np.nonzero(S)[0].tolist()


@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 7, 8])
def test_sparse_model_matches_oracle(n):
    for seed in range(6):
        for p in (0.2, 0.5, 0.8):
            on, _ = synth.random_function(n, seed + 10 * n, p)
            sup = np.unpackbits(on, bitorder="little")[: 1 << n].astype(bool)
            assert sparse_primes(n, sup) == oracle_rho(n, sup), (n, seed, p)


def test_sparse_model_every_function_n3():
    for _, sup in bf.all_functions(3):
        assert sparse_primes(3, sup) == np.nonzero(bf.primes(3, sup))[0].tolist()


def test_sparse_model_needs_the_marking_pass():
    """Marking only the pair a cube was made from leaves non-primes: for the
    constant 1 on two variables, ** is made only from (0*, 1*) (its first
    wildcard), so *0 and *1 would stay; the full pass leaves only **."""
    n = 2
    sup = np.ones(4, dtype=bool)
    assert sparse_primes(n, sup) == [8]
    assert sparse_primes(n, sup, mark_all_pairs=False) != [8]
