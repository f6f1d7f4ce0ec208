"""dqmc_cover (the second step of the Quine-McCluskey method, Section 1: a
cover of the ON-set by primes; essentials, then greedy) through the C ABI,
against the same rule restated on the host: the selection must be identical,
and it must cover every ON minterm with primes only."""
import numpy as np
import pytest

import oracle
from paper_2302_10083_gb300 import dqmc, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def minterms_of(n, m, v):
    free = [i for i in range(n) if not (m >> i) & 1]
    out = []
    for k in range(1 << len(free)):
        t = v
        for j, i in enumerate(free):
            if (k >> j) & 1:
                t |= 1 << i
        out.append(t)
    return out


def host_cover(n, on, dc, pairs):
    """Essential primes, then the prime covering the most uncovered ON
    minterms (ties: lowest index), until the ON-set is covered."""
    sup_on = np.unpackbits(on, bitorder="little")[: 1 << n].astype(bool)
    sup_dc = np.zeros_like(sup_on) if dc is None else np.unpackbits(dc, bitorder="little")[: 1 << n].astype(bool)
    todo = sup_on & ~sup_dc
    cov = [minterms_of(n, int(m), int(v)) for m, v in pairs]
    who = {}
    cnt = np.zeros(1 << n, dtype=np.int64)
    for p, ts in enumerate(cov):
        for t in ts:
            if todo[t]:
                cnt[t] += 1
                who.setdefault(t, p)
    sel = set(who[t] for t in range(1 << n) if todo[t] and cnt[t] == 1)
    for p in sel:
        todo[cov[p]] = False
    while todo.any():
        best, bp = 0, -1
        for p, ts in enumerate(cov):
            if p in sel:
                continue
            c = int(todo[ts].sum())
            if c > best:
                best, bp = c, p
        sel.add(bp)
        todo[cov[bp]] = False
    return sorted(sel)


@pytest.mark.parametrize("n,p,q", [(0, 0.9, 0.0), (3, 0.6, 0.0), (6, 0.5, 0.1), (8, 0.7, 0.0), (10, 0.5, 0.05)])
def test_cover_matches_host_rule(n, p, q):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    on, dc = synth.random_function(n, 90 + n, p, q)
    pairs = oracle.pairs(n, oracle.sweep(n, on, dc))
    got = dqmc.dqmc_cover(n, on, dc, pairs)
    assert got.tolist() == host_cover(n, on, dc, pairs)


@pytest.mark.parametrize("n", [14, 18])
def test_cover_is_a_cover(n):
    """Larger n: every selected cube is one of the primes and the selection
    covers every ON minterm and no OFF minterm; the essential primes are in it."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    on, dc = synth.random_function(n, 3, 0.6, 0.05)
    pairs, c = dqmc.dqmc_list(n, on, dc)
    sel = dqmc.dqmc_cover(n, on, dc, pairs)
    assert 0 < len(sel) <= c and np.all(np.diff(sel) > 0)
    sup_on = np.unpackbits(on, bitorder="little")[: 1 << n].astype(bool)
    sup_dc = np.unpackbits(dc, bitorder="little")[: 1 << n].astype(bool)
    covered = np.zeros(1 << n, dtype=bool)
    t = np.arange(1 << n, dtype=np.int64)
    for m, v in pairs[sel]:
        covered |= (t & int(m)) == int(v)
    assert np.all(covered[sup_on & ~sup_dc])
    assert not np.any(covered & ~(sup_on | sup_dc))


def test_cover_refuses_a_non_cover():
    n = 4
    on = np.array([0xFF, 0x00], dtype=np.uint8)      # x4 = 0
    pairs = np.array([[0b1001, 0b0000]], dtype=np.uint32)   # covers only minterms with x1 = x4 = 0
    with pytest.raises(dqmc.DqmcError):
        dqmc.dqmc_cover(n, on, None, pairs)
