"""SparseQMC on the GPU (dqmc_sparse_list, Section 5) through the C ABI:
the same primes, in the same ascending-rho (mask, value) list, as the oracle
and as the dense sweep."""
import numpy as np
import pytest

import bruteforce as bf
import oracle
from paper_2302_10083_gb300 import dqmc, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dqmc.lib()


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 6, 9, 12, 13, 16])
def test_sparse_matches_oracle(n):
    for seed, (p, q) in enumerate(((0.2, 0.0), (0.5, 0.1), (0.9, 0.0))):
        on, dc = synth.random_function(n, 80 + seed + n, p, q)
        want = oracle.pairs(n, oracle.sweep(n, on, dc))
        got, c = dqmc.dqmc_sparse_list(n, on, dc, cap=len(want) + 4)
        assert c == len(want)
        assert np.array_equal(got, want)      # bit-exact, same order


def test_sparse_n20_workload_and_complement():
    """n = 20 (ON 0.7, DC 0.1), and the complement mode, against the oracle."""
    on, dc = synth.single_n20(1)
    want = oracle.pairs(20, oracle.sweep(20, on, dc))
    got, c = dqmc.dqmc_sparse_list(20, on, dc)
    assert c == len(want) and np.array_equal(got, want)
    on_c = (~(on | dc)).astype(np.uint8)
    want_c = oracle.pairs(20, oracle.sweep(20, on_c, dc))
    got_c, cc = dqmc.dqmc_sparse_list(20, on, dc, flags=dqmc.DQMC_COMPLEMENT)
    assert cc == len(want_c) and np.array_equal(got_c, want_c)


@pytest.mark.parametrize("n,p", [(22, 0.3), (23, 0.5)])
def test_sparse_matches_dense(n, p):
    """Larger n: the sparse list equals the dense sweep's list (which is
    bit-exact against the oracle's digests at these sizes)."""
    on, _ = synth.random_function(n, 5, p)
    want, c0 = dqmc.dqmc_list(n, on)
    got, c = dqmc.dqmc_sparse_list(n, on, cap=c0)
    assert c == c0 and np.array_equal(got, want)


def test_sparse_closed_forms():
    """Parity (its minterms), constant 1 (only *...*), constant 0 (none), and
    n = 27 beyond the dense range: a single minterm."""
    n = 14
    t = np.arange(1 << n)
    par = bf.bitmap_from_bool(np.array([bin(x).count("1") % 2 == 1 for x in t]))
    got, c = dqmc.dqmc_sparse_list(n, par)
    assert c == 2 ** (n - 1) and np.all(got[:, 0] == (1 << n) - 1)
    ones = np.full(synth.tt_bytes(n), 0xFF, dtype=np.uint8)
    got, c = dqmc.dqmc_sparse_list(n, ones)
    assert c == 1 and got.tolist() == [[0, 0]]
    assert dqmc.dqmc_sparse_list(n, np.zeros_like(ones))[1] == 0
    n = 27
    on = np.zeros(synth.tt_bytes(n), dtype=np.uint8)
    t0 = 0x5A5A5A5 & ((1 << n) - 1)
    on[t0 >> 3] = 1 << (t0 & 7)
    got, c = dqmc.dqmc_sparse_list(n, on)
    assert c == 1 and got.tolist() == [[(1 << n) - 1, t0]]
