"""The (mask, value) list at n = 22 by closed forms.  Each bitmap tile's
pairs are placed by a decoupled look-back over the tiles before it (in the
order the tiles start); a tile whose 96-row regions hold more pairs than their
shared-memory slots lists itself from the bitmap it wrote.

For a parity function every prime is an ON minterm of the variables it
depends on, with '*' on the others, and the list is those minterms in
ascending order (rho grows with the minterm's number when the '*' digits are
fixed); a band function of ten variables with the other twelve fixed to 1 puts
4200 primes into a few regions of one tile deep in the sweep.  The list also
equals the library's separate compaction of the bitmap.  A truncated list and
a list in pinned host memory at n = 22 are checked in test_gpu_parity.py."""
import numpy as np
import pytest

import oracle
from paper_2302_10083_gb300 import dqmc, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dqmc.lib()
    yield
    dqmc.dqmc_release()


def parity_bits(n, k):
    """x0 xor ... xor x(k-1) for every minterm of n variables (bool array)."""
    m = np.arange(1 << n, dtype=np.uint32)
    par = np.zeros(1 << n, dtype=np.uint32)
    for i in range(k):
        par ^= (m >> i) & 1
    return par.astype(bool)


def test_parity_n22_every_minterm_listed():
    """Parity of all 22 variables: the 2^21 odd minterms, 2^7 * 2^5 / 2 = 2048
    in each bitmap tile whose fixed digits are all 0/1 and none in the others."""
    n = 22
    bits = parity_bits(n, n)
    pairs, count = dqmc.dqmc_list(n, synth.pack(bits), cap=1 << 21)
    assert count == 1 << 21
    want = np.nonzero(bits)[0].astype(np.uint32)
    assert np.array_equal(pairs[:, 0], np.full(count, (1 << n) - 1, np.uint32))
    assert np.array_equal(pairs[:, 1], want)
    assert dqmc.dqmc_count(n, synth.pack(bits)) == count


def test_parity_of_low_variables_n22_one_tile():
    """Parity of x0 .. x11 over 22 variables: 2^11 primes, each an odd
    minterm of x0 .. x11 with '*' on x12 .. x21, all in the last bitmap tile."""
    n, k = 22, 12
    bits = parity_bits(n, k)
    pairs, count = dqmc.dqmc_list(n, synth.pack(bits), cap=1 << 12)
    assert count == 1 << (k - 1)
    m = np.arange(1 << k, dtype=np.uint32)
    want = m[parity_bits(k, k)]
    assert np.array_equal(pairs[:, 0], np.full(count, (1 << k) - 1, np.uint32))
    assert np.array_equal(pairs[:, 1], want)


@pytest.mark.parametrize("p_on", [0.55, 0.97])
def test_list_matches_bitmap_compaction_n22(p_on):
    """The list equals the library's separate compaction of the same
    sweep's bitmap (dqmc_compact_dev, a scan over the bitmap words that shares
    no code with the bitmap pass), for random functions of two ON densities."""
    n = 22
    on, dc = synth.random_function(n, 60, p_on, 0.02)
    want_pairs, want_count = dqmc.dqmc_list(n, on, dc)
    bm = dqmc.dqmc_primes(n, on, dc)
    dev = torch.device("cuda")
    d_bm = torch.from_numpy(bm).to(dev)
    cap = want_count
    d_pairs = torch.empty(2 * max(cap, 1), dtype=torch.int32, device=dev)
    d_count = torch.zeros(1, dtype=torch.int64, device=dev)
    work_bytes = dqmc.dqmc_workspace_bytes(n)
    work = torch.empty(work_bytes, dtype=torch.uint8, device=dev)
    L = dqmc.lib()
    st = L.dqmc_compact_dev(n, d_bm.data_ptr(), d_pairs.data_ptr(), cap, d_count.data_ptr(), work.data_ptr(),
                            work_bytes, None)
    torch.cuda.synchronize()
    assert st == dqmc.DQMC_OK
    assert int(d_count.item()) == want_count
    got = d_pairs.cpu().numpy().view(np.uint32)[: 2 * cap].reshape(cap, 2)
    assert np.array_equal(got, want_pairs)


def test_overflowing_tile_deep_in_the_sweep_n22():
    """f = [3 <= weight(x0 .. x9) <= 6] and x10 .. x21 all 1 (else 0): the
    primes are the band's C(10, 3) * C(7, 4) = 4200 primes of x0 .. x9 with
    the twelve literals x10 .. x21 = 1, all in bitmap tile 29524 (fixed digits
    x12 .. x21 = 1) at tile rows 972 + (0 .. 242) (x10 = x11 = 1).  Some of its
    96-row regions hold more than 12 * 32 pairs, so that tile lists itself
    from its bitmap."""
    n, k = 22, 10
    x = np.arange(1 << k)
    w = np.zeros(x.size, dtype=np.int64)
    for i in range(k):
        w += (x >> i) & 1
    band = (w >= 3) & (w <= 6)
    on_k = synth.pack(band)
    band_pairs = oracle.pairs(k, oracle.sweep(k, on_k))
    assert len(band_pairs) == 120 * 35
    high = ((1 << n) - 1) ^ ((1 << k) - 1)
    bits = np.zeros(1 << n, dtype=bool)
    bits[high | x[band]] = True
    want = band_pairs.copy()
    want[:, 0] |= np.uint32(high)
    want[:, 1] |= np.uint32(high)
    # where the primes fall: rho, its row, the row's tile and 96-row region
    rho = np.zeros(len(want), dtype=np.int64)
    for i in range(n):
        lit = (want[:, 0] >> i) & 1
        one = (want[:, 1] >> i) & 1
        rho += np.where(lit == 1, one, 2).astype(np.int64) * 3 ** i
    row = rho // 243
    assert set((row // 2187).tolist()) == {(3 ** 10 - 1) // 2}
    assert np.bincount((row % 2187) // 96).max() > 12 * 32
    pairs, count = dqmc.dqmc_list(n, synth.pack(bits), cap=8192)
    assert count == len(want)
    assert np.array_equal(pairs, want)
