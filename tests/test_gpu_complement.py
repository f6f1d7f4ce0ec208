"""Complement (CNF) mode through the C ABI: dqmc_primes_ex / dqmc_list_ex /
dqmc_list_dev_ex with DQMC_COMPLEMENT give the oracle's primes of not-f,
whose support is (not ON) or DC (Section 1, the DNF / CNF duality)."""
import numpy as np
import pytest

import bruteforce as bf
import oracle
from paper_2302_10083_gb300 import dqmc, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _complement_tables(n, on, dc):
    """ON' = not(ON or DC), DC' = DC as byte tables (tail bits are ignored)."""
    m = ((1 << n) + 7) >> 3
    on_b = np.asarray(on, dtype=np.uint8)[:m]
    dc_b = np.zeros(m, dtype=np.uint8) if dc is None else np.asarray(dc, dtype=np.uint8)[:m]
    return (~(on_b | dc_b)).astype(np.uint8), (None if dc is None else dc_b)


def _want(n, on, dc):
    on_c, dc_c = _complement_tables(n, on, dc)
    S = oracle.sweep(n, on_c, dc_c)
    return oracle.bitmap(n, S), oracle.count(n, S), oracle.pairs(n, S)


@pytest.mark.parametrize("n,p,q", [(0, 0.5, 0.0), (1, 0.5, 0.0), (2, 0.3, 0.2), (3, 0.6, 0.0), (4, 0.5, 0.1),
                                   (5, 0.4, 0.0), (8, 0.3, 0.1), (12, 0.2, 0.0), (13, 0.25, 0.1),
                                   (14, 0.15, 0.0), (16, 0.2, 0.05), (19, 0.15, 0.0)])
def test_complement_host_api(n, p, q):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    on, dc = synth.random_function(n, 7 + n, p, q)
    want_bm, want_c, want_pairs = _want(n, on, dc)
    bm, c = dqmc.dqmc_primes_ex(n, on, dc, dqmc.DQMC_COMPLEMENT)
    assert c == want_c
    assert np.array_equal(bm, want_bm)        # integer results: bit-exact
    pairs, c2 = dqmc.dqmc_list_ex(n, on, dc, dqmc.DQMC_COMPLEMENT, cap=want_c)
    assert c2 == want_c
    assert np.array_equal(pairs, want_pairs)
    # flags 0 is the plain sweep
    bm0, c0 = dqmc.dqmc_primes_ex(n, on, dc, 0)
    assert np.array_equal(bm0, dqmc.dqmc_primes(n, on, dc)) and c0 == dqmc.dqmc_count(n, on, dc)


def test_complement_device_api_list():
    """dqmc_list_dev_ex on device buffers (a multi-pass plan: n = 17)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = 17
    on, dc = synth.random_function(n, 3, 0.2, 0.1)
    want_bm, want_c, want_pairs = _want(n, on, dc)
    buf = dqmc.DeviceBuffers(n, with_dc=True, cap=want_c)
    buf.on[: on.size].copy_(torch.from_numpy(on))
    buf.dc[: dc.size].copy_(torch.from_numpy(dc))
    sh = torch.cuda.current_stream().cuda_stream
    st = dqmc.lib().dqmc_list_dev_ex(n, buf.on.data_ptr(), buf.dc.data_ptr(), dqmc.DQMC_COMPLEMENT,
                                     buf.bitmap.data_ptr(), buf.pairs.data_ptr(), want_c, buf.count.data_ptr(),
                                     buf.work.data_ptr(), buf.work_bytes, sh)
    assert st == dqmc.DQMC_OK
    assert buf.status() == dqmc.DQMC_OK
    assert int(buf.count.item()) == want_c
    assert np.array_equal(buf.bitmap[: want_bm.size].cpu().numpy(), want_bm)
    got = buf.pairs[: 2 * want_c].cpu().numpy().view(np.uint32).reshape(-1, 2)
    assert np.array_equal(got, want_pairs)


@pytest.mark.parametrize("n", [3, 9, 14])
def test_complement_majority_closed_form(n):
    """not-majority is the symmetric function of weights 0 .. (n-1)/2."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    W = set(range((n + 1) // 2, n + 1))
    on = bf.bitmap_from_bool(bf.symmetric_support(n, W))
    bm, c = dqmc.dqmc_primes_ex(n, on, None, dqmc.DQMC_COMPLEMENT)
    Wc = set(range(n + 1)) - W
    assert c == bf.symmetric_prime_count(n, Wc)
    assert np.array_equal(bf.bool_from_bitmap(bm, n), bf.symmetric_prime_cells(n, Wc))
