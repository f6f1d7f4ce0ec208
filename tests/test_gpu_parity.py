"""GPU parity: libdqmc.so (through its C ABI) against the CPU oracle.

Bit-exact on the prime bitmap, the count and the (mask, value) list.  Small
and medium n are compared element by element (up to n = 21 against the
byte-per-cube oracle; n = 22 against its bit-per-cube mode in
test_zz_parity_n22_exact.py); n = 22 .. 25,
with n = 24 the full-size workload, are also checked on sampled cells with the
oracle's pointwise definition, on every sampled listed prime, and by the
structural properties that hold at any size.
"""
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
    yield
    dqmc.dqmc_release()


def check_all(n, on, dc=None):
    S = oracle.sweep(n, on, dc)
    want_bm = oracle.bitmap(n, S)
    want_pairs = oracle.pairs(n, S)
    got_bm = dqmc.dqmc_primes(n, on, dc)
    assert got_bm.shape == want_bm.shape
    if not np.array_equal(got_bm, want_bm):
        bad = np.nonzero(got_bm != want_bm)[0]
        raise AssertionError(f"n={n}: bitmap differs at {bad.size} bytes, first {bad[:8]}")
    assert dqmc.dqmc_count(n, on, dc) == len(want_pairs)
    pairs, cnt = dqmc.dqmc_list(n, on, dc)
    assert cnt == len(want_pairs)
    assert np.array_equal(pairs, want_pairs)


@pytest.mark.parametrize("n", list(range(0, 13)))
def test_whole_function_tile(n):
    """n <= 12: one CTA holds the whole state in shared memory."""
    for seed in (1, 2, 3):
        for p in (0.3, 0.5, 0.85):
            on, dc = synth.random_function(n, seed, p, 0.1 if seed == 2 else 0.0)
            check_all(n, on, dc)


def test_n10_workload():
    for seed in (1, 2, 3):
        on, dc = synth.single_n10(seed)
        check_all(10, on, dc)


@pytest.mark.parametrize("n", [13, 14, 15, 16, 17])
def test_multipass(n):
    """n >= 13: First / Merge / fused Merge+Reduce / Reduce / bitmap passes."""
    for seed, (p, q) in zip((1, 2), ((0.8, 0.0), (0.6, 0.15))):
        on, dc = synth.random_function(n, seed, p, q)
        check_all(n, on, dc)


def _embedded_band(n, k, lo, hi):
    """f(x) = [lo <= weight(x_0 .. x_{k-1}) <= hi] when x_k .. x_{n-1} are all
    0, else 0: C(k, lo) * C(k - lo, k - hi) primes, all in the first 3^(k-5)
    rows."""
    x = np.arange(1 << k)
    w = np.zeros(x.size, dtype=np.int64)
    for i in range(k):
        w += (x >> i) & 1
    h = np.packbits(((w >= lo) & (w <= hi)).astype(np.uint8), bitorder="little")
    on = np.zeros(synth.tt_bytes(n), dtype=np.uint8)
    on[: h.size] = h
    return on


@pytest.mark.parametrize("n", [13, 16])
def test_dense_primes_in_few_rows(n):
    """More primes in 96 rows of the first bitmap tile than their shared-memory
    slots hold (12 pairs per three-row unit): the bitmap pass lists that tile
    from the bitmap it wrote instead."""
    on = _embedded_band(n, 10, 3, 6)
    S = oracle.sweep(n, on)
    rows = oracle.pairs(n, S)
    assert len(rows) == 120 * 35   # C(10, 3) * C(7, 4)
    rho = np.zeros(len(rows), dtype=np.int64)
    for i in range(n):   # rho of each listed cube from its (mask, value) pair
        lit = (rows[:, 0] >> i) & 1
        one = (rows[:, 1] >> i) & 1
        rho += np.where(lit == 1, one, 2).astype(np.int64) * 3 ** i
    per_region = np.bincount(rho // 243 // 96)
    assert per_region.max() > 12 * 32
    check_all(n, on)


@pytest.mark.parametrize("n", [18, 19])
def test_multipass_larger(n):
    on, dc = synth.random_function(n, 5, 0.9, 0.05)
    check_all(n, on, dc)


def test_n20_workload():
    """n = 20, ON ~ Bernoulli(0.7), DC ~ Bernoulli(0.1): bit-exact against the byte oracle."""
    on, dc = synth.single_n20(1)
    check_all(20, on, dc)


def test_every_function_n3_and_sampled_n4():
    for n in (2, 3):
        for f, sup in bf.all_functions(n):
            on = bf.bitmap_from_bool(sup)
            want = oracle.bitmap(n, oracle.sweep(n, on))
            assert np.array_equal(dqmc.dqmc_primes(n, on), want), (n, f)
    for f in range(0, 1 << 16, 97):
        on = np.array([f & 0xFF, f >> 8], dtype=np.uint8)
        want = oracle.bitmap(4, oracle.sweep(4, on))
        assert np.array_equal(dqmc.dqmc_primes(4, on), want), f


@pytest.mark.parametrize("n", [0, 5, 12, 13, 17])
def test_constants(n):
    ones = np.full(synth.tt_bytes(n), 0xFF, dtype=np.uint8)
    zeros = np.zeros(synth.tt_bytes(n), dtype=np.uint8)
    pairs, c = dqmc.dqmc_list(n, ones)
    assert c == 1 and pairs.tolist() == [[0, 0]]
    bm = dqmc.dqmc_primes(n, ones)
    assert bf.bool_from_bitmap(bm, n).nonzero()[0].tolist() == [3 ** n - 1]
    assert dqmc.dqmc_count(n, zeros) == 0


@pytest.mark.parametrize("n,W", [(3, {2, 3}), (12, {1, 2, 6, 7, 8, 12}), (15, {7, 8, 9, 10, 11, 12, 13, 14, 15}),
                                 (16, set(range(1, 17, 2)))])
def test_symmetric(n, W):
    on = bf.bitmap_from_bool(bf.symmetric_support(n, W))
    assert dqmc.dqmc_count(n, on) == bf.symmetric_prime_count(n, W)
    if n <= 15:
        got = bf.bool_from_bitmap(dqmc.dqmc_primes(n, on), n)
        assert np.array_equal(got, bf.symmetric_prime_cells(n, W))


@pytest.mark.parametrize("n,seed", [(12, 4), (13, 5), (16, 7), (20, 8)])
def test_monotone(n, seed):
    """Monotone functions with no symmetry: the primes are the positive terms
    of the minimal true points (closed form, Section 2's definitions), across
    the one-tile kernel (n = 12) and the pass kernels (n >= 13)."""
    sup, mins = bf.monotone_case(n, seed)
    on = bf.bitmap_from_bool(sup)
    pairs, cnt = dqmc.dqmc_list(n, on, None, cap=len(mins) + 8)
    assert cnt == len(mins)
    assert pairs.tolist() == [[m, m] for m in mins]
    want = np.zeros((3 ** n + 7) // 8, dtype=np.uint8)
    for r in (bf.rho_positive(n, m) for m in mins):
        want[r >> 3] |= np.uint8(1 << (r & 7))
    assert np.array_equal(dqmc.dqmc_primes(n, on), want)


@pytest.mark.parametrize("n,seed,nu", [(11, 13, 0b01010101010), (14, 14, 0b10110011100101),
                                       (17, 15, 0b01101001011010011)])
def test_unate(n, seed, nu):
    """Unate functions (monotone with the inputs in nu negated): primes with
    both 0 and 1 literals, in closed form."""
    sup, want = bf.unate_case(n, seed, nu)
    pairs, cnt = dqmc.dqmc_list(n, bf.bitmap_from_bool(sup), None, cap=len(want) + 8)
    assert cnt == len(want)
    assert pairs.tolist() == [[m, v] for m, v in want]


def test_list_truncation():
    n = 11
    on, _ = synth.random_function(n, 4, 0.6)
    want = oracle.pairs(n, oracle.sweep(n, on))
    cap = len(want) // 3
    pairs, cnt = dqmc.dqmc_list(n, on, None, cap=cap)
    assert cnt == len(want)
    assert np.array_equal(pairs, want[:cap])
    L = dqmc.lib()
    import ctypes
    out = np.empty(2 * cap, dtype=np.uint32)
    c = ctypes.c_uint64()
    st = L.dqmc_list(n, on.ctypes.data_as(dqmc.c_u8p), None, out.ctypes.data_as(dqmc.c_u32p), cap,
                     ctypes.byref(c))
    assert st == dqmc.DQMC_ETRUNC and c.value == len(want)


def test_device_api_with_torch_stream():
    """dqmc_primes_dev / dqmc_list_dev on torch tensors and a side stream."""
    n = 16
    on, dc = synth.random_function(n, 8, 0.8, 0.1)
    S = oracle.sweep(n, on, dc)
    want_bm = oracle.bitmap(n, S)
    want_pairs = oracle.pairs(n, S)
    buf = dqmc.DeviceBuffers(n, with_dc=True, cap=len(want_pairs) + 5)
    buf.on[: on.size].copy_(torch.from_numpy(on))
    buf.dc[: dc.size].copy_(torch.from_numpy(dc))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    buf.list(stream=s)
    s.synchronize()
    got_bm = buf.bitmap[: want_bm.size].cpu().numpy()
    assert np.array_equal(got_bm, want_bm)
    assert not buf.bitmap[want_bm.size:].cpu().numpy().any()
    assert int(buf.count.item()) == len(want_pairs)
    got_pairs = buf.pairs[: 2 * len(want_pairs)].cpu().numpy().view(np.uint32).reshape(-1, 2)
    assert np.array_equal(got_pairs, want_pairs)


def test_repeat_calls_identical():
    """The same call twice (workspace reused, stale state present) gives the same result."""
    n = 15
    a, _ = synth.random_function(n, 1, 0.9)
    b, _ = synth.random_function(n, 2, 0.4)
    ra = dqmc.dqmc_primes(n, a)
    rb = dqmc.dqmc_primes(n, b)
    assert np.array_equal(dqmc.dqmc_primes(n, a), ra)
    assert np.array_equal(dqmc.dqmc_primes(n, b), rb)


def test_n21_three_phase_pass_bit_exact():
    """n = 21 (two groups of high digits above the tile, so every kind of pass:
    first, sparse Merge, last Merge + Reduce, middle Reduce, bitmap) with the
    bitmap and list bit-exact against the byte oracle (10.5 GB of state)."""
    on, dc = synth.random_function(21, 6, 0.8, 0.05)
    check_all(21, on, dc)


def test_per_pass_entry_points_match():
    """dqmc_sweep_pass_dev over all passes equals dqmc_list_dev."""
    n = 17
    on, _ = synth.random_function(n, 12, 0.7)
    S = oracle.sweep(n, on)
    want_bm, want_pairs = oracle.bitmap(n, S), oracle.pairs(n, S)
    buf = dqmc.DeviceBuffers(n, cap=len(want_pairs))
    buf.on[: on.size].copy_(torch.from_numpy(on))
    sh = torch.cuda.current_stream().cuda_stream
    for p in range(dqmc.dqmc_plan_passes(n)):
        dqmc.dqmc_sweep_pass_dev(n, p, buf.on.data_ptr(), None, buf.bitmap.data_ptr(), buf.pairs.data_ptr(),
                                 buf.cap, buf.count.data_ptr(), buf.work.data_ptr(), buf.work_bytes, sh)
    buf.status()
    assert np.array_equal(buf.bitmap[: want_bm.size].cpu().numpy(), want_bm)
    assert int(buf.count.item()) == len(want_pairs)
    got = buf.pairs[: 2 * len(want_pairs)].cpu().numpy().view(np.uint32).reshape(-1, 2)
    assert np.array_equal(got, want_pairs)


def test_bounded_wait_times_out_and_context_survives():
    """A device wait on a counter nothing sets gives up (50 ms limit) and the
    host reads DQMC_ETIMEOUT; the same workspace then sweeps normally."""
    n = 14
    on, _ = synth.random_function(n, 3, 0.8)
    buf = dqmc.DeviceBuffers(n, cap=1 << 20)
    buf.on[: on.size].copy_(torch.from_numpy(on))
    sh = torch.cuda.current_stream().cuda_stream
    dqmc.dqmc_selftest_timeout(n, buf.work.data_ptr(), buf.work_bytes, 50_000_000, sh)
    with pytest.raises(dqmc.DqmcError) as ei:
        buf.status()
    assert ei.value.status == dqmc.DQMC_ETIMEOUT
    buf.list()
    buf.status()
    S = oracle.sweep(n, on)
    assert np.array_equal(buf.bitmap[: (3 ** n + 7) // 8].cpu().numpy(), oracle.bitmap(n, S))


@pytest.mark.parametrize("with_list", [False, True])
def test_bitmap_pass_after_a_timeout_sweeps_nothing(with_list):
    """The bitmap pass's error path, driven without a fault: after a bounded
    wait has given up (the self test leaves DQMC_ETIMEOUT in the error word),
    every tile of a bitmap pass on that workspace sees the error word before
    it issues its bulk copies and leaves without sweeping, so the bitmap keeps
    its old contents, the status stays DQMC_ETIMEOUT, and the next whole sweep
    on the same workspace is bit-exact."""
    n = 16
    on, _ = synth.random_function(n, 5, 0.8)
    buf = dqmc.DeviceBuffers(n, cap=1 << 20)
    buf.on[: on.size].copy_(torch.from_numpy(on))
    sh = torch.cuda.current_stream().cuda_stream
    last = dqmc.dqmc_plan_passes(n) - 1
    cap = buf.cap if with_list else 0
    pairs = buf.pairs.data_ptr() if with_list else None
    L = dqmc.lib()
    assert L.dqmc_sweep_passes_dev(n, 0, last, buf.on.data_ptr(), None, buf.bitmap.data_ptr(), pairs, cap,
                                   buf.count.data_ptr(), buf.work.data_ptr(), buf.work_bytes, sh) == dqmc.DQMC_OK
    torch.cuda.synchronize()
    dqmc.dqmc_selftest_timeout(n, buf.work.data_ptr(), buf.work_bytes, 1_000_000, sh)
    buf.bitmap.fill_(0xA5)
    assert L.dqmc_sweep_pass_dev(n, last, buf.on.data_ptr(), None, buf.bitmap.data_ptr(), pairs, cap,
                                 buf.count.data_ptr(), buf.work.data_ptr(), buf.work_bytes, sh) == dqmc.DQMC_OK
    with pytest.raises(dqmc.DqmcError) as ei:
        buf.status()
    assert ei.value.status == dqmc.DQMC_ETIMEOUT
    assert bool((buf.bitmap == 0xA5).all())
    buf.list()
    buf.status()
    S = oracle.sweep(n, on)
    assert np.array_equal(buf.bitmap[: (3 ** n + 7) // 8].cpu().numpy(), oracle.bitmap(n, S))
    assert int(buf.count.item()) == oracle.count(n, S)


# ------------------------------------------------------ large n, sampled

def _sample_bits(bitmap_dev, rhos):
    idx = torch.from_numpy((rhos >> 3).astype(np.int64)).to(bitmap_dev.device)
    bytes_ = bitmap_dev[idx].cpu().numpy()
    return ((bytes_ >> (rhos & 7).astype(np.uint8)) & 1).astype(bool)


def sampled_check(n, on, dc, p_support, n_list=20000, n_cells=200000, seed=24, inplace=False):
    """Sweep + list in the benchmark's launch configuration (device API), then:
    every sampled listed prime is prime by definition and set in the bitmap, the
    list is ascending, sampled cells agree with the pointwise oracle, the two
    independent counts agree, and the count is within 1% of its expectation.
    inplace: the bitmap is written over the state (one array).  Returns the
    prime count."""
    expected = bf.expected_primes(n, p_support)
    cap = int(expected * 1.05) + 4096
    buf = dqmc.DeviceBuffers(n, with_dc=dc is not None, cap=cap, inplace=inplace)
    buf.on[: on.size].copy_(torch.from_numpy(on))
    if dc is not None:
        buf.dc[: dc.size].copy_(torch.from_numpy(dc))
    buf.list()
    buf.status()
    count = int(buf.count.item())
    assert abs(count - expected) / expected < 0.01
    assert count <= cap
    rng = np.random.default_rng(seed)
    k = np.unique(rng.integers(0, count, size=n_list))
    pairs = buf.pairs.view(-1, 2)[torch.from_numpy(k).cuda()].cpu().numpy().view(np.uint32)
    rho = np.zeros(len(k), dtype=np.int64)
    for i in range(n):
        d = np.where(((pairs[:, 0] >> i) & 1) == 0, 2, (pairs[:, 1] >> i) & 1).astype(np.int64)
        rho += d * 3 ** i
    assert np.all(np.diff(rho) > 0)
    assert np.all(_sample_bits(buf.bitmap, rho))
    assert np.all(oracle.is_prime_many(n, on, dc, rho))
    cells = rng.integers(0, 3 ** n, size=n_cells, dtype=np.int64)
    assert np.array_equal(_sample_bits(buf.bitmap, cells), oracle.is_prime_many(n, on, dc, cells))
    # the sweep's own popcount (bitmap pass, no list) equals the list's count
    c2 = torch.zeros(1, dtype=torch.int64, device="cuda")
    dqmc.dqmc_primes_dev(n, buf.on.data_ptr(), buf.dc.data_ptr() if dc is not None else None,
                         buf.bitmap.data_ptr(), c2.data_ptr(), buf.work.data_ptr(), buf.work_bytes,
                         torch.cuda.current_stream().cuda_stream)
    buf.status()
    assert int(c2.item()) == count
    nb = dqmc.dqmc_bitmap_bytes(n)
    tail_bits = 3 ** n - 8 * (nb - 1)
    assert int(buf.bitmap[nb - 1].item()) >> tail_bits == 0
    assert not buf.bitmap[nb:].any().item()
    del buf
    torch.cuda.empty_cache()
    return count


@pytest.mark.parametrize("n", [22, 23])
def test_large_n_sampled(n):
    on, dc = synth.random_function(n, 2, 0.8, 0.05)
    p_sup = 0.8 + 0.2 * 0.05
    sampled_check(n, on, dc, p_sup, n_list=5000, n_cells=50000)


def test_n24_workload_sampled():
    """n = 24, ON ~ Bernoulli(0.85), seed 1 (the benchmark workload)."""
    on, _ = synth.single_n24(1)
    sampled_check(24, on, None, 0.85)


def test_n25_stretch_sampled():
    """n = 25, ON ~ Bernoulli(0.85), seed 1: the largest size, in one array
    (the bitmap written over the 111.6 GB state, as the paper's in-place
    array of Table 1), sampled as at n = 24."""
    free, _ = torch.cuda.mem_get_info()
    need = dqmc.dqmc_workspace_bytes(25) + int(1.1e9) * 8
    if free < need:
        pytest.skip(f"needs {need / 1e9:.0f} GB of free device memory, {free / 1e9:.0f} GB free")
    on, _ = synth.random_function(25, 1, 0.85)
    count = sampled_check(25, on, None, 0.85, n_list=5000, n_cells=50000, inplace=True)
    # the host entry points write the bitmap over the state at n = 25 too
    dqmc.dqmc_release()
    assert dqmc.dqmc_count(25, on) == count
    dqmc.dqmc_release()


@pytest.mark.parametrize("n,with_list", [(13, True), (16, False), (16, True), (19, True)])
def test_inplace_bitmap_exact(n, with_list):
    """The bitmap written over the state (d_bitmap = d_work): bit-exact
    against the oracle, with and without the list."""
    on, dc = synth.random_function(n, 60 + n, 0.8, 0.05)
    S = oracle.sweep(n, on, dc)
    want_bm, want_pairs = oracle.bitmap(n, S), oracle.pairs(n, S)
    buf = dqmc.DeviceBuffers(n, with_dc=True, cap=len(want_pairs) if with_list else 0, inplace=True)
    buf.on[: on.size].copy_(torch.from_numpy(on))
    buf.dc[: dc.size].copy_(torch.from_numpy(dc))
    if with_list:
        buf.list()
    else:
        buf.primes()
    buf.status()
    assert int(buf.count.item()) == len(want_pairs)
    assert np.array_equal(buf.bitmap[: want_bm.size].cpu().numpy(), want_bm)
    if with_list:
        got = buf.pairs[: 2 * len(want_pairs)].cpu().numpy().view(np.uint32).reshape(-1, 2)
        assert np.array_equal(got, want_pairs)


def test_inplace_bitmap_overlap_refused():
    """Any overlap of the bitmap with the workspace other than the in-place
    start is refused before any work is enqueued."""
    n = 14
    buf = dqmc.DeviceBuffers(n, inplace=True)
    L = dqmc.lib()
    st = L.dqmc_primes_dev(n, buf.on.data_ptr(), None, buf.work.data_ptr() + 256, buf.count.data_ptr(),
                           buf.work.data_ptr(), buf.work_bytes, None)
    assert st == dqmc.DQMC_EINVAL


@pytest.mark.parametrize("n", [11, 17, 20, 22])
def test_list_into_pinned_host_memory(n):
    """dqmc_list into pinned host memory (written by the kernels directly)
    equals the list through pageable memory (device buffer and a copy), also
    when truncated."""
    import ctypes
    on, dc = synth.random_function(n, 40 + n, 0.75, 0.05)
    want, count = dqmc.dqmc_list(n, on, dc)
    L = dqmc.lib()
    for cap in (count, count // 3):
        pinned = torch.full((2 * max(cap, 1) + 2,), -1, dtype=torch.int32).pin_memory()
        c = ctypes.c_uint64()
        st = L.dqmc_list(n, dqmc._p8(on), dqmc._p8(dc), ctypes.cast(pinned.data_ptr(), dqmc.c_u32p), cap,
                         ctypes.byref(c))
        assert st == (dqmc.DQMC_OK if cap >= count else dqmc.DQMC_ETRUNC)
        assert int(c.value) == count
        got = pinned.numpy().view(np.uint32)[: 2 * cap].reshape(cap, 2)
        assert np.array_equal(got, want[:cap])
        assert (pinned.numpy()[2 * cap:] == -1).all()   # nothing past cap
