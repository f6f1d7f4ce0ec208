"""Batched sweep (dqmc_batch_run) on the GPU: every function of a batch is
bit-exact against the oracle (bitmap, tail bytes of its slot, count), the
captured graph gives the same result when launched again, and a new set of
buffers or functions is captured anew."""
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
    dqmc.dqmc_batch_release()


def run_batch(b, with_dc=True):
    ns = b["n"].astype(np.uint32)
    dev = "cuda:0"
    arena = torch.from_numpy(b["arena"]).to(dev)
    bm_off, total = dqmc.batch_bitmap_layout(ns)
    bitmaps = torch.full((max(total, 16),), 0xA5, dtype=torch.uint8, device=dev)   # junk to be overwritten
    counts = torch.full((len(ns),), -1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    dc_off = b["dc_off"] if with_dc else None
    st = dqmc.dqmc_batch_run(ns, b["tt_off"], arena.data_ptr(), dc_off, counts.data_ptr(), bitmaps.data_ptr(),
                             bm_off, stream)
    assert st == dqmc.DQMC_OK, dqmc.strerror(st)
    torch.cuda.synchronize()
    return arena, bitmaps, counts, bm_off, dc_off


def check_batch(b, bitmaps, counts, bm_off, dc_off):
    bm = bitmaps.cpu().numpy()
    cnt = counts.cpu().numpy()
    ns = b["n"]
    for f in range(len(ns)):
        n = int(ns[f])
        tt = (1 << n) + 7 >> 3
        on = b["arena"][int(b["tt_off"][f]): int(b["tt_off"][f]) + tt]
        dc = None
        if dc_off is not None and int(dc_off[f]) != np.iinfo(np.uint64).max:
            dc = b["arena"][int(dc_off[f]): int(dc_off[f]) + tt]
        S = oracle.sweep(n, on, dc)
        want = oracle.bitmap(n, S)
        o = int(bm_off[f])
        got = bm[o: o + len(want)]
        assert np.array_equal(got, want), f"function {f}, n={n}: bitmap differs"
        slot = dqmc.dqmc_bitmap_alloc_bytes(n)
        assert not bm[o + len(want): o + slot].any(), f"function {f}: slot tail not zero"
        assert int(cnt[f]) == oracle.count(n, S), f"function {f}, n={n}: count"


def test_batch_mixed_sizes_bit_exact():
    """n = 4..14 (the batched workload's distribution), ON density in
    [0.3, 0.9], 10% with don't-cares; then the same batch again (graph
    launched a second time, outputs cleared in between)."""
    b = synth.batch_functions(count=240, seed=1)
    assert set(int(x) for x in b["n"]) == set(range(4, 15))
    assert b["has_dc"].any()
    arena, bitmaps, counts, bm_off, dc_off = run_batch(b)
    check_batch(b, bitmaps, counts, bm_off, dc_off)
    bitmaps.fill_(0x5A)
    counts.fill_(-1)
    stream = torch.cuda.current_stream().cuda_stream
    st = dqmc.dqmc_batch_run(b["n"].astype(np.uint32), b["tt_off"], arena.data_ptr(), dc_off, counts.data_ptr(),
                             bitmaps.data_ptr(), bm_off, stream)
    assert st == dqmc.DQMC_OK
    torch.cuda.synchronize()
    check_batch(b, bitmaps, counts, bm_off, dc_off)


def test_batch_small_n_and_no_dc_table():
    """n = 0..8 including the degenerate n = 0..4 (one chunk row) and no
    don't-care table at all."""
    b = synth.batch_functions(count=90, seed=2, n_lo=0, n_hi=8)
    arena, bitmaps, counts, bm_off, dc_off = run_batch(b, with_dc=False)
    check_batch(b, bitmaps, counts, bm_off, None)


def test_batch_large_classes_only():
    """Only n = 13 and 14: the streaming pass kernels in batch mode, several
    functions per launch."""
    b = synth.batch_functions(count=24, seed=3, n_lo=13, n_hi=14)
    arena, bitmaps, counts, bm_off, dc_off = run_batch(b)
    check_batch(b, bitmaps, counts, bm_off, dc_off)


def test_batch_matches_single_function_calls():
    """Each function's result in the batch equals its own dqmc_primes call."""
    b = synth.batch_functions(count=40, seed=4, n_lo=10, n_hi=14)
    arena, bitmaps, counts, bm_off, dc_off = run_batch(b)
    bm = bitmaps.cpu().numpy()
    for f in range(len(b["n"])):
        n = int(b["n"][f])
        tt = (1 << n) + 7 >> 3
        on = b["arena"][int(b["tt_off"][f]): int(b["tt_off"][f]) + tt]
        dc = None
        if int(dc_off[f]) != np.iinfo(np.uint64).max:
            dc = b["arena"][int(dc_off[f]): int(dc_off[f]) + tt]
        single = dqmc.dqmc_primes(n, on, dc)
        o = int(bm_off[f])
        assert np.array_equal(bm[o: o + len(single)], single)
