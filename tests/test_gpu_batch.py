"""Batched sweep (dqmc_batch_run) on the GPU: every function of a batch is
bit-exact against the oracle (bitmap, tail bytes of its slot, count) on both
paths (whole functions in shared memory, and the tile / streaming kernels) and
for every launch shape the autotuner may pick; the captured graph gives the
same result when launched again, and a new set of buffers, functions or
configurations is captured anew."""
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
    saved = dqmc.batch_tuning_table()
    yield
    dqmc.load_batch_tuning(saved)
    dqmc.dqmc_batch_release()


@pytest.fixture
def table():
    """Restores the configuration table after the test."""
    saved = dqmc.batch_tuning_table()
    yield saved
    dqmc.load_batch_tuning(saved)


def set_all(path, **shape):
    for n in range(dqmc.DQMC_BATCH_MAX_N + 1):
        if path == dqmc.DQMC_BATCH_PATH_TILES or n >= 5:
            cfg = dict(path=path, threads_per_fn=256, fns_per_cta=1, digits_per_step=2,
                       ctas_per_fn=3 if n == 14 else 1)
            cfg.update(shape)
            assert dqmc.dqmc_batch_set_config(n, cfg) == dqmc.DQMC_OK


def run_batch(b, with_dc=True, one_launch=False):
    ns = b["n"].astype(np.uint32)
    dev = "cuda:0"
    arena = torch.from_numpy(b["arena"]).to(dev)
    bm_off, total = dqmc.batch_bitmap_layout(ns)
    bitmaps = torch.full((max(total, 16),), 0xA5, dtype=torch.uint8, device=dev)   # junk to be overwritten
    counts = torch.full((len(ns),), -1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    dc_off = b["dc_off"] if with_dc else None
    st = dqmc.dqmc_batch_run(ns, b["tt_off"], arena.data_ptr(), dc_off, counts.data_ptr(), bitmaps.data_ptr(),
                             bm_off, stream, one_launch=one_launch)
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


@pytest.mark.parametrize("path", ["tiles", "smem"])
def test_batch_each_path_bit_exact(path, table):
    """The whole mixed batch on one path: the tile / streaming kernels for
    every n, or shared memory for every n >= 5."""
    if path == "tiles":
        set_all(dqmc.DQMC_BATCH_PATH_TILES)
    else:
        set_all(dqmc.DQMC_BATCH_PATH_SMEM, threads_per_fn=256, digits_per_step=3)
    b = synth.batch_functions(count=120, seed=11)
    arena, bitmaps, counts, bm_off, dc_off = run_batch(b)
    check_batch(b, bitmaps, counts, bm_off, dc_off)


# (n, threads per function, functions per CTA, digits per step, CTAs per
# function): every n of the shared-memory path, both step sizes, one warp up
# to 1024 threads, clusters of 3 and 9, one CTA doing the thirds of n = 14 in
# turn, and CTAs whose last functions are missing (13 functions per batch).
SMEM_SHAPES = [
    (5, 32, 8, 2, 1), (5, 64, 3, 3, 1), (6, 32, 6, 3, 1), (7, 32, 4, 2, 1), (8, 64, 4, 3, 1), (8, 32, 15, 2, 1),
    (9, 128, 2, 2, 1), (9, 32, 1, 3, 1), (10, 96, 3, 3, 1), (10, 1024, 1, 2, 1), (11, 256, 2, 2, 1),
    (11, 32, 1, 3, 1), (12, 512, 1, 3, 1), (12, 128, 3, 2, 1), (12, 1024, 1, 3, 1), (13, 512, 1, 3, 1),
    (13, 1024, 1, 2, 1), (13, 64, 1, 2, 1), (13, 256, 1, 3, 3), (13, 1024, 1, 2, 3), (14, 512, 1, 3, 3),
    (14, 1024, 1, 2, 3), (14, 128, 1, 3, 3), (14, 256, 1, 3, 9), (14, 1024, 1, 2, 9), (14, 64, 1, 3, 9),
    (14, 1024, 1, 3, 1), (14, 256, 1, 2, 1),
]


@pytest.mark.parametrize("n,tg,fpc,d,ctas", SMEM_SHAPES)
def test_batch_smem_shapes_bit_exact(n, tg, fpc, d, ctas, table):
    cfg = dict(path=dqmc.DQMC_BATCH_PATH_SMEM, threads_per_fn=tg, fns_per_cta=fpc, digits_per_step=d,
               ctas_per_fn=ctas)
    assert dqmc.dqmc_batch_set_config(n, cfg) == dqmc.DQMC_OK
    b = synth.batch_functions(count=13, seed=100 + n, n_lo=n, n_hi=n)
    arena, bitmaps, counts, bm_off, dc_off = run_batch(b)
    check_batch(b, bitmaps, counts, bm_off, dc_off)


def test_batch_smem_constant_and_parity_functions(table):
    """Closed forms through the shared-memory path: constant 1 (only the
    all-'*' cube), constant 0 (no primes) and parity (its 2^(n-1) minterms),
    for n = 5, 9, 13 and 14."""
    set_all(dqmc.DQMC_BATCH_PATH_SMEM, threads_per_fn=256, digits_per_step=3)
    ns, tabs = [], []
    for n in (5, 9, 13, 14):
        nb = (1 << n) // 8
        x = np.arange(1 << n)
        par = np.packbits((np.unpackbits(x.astype(">u4").view(np.uint8)).reshape(-1, 32).sum(1) & 1).astype(np.uint8),
                          bitorder="little")
        for t in (np.full(nb, 0xFF, np.uint8), np.zeros(nb, np.uint8), par):
            ns.append(n)
            tabs.append(t)
    off, pos, parts = [], 0, []
    for t in tabs:
        off.append(pos)
        parts.append(t)
        pos += len(t)
    b = {"n": np.array(ns), "tt_off": np.array(off, np.uint64), "arena": np.concatenate(parts),
         "dc_off": np.full(len(ns), np.iinfo(np.uint64).max, np.uint64)}
    arena, bitmaps, counts, bm_off, _ = run_batch(b, with_dc=False)
    cnt = counts.cpu().numpy()
    bm = bitmaps.cpu().numpy()
    for f, n in enumerate(ns):
        kind = f % 3
        want = [1, 0, 1 << (n - 1)][kind]
        assert int(cnt[f]) == want, (n, kind)
        bits = np.unpackbits(bm[int(bm_off[f]): int(bm_off[f]) + (3 ** n + 7) // 8], bitorder="little")[: 3 ** n]
        if kind == 0:
            assert bits[3 ** n - 1] == 1   # the all-'*' cube: every digit 2
    check_batch(b, bitmaps, counts, bm_off, None)


def test_autotune_then_run_bit_exact(table):
    """The autotuner picks a launchable configuration for every n present,
    reports a time for each, and the batch run with its choices is exact."""
    b = synth.batch_functions(count=200, seed=21)
    ns = b["n"].astype(np.uint32)
    dev = "cuda:0"
    arena = torch.from_numpy(b["arena"]).to(dev)
    bm_off, total = dqmc.batch_bitmap_layout(ns)
    bitmaps = torch.zeros(total, dtype=torch.uint8, device=dev)
    counts = torch.zeros(len(ns), dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    best = dqmc.dqmc_batch_autotune(ns, b["tt_off"], arena.data_ptr(), b["dc_off"], counts.data_ptr(),
                                    bitmaps.data_ptr(), bm_off, stream, reps=1)
    assert sorted(best) == sorted(set(int(n) for n in ns)) and all(ms > 0 for ms in best.values())
    for n in best:
        c = dqmc.dqmc_batch_get_config(n)
        assert c["path"] in (dqmc.DQMC_BATCH_PATH_SMEM, dqmc.DQMC_BATCH_PATH_TILES)
        assert dqmc.dqmc_batch_set_config(n, c) == dqmc.DQMC_OK
    _, bitmaps, counts, bm_off, dc_off = run_batch(b)
    check_batch(b, bitmaps, counts, bm_off, dc_off)


# ------------------------------------------------------- one persistent launch

def test_one_launch_mixed_sizes_bit_exact():
    """dqmc_batch_run_one_launch on the workload's n = 4..14 mix with
    don't-cares: every function bit-exact against the oracle; the graph
    launched again gives the same; then the graph path on the same buffers
    (a new capture) gives the same bytes."""
    b = synth.batch_functions(count=240, seed=11)
    arena, bitmaps, counts, bm_off, dc_off = run_batch(b, one_launch=True)
    check_batch(b, bitmaps, counts, bm_off, dc_off)
    first = bitmaps.clone()
    bitmaps.fill_(0x5A)
    counts.fill_(-1)
    stream = torch.cuda.current_stream().cuda_stream
    ns = b["n"].astype(np.uint32)
    for one in (True, False):
        st = dqmc.dqmc_batch_run(ns, b["tt_off"], arena.data_ptr(), dc_off, counts.data_ptr(), bitmaps.data_ptr(),
                                 bm_off, stream, one_launch=one)
        assert st == dqmc.DQMC_OK
        torch.cuda.synchronize()
        assert torch.equal(bitmaps, first)


def test_one_launch_degenerate_and_small_n():
    """n = 0..8 without a don't-care table (n <= 4 by one warp each, from the
    definitions), and closed forms through the same launch: constant 1 (only
    the all-'*' cube), constant 0 (no primes) and parity (its 2^(n-1)
    minterms) for n = 0..14."""
    b = synth.batch_functions(count=90, seed=12, n_lo=0, n_hi=8)
    arena, bitmaps, counts, bm_off, dc_off = run_batch(b, with_dc=False, one_launch=True)
    check_batch(b, bitmaps, counts, bm_off, None)
    ns, tabs = [], []
    for n in range(0, 15):
        nb = ((1 << n) + 7) >> 3
        x = np.arange(1 << n)
        par = np.zeros(1 << n, dtype=np.uint8)
        for i in range(n):
            par ^= ((x >> i) & 1).astype(np.uint8)
        for t in (np.full(nb, 0xFF, np.uint8) if n >= 3 else synth.pack(np.ones(1 << n, bool)),
                  np.zeros(nb, np.uint8), synth.pack(par.astype(bool))):
            ns.append(n)
            tabs.append(np.asarray(t, np.uint8))
    off, pos = [], 0
    for t in tabs:
        off.append(pos)
        pos += (len(t) + 3) // 4 * 4
    arena = np.zeros(pos, np.uint8)
    for o, t in zip(off, tabs):
        arena[o: o + len(t)] = t
    bb = {"n": np.array(ns), "tt_off": np.array(off, np.uint64), "arena": arena,
          "dc_off": np.full(len(ns), np.iinfo(np.uint64).max, np.uint64)}
    _, bitmaps, counts, bm_off, _ = run_batch(bb, with_dc=False, one_launch=True)
    cnt = counts.cpu().numpy()
    bm = bitmaps.cpu().numpy()
    for f, n in enumerate(ns):
        kind = f % 3
        want = [1, 0, 1 << (n - 1) if n else 0][kind]
        assert int(cnt[f]) == want, (n, kind)
        bits = np.unpackbits(bm[int(bm_off[f]): int(bm_off[f]) + (3 ** n + 7) // 8], bitorder="little")[: 3 ** n]
        if kind == 0:
            assert bits.sum() == 1 and bits[3 ** n - 1] == 1
        elif kind == 1:
            assert not bits.any()
    check_batch(bb, bitmaps, counts, bm_off, None)


def test_one_launch_large_classes_and_tuned_shapes(table):
    """Only n = 12..14 (groups of 256 threads, the whole CTA, the thirds of
    n = 14), then with every n's shared-memory shape set to 128 threads and
    two digits per step: bit-exact both times."""
    b = synth.batch_functions(count=30, seed=13, n_lo=12, n_hi=14)
    arena, bitmaps, counts, bm_off, dc_off = run_batch(b, one_launch=True)
    check_batch(b, bitmaps, counts, bm_off, dc_off)
    for n in range(5, 15):
        cfg = dict(path=dqmc.DQMC_BATCH_PATH_SMEM, threads_per_fn=128, fns_per_cta=1, digits_per_step=2,
                   ctas_per_fn=1)
        if n == 14:
            cfg["threads_per_fn"] = 1024
        assert dqmc.dqmc_batch_set_config(n, cfg) == dqmc.DQMC_OK
    b2 = synth.batch_functions(count=120, seed=14, n_lo=5, n_hi=14)
    arena, bitmaps, counts, bm_off, dc_off = run_batch(b2, one_launch=True)
    check_batch(b2, bitmaps, counts, bm_off, dc_off)
