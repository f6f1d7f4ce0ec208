"""n = 22, 23 and 24 (the benchmark workload) bit-exact, at sizes where the
oracle cannot run beside the test: the SHA-256 of libdqmc.so's prime bitmap
and of its (mask, value) list (through the C ABI), and its prime count,
against the oracle's.  The oracle's values are in
tests/golden/bitmap_digests.txt, written by tests/golden/make_digests.py,
which runs only the oracle (its bit-per-cube sweep, Algorithm 3, Section 4.1)
and the seeded input generator.  Equal digests mean equal bitmaps and lists,
bit for bit.  In a module collected after the other parity tests (the n = 24 bitmap
takes 35 GB of host memory); only the static-workspace test follows it."""
import hashlib
import os

import numpy as np
import pytest

from paper_2302_10083_gb300 import dqmc, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "bitmap_digests.txt")


def _cases():
    out = {}
    if os.path.exists(GOLDEN):
        for line in open(GOLDEN):
            if line.strip() and not line.startswith("#"):
                n, seed, p_on, p_dc, count, h, hl = line.split()
                out[int(n)] = (int(seed), float(p_on), float(p_dc), int(count), h, hl)
    return out


CASES = _cases()


def _mem_available_bytes():
    """MemAvailable, capped by the cgroup's limit less its usage when one is set."""
    avail = 0
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) * 1024
    except OSError:
        return 0
    for limit_file, usage_file in (("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory.current"),
                                   ("/sys/fs/cgroup/memory/memory.limit_in_bytes",
                                    "/sys/fs/cgroup/memory/memory.usage_in_bytes")):
        try:
            with open(limit_file) as f:
                limit = f.read().strip()
            with open(usage_file) as f:
                usage = int(f.read().strip())
        except (OSError, ValueError):
            continue
        if limit.isdigit():
            avail = min(avail, max(int(limit) - usage, 0))
        break
    return avail


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dqmc.lib()
    yield
    dqmc.dqmc_release()


@pytest.mark.parametrize("n", [22, 23, 24])
def test_bitmap_list_digests_and_count(n):
    if n not in CASES:
        pytest.skip(f"no stored digest for n = {n}")
    seed, p_on, p_dc, count, want, want_list = CASES[n]
    A = (3 ** n + 7) // 8
    if _mem_available_bytes() < A + (4 << 30):
        pytest.skip(f"needs about {(A >> 30) + 4} GiB of available host memory")
    free, _ = torch.cuda.mem_get_info()
    need = dqmc.dqmc_workspace_bytes(n) + dqmc.dqmc_bitmap_alloc_bytes(n) + (1 << 30)
    if free < need:
        pytest.skip(f"needs {need >> 30} GiB of free device memory")
    on, dc = synth.random_function(n, seed, p_on, p_dc)
    got = dqmc.dqmc_primes(n, on, dc)
    assert got.size == A
    assert hashlib.sha256(memoryview(got)).hexdigest() == want
    del got
    assert dqmc.dqmc_count(n, on, dc) == count
    pairs, c = dqmc.dqmc_list(n, on, dc, cap=count)
    assert c == count and pairs.shape == (count, 2)
    assert hashlib.sha256(memoryview(np.ascontiguousarray(pairs, dtype="<u4"))).hexdigest() == want_list


@pytest.mark.parametrize("n", [22, 23])
def test_inplace_bitmap_digests(n):
    """The bitmap written over the state (d_bitmap = d_work, one array): the
    same SHA-256 of the bitmap and the list as the oracle's."""
    if n not in CASES:
        pytest.skip(f"no stored digest for n = {n}")
    seed, p_on, p_dc, count, want, want_list = CASES[n]
    A = (3 ** n + 7) // 8
    if _mem_available_bytes() < A + (4 << 30):
        pytest.skip(f"needs about {(A >> 30) + 4} GiB of available host memory")
    on, dc = synth.random_function(n, seed, p_on, p_dc)
    buf = dqmc.DeviceBuffers(n, with_dc=dc is not None, cap=count, inplace=True)
    assert buf.bitmap.data_ptr() == buf.work.data_ptr()
    buf.on[: on.size].copy_(torch.from_numpy(on))
    if dc is not None:
        buf.dc[: dc.size].copy_(torch.from_numpy(dc))
    buf.list()
    buf.status()
    assert int(buf.count.item()) == count
    got = buf.bitmap[:A].cpu().numpy()
    assert hashlib.sha256(memoryview(got)).hexdigest() == want
    del got
    pairs = buf.pairs[: 2 * count].cpu().numpy().view(np.uint32)
    assert hashlib.sha256(memoryview(np.ascontiguousarray(pairs, dtype="<u4"))).hexdigest() == want_list
    del buf
    torch.cuda.empty_cache()
