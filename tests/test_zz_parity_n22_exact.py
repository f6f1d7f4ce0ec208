"""n = 22 bit-exact: the prime bitmap and count of libdqmc.so (through its C
ABI) against the oracle's bit-per-cube mode (3.9 GB; the byte-per-cube state
would be 31 GB).  The same function as the sampled n = 22 case.  In a module
of its own, collected near the end: it holds about 12 GB of host memory
and runs the oracle for a minute or two."""
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


def _mem_available_bytes():
    """Host memory this process can still use: MemAvailable, capped by the
    cgroup's limit less its usage when one is set (inside a container
    /proc/meminfo shows the whole machine)."""
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


def test_n22_bit_exact_packed_oracle():
    """Every bit of the n = 22 bitmap, and the count."""
    n = 22
    A = (3 ** n + 7) // 8
    if _mem_available_bytes() < 4 * A + (2 << 30):
        pytest.skip("needs about 18 GB of available host memory")
    on, dc = synth.random_function(n, 2, 0.8, 0.05)
    S = oracle.sweep_packed(n, on, dc)
    want = oracle.packed_bitmap(n, S)
    del S
    got = dqmc.dqmc_primes(n, on, dc)
    assert got.shape == want.shape
    assert np.array_equal(got, want)
    pop = np.array([bin(i).count("1") for i in range(256)], dtype=np.uint8)
    count = sum(int(pop[want[i: i + (1 << 26)]].sum(dtype=np.uint64)) for i in range(0, A, 1 << 26))
    assert dqmc.dqmc_count(n, on, dc) == count
