"""The entry point for callers that cannot allocate device memory.

dqmc_primes_dev_static computes the same prime bitmap and count as
dqmc_primes_dev, using a static workspace inside the library instead of one
the caller allocates.  Such callers exist: an application whose own pool owns
the device memory, or code that may not risk an allocation's device
synchronisation on its latency path.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2302_10083_gb300 import dqmc, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _run_both(n, on, dc):
    """Bitmap and count from the static-workspace entry point and from the
    caller-workspace entry point, on the same inputs."""
    buf = dqmc.DeviceBuffers(n, with_dc=dc is not None)
    buf.on[: on.size].copy_(torch.from_numpy(on))
    if dc is not None:
        buf.dc[: dc.size].copy_(torch.from_numpy(dc))
    sh = torch.cuda.current_stream().cuda_stream
    bm2 = torch.empty_like(buf.bitmap)
    c2 = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = dqmc.lib().dqmc_primes_dev_static(n, buf.on.data_ptr(),
                                           buf.dc.data_ptr() if dc is not None else None,
                                           bm2.data_ptr(), c2.data_ptr(), sh)
    assert st == dqmc.DQMC_OK, dqmc.strerror(st)
    # the static sweep's bounded waits and bounds checks report through the
    # error word in the static array
    assert dqmc.lib().dqmc_dev_status_static(n, sh) == dqmc.DQMC_OK
    buf.primes()
    torch.cuda.synchronize()
    return (buf.bitmap.cpu().numpy(), int(buf.count.item())), (bm2.cpu().numpy(), int(c2.item()))


def test_static_workspace_matches_caller_workspace():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    # two calls in a row on the static array (its contents are left from the
    # previous call), at the largest accepted n and at a one-tile n
    for n, seed, p, q in ((15, 1, 0.8, 0.0), (15, 2, 0.6, 0.15), (11, 3, 0.7, 0.1), (11, 4, 0.9, 0.0)):
        on, dc = synth.random_function(n, seed, p, q)
        (bm1, c1), (bm2, c2) = _run_both(n, on, dc)
        assert c1 == c2
        assert np.array_equal(bm1, bm2)   # integer results: bit-exact


def test_static_workspace_rejects_large_n():
    """n = 16 does not fit the 2 MiB array: rejected before any device work."""
    st = dqmc.lib().dqmc_primes_dev_static(16, ctypes.c_void_p(256), None, ctypes.c_void_p(256), None, None)
    assert st == dqmc.DQMC_EINVAL
    assert dqmc.lib().dqmc_dev_status_static(16, None) == dqmc.DQMC_EINVAL
