"""Serving loop (dqmc_server_*) on the GPU: each job's result in a mix of
concurrent jobs is bit-exact against the same function swept alone
(dqmc_primes) and against the oracle; the one-at-a-time server gives the same
results; admission under a tight memory budget still completes every job
within the budget; the load generator's counts match."""
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


def job_mix(count, seed, n_hi):
    req = synth.serving_requests(count, seed, rate=1e4, n_lo=6, n_hi=n_hi)
    jobs = []
    for j in range(count):
        n = int(req["n"][j])
        dens = float(req["density"][j])
        on, dc = synth.random_function(n, int(req["seed"][j]) & 0x7FFFFFFF, dens, 0.05 if j % 5 == 0 else 0.0)
        jobs.append((n, on, dc))
    return req, jobs


def run_mix(server, jobs):
    ids = [server.submit(n, on, dc) for n, on, dc in jobs]
    out = []
    for (n, _, _), i in zip(jobs, ids):
        server.wait(i)
        q = server.query(i)
        assert q["state"] == dqmc.DQMC_JOB_DONE
        out.append((q["count"], server.bitmap(i, n)))
        server.free(i)
    return out


def test_mix_matches_alone_and_oracle():
    req, jobs = job_mix(80, 1, 18)
    assert max(n for n, _, _ in jobs) >= 16 and min(n for n, _, _ in jobs) <= 8
    with dqmc.Server(4 << 30, streams=4) as srv:
        got = run_mix(srv, jobs)
        st = srv.stats()
    assert st["done"] == len(jobs) and st["batched_jobs"] > 0
    for (n, on, dc), (cnt, bm) in zip(jobs, got):
        alone = dqmc.dqmc_primes(n, on, dc)
        assert np.array_equal(bm, alone), f"n={n}: bitmap differs from the function swept alone"
        assert cnt == int(np.unpackbits(alone).sum())
        if n <= 14:
            S = oracle.sweep(n, on, dc)
            assert np.array_equal(bm, oracle.bitmap(n, S))


def test_serial_server_gives_same_results():
    req, jobs = job_mix(30, 2, 16)
    with dqmc.Server(2 << 30, streams=4) as a:
        ra = run_mix(a, jobs)
    with dqmc.Server(2 << 30, streams=1, mode=dqmc.DQMC_SERVER_SERIAL) as b:
        rb = run_mix(b, jobs)
        assert b.stats()["peak_running"] == 1
    for (ca, ba), (cb, bb) in zip(ra, rb):
        assert ca == cb and np.array_equal(ba, bb)


def test_tight_budget_admits_as_memory_frees():
    """A budget that holds two n = 18 jobs at a time: ten of them plus small
    ones all finish, correct, and the device bytes in use never pass it."""
    big = dqmc.dqmc_server_job_bytes(18)
    budget = int(2.2 * big) + (64 << 20)
    jobs = [(18, *synth.random_function(18, 100 + j, 0.8)) for j in range(10)]
    jobs += [(8, *synth.random_function(8, 200 + j, 0.5)) for j in range(40)]
    with dqmc.Server(budget, streams=8) as srv:
        got = run_mix(srv, jobs)
        st = srv.stats()
    assert st["peak_bytes"] <= budget
    for (n, on, dc), (cnt, bm) in zip(jobs, got):
        assert np.array_equal(bm, dqmc.dqmc_primes(n, on, dc))


def test_oversize_job_rejected():
    with dqmc.Server(64 << 20, streams=1) as srv:
        on, _ = synth.random_function(20, 1, 0.5)
        with pytest.raises(dqmc.DqmcError):
            srv.submit(20, on)


def test_replay_counts_match_alone():
    req, jobs = job_mix(200, 3, 16)
    with dqmc.Server(4 << 30, streams=8) as srv:
        counts, lat, span = srv.replay(req["t_arrive"], [n for n, _, _ in jobs], [on for _, on, _ in jobs],
                                       [dc for _, _, dc in jobs])
    assert span > 0 and (lat >= 0).all()
    for (n, on, dc), c in zip(jobs, counts):
        assert int(c) == dqmc.dqmc_count(n, on, dc)


@pytest.mark.parametrize("mode", ["concurrent", "serial"])
def test_shared_memory_sizes_in_both_modes(mode):
    """Jobs of n = 13 and 14 (batched on the shared-memory path, no
    workspace in their footprint) next to small and large jobs, in either
    mode: each bitmap equals the function swept alone."""
    jobs = []
    for j, n in enumerate([13, 14, 8, 15, 14, 13, 6, 14]):
        on, dc = synth.random_function(n, 300 + j, 0.6 + 0.04 * j, 0.05 if j % 2 else 0.0)
        jobs.append((n, on, dc))
    m = dqmc.DQMC_SERVER_SERIAL if mode == "serial" else dqmc.DQMC_SERVER_CONCURRENT
    with dqmc.Server(2 << 30, streams=1 if mode == "serial" else 4, mode=m) as srv:
        got = run_mix(srv, jobs)
    for (n, on, dc), (cnt, bm) in zip(jobs, got):
        alone = dqmc.dqmc_primes(n, on, dc)
        assert np.array_equal(bm, alone), f"n={n}"
        assert cnt == int(np.unpackbits(alone).sum())
