"""The bench's host logic (no GPU).  As two gloo ranks: every rank takes the
largest step time over the ranks, and the whole-job value is the units all
ranks processed over that time; the reference arm under a two-process launch
prints one JSON line, from rank 0, and every rank exits 0.  The sweep itself
has no exchange step (one function per rank), so these are the only
cross-rank paths.  Also the kernel count the batched line claims."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _ranks_body(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 20.25][rank]
        got = bench.max_over_ranks(ms, world, "cpu")
        one = bench.max_over_ranks(ms, 1, "cpu")   # world 1: no collective, the rank's own value
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"got": got, "one": one}, f)
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks(tmp_path):
    world = 2
    mp.start_processes(_ranks_body, args=(world, free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    assert [r["got"] for r in res] == [20.25, 20.25]
    assert [r["one"] for r in res] == [12.5, 20.25]


def test_reference_arm_two_ranks_prints_one_line():
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "2", "--warmup", "1", "--ref-n", "10"]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 2 and d["warmup"] == 1
    assert d["unit"] == "cubes/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["sample_n"] == 10
    # the same metric string as the main arm's line, so the two can be divided
    sys.path.insert(0, ROOT)
    import bench
    assert d["metric"] == bench.single_metric(bench.N_MAIN)
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "cubes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_launches_per_graph_counts_kernels():
    """The batched line's kernel count: one launch per n on the shared-memory
    path and for the one-tile kernel (n <= 12), one per pass for n = 13, 14 on
    the streaming path.  With the built-in table the workload's n = 4..14 take
    11 launches per graph (10 shared-memory classes and the one-tile n = 4)."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2302_10083_gb300 import dqmc
    table = dqmc.batch_tuning_table()
    ns = list(range(4, 15)) * 3
    assert bench.launches_per_graph(ns, table) == 11
    tiles = dict(table)
    for n in (13, 14):
        tiles[str(n)] = dict(table[str(n)], path=dqmc.DQMC_BATCH_PATH_TILES)
    assert bench.launches_per_graph(ns, tiles) == 9 + dqmc.dqmc_plan_passes(13) + dqmc.dqmc_plan_passes(14)
    assert bench.launches_per_graph([4, 4, 7], table) == 2


def test_cpu_baseline_fields():
    """The bench's cpu_baseline: the oracle on every host thread, and the same
    oracle on one thread beside it, without changing the thread count later
    calls get."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    cores = oracle.max_threads()
    d = bench.cpu_baseline(12)
    assert d["kind"] == "oracle" and d["unit"] == "cubes/s" and d["value"] > 0 and d["cores"] == cores
    assert d["one_core"]["cores"] == 1 and d["one_core"]["value"] > 0 and "n=9" in d["one_core"]["sample"]
    assert oracle.max_threads() == cores
