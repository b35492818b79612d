"""The benchmark's multi-process logic on CPU (gloo, world size 2): every rank
runs its own replica (the solves do not shard), the reported time is the
slowest rank's and the solve count is summed over ranks; the reference arm
runs on rank 0 only.  No GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    bench.dist_init(world, "gloo")
    r, w, lr = bench.dist_env()
    t = bench.reduce_max(10.0 * (rank + 1), w)
    n = bench.reduce_sum(3.0, w)
    bench.barrier(w)
    rc = bench.run_reference(bench.parse_args(["--impl", "reference", "--steps", "1", "--warmup", "0"])) \
        if rank == 1 else 0
    out.put((rank, r, w, t, n, rc))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_replicas_max_time_and_summed_solves():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=100) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    assert [x[1] for x in res] == [0, 1] and all(x[2] == 2 for x in res)
    assert all(x[3] == 20.0 for x in res)          # slowest rank's time on every rank
    assert all(x[4] == 6.0 for x in res)           # solves summed over ranks
    assert res[1][5] == 0                          # reference arm: rank 1 exits 0 without work


def test_bench_defaults():
    import bench
    a = bench.parse_args([])
    assert a.gpus == 1 and a.warmup >= 3 and a.workload == "dense" and a.n == 8192
    assert a.methods == "bicgstab,cgnr,qmr" and a.tol == 1e-10
    d = bench.parse_args(["--workload", "dipole"])
    assert d.L == 64 and d.methods == "cocg,bicgstab" and d.tol == 1e-8
    b = bench.parse_args(["--workload", "batched"])
    assert b.nrhs == 256 and b.methods == "bicgstab"
    assert a.default_run and not a.no_other and a.requests == 2000 and a.baseline_requests >= 200
    assert not d.default_run and not b.default_run


def test_cpu_baseline_rows_and_reference_line(capsys, monkeypatch):
    """The CPU baseline times the oracle's serial and OpenMP builds on both
    paths with every method, and states the threads used; the reference arm
    prints one JSON line of the same metric (a small system here)."""
    import json

    import bench
    from paper_1208_4869_gb300 import workloads as W
    A, y = W.dense_system(96, 3.0, 0)
    rows = bench.cpu_baseline_rows(A, y, ["bicgstab", "cgnr", "qmr"], 1e-10, 300, 1e-5, budget_s=0.0)
    got = {(r["build"], r.get("path")) for r in rows}
    assert ("serial", "mixed") in got and ("serial", "fp64") in got
    for r in rows:
        if "unavailable" in r:
            continue
        assert r["solves"] == 3 and r["value"] > 0 and r["threads"] >= 1
        assert r["max_true_relres"] <= 1e-10
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert bench.run_reference(bench.parse_args(["--impl", "reference", "--n", "96", "--steps", "3",
                                                 "--warmup", "0"])) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["steps"] == 3
    assert line["cpu_baseline"]["cores"] >= 1 and line["max_true_relres"] <= 1e-10
    assert line["config"]["path"] == "mixed"
