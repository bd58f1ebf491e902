"""Host logic of the benchmark's multi-replica path, on CPU with gloo ranks:
per-rank seeds, max-over-ranks timing, and the reference arm's rank rule."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_env()
    t = bench.max_over_ranks(10.0 * (r + 1), w)
    bench.barrier(w)
    q.put((r, local, bench.replica_seed(1234, r), t))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    assert [o[2] for o in out] == [1234, 1235]  # independent replicas
    assert all(o[3] == 20.0 for o in out)  # max over ranks


def test_reference_arm_runs_on_rank_zero_only():
    args = bench.parse_args(["--impl", "reference", "--steps", "2", "--warmup", "1", "--ref-L", "64"])
    assert bench.run_reference(args, 2, 1) is None
    res = bench.run_reference(args, 1, 0)
    assert res["impl"] == "reference" and res["unit"] == "flips/ns" and res["value"] > 0
    assert res["e2e"]["h2d_bytes_per_step"] == 0 and res["cpu_baseline"]["kind"] == "oracle"


def test_cpu_baseline_reports_the_host():
    """The CPU baseline names the host it ran on (core count, CPU model) and
    the threads the oracle used."""
    args = bench.parse_args(["--cpu-L", "64", "--cpu-sweeps", "2", "--cpu-short"])
    res = bench.cpu_baseline(args)
    assert res["kind"] == "oracle" and res["value"] > 0 and res["cores"] >= 1
    assert res["nproc"] == os.cpu_count() and isinstance(res["cpu_model"], str)


def test_integrated_time_of_an_ar1_series():
    """The package's effective-sample estimator: tau_int of AR(1) with
    coefficient phi is (1 + phi) / (2 (1 - phi))."""
    import numpy as np

    from paper_1906_06297_gb300 import analysis

    rng = np.random.default_rng(1)
    phi, n = 0.7, 300_000
    eps = rng.standard_normal(n)
    x = np.empty(n)
    x[0] = 0.0
    for i in range(1, n):
        x[i] = phi * x[i - 1] + eps[i]
    tau = analysis.integrated_time(x)
    assert abs(tau - (1 + phi) / (2 * (1 - phi))) < 0.2
    e = analysis.effective_samples([x[: n // 2], x[n // 2:]])
    assert abs(e["effective"] - n / (2 * e["tau_int"])) < 1e-6
