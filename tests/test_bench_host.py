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


def test_seconds_to_error_of_ar1_series():
    """For AR(1) with coefficient phi and unit innovations the per-sample
    variance is 1/(1 - phi^2) and tau = (1 + phi)/(2(1 - phi)); the time to a
    standard error eps is seconds * 2 tau var / (eps^2 N), and halving eps
    quadruples it."""
    import numpy as np

    from paper_1906_06297_gb300 import analysis

    rng = np.random.default_rng(3)
    phi, n, chains = 0.6, 100_000, 4
    xs = []
    for _ in range(chains):
        eps_ = rng.standard_normal(n)
        x = np.empty(n)
        x[0] = eps_[0] / np.sqrt(1 - phi * phi)
        for i in range(1, n):
            x[i] = phi * x[i - 1] + eps_[i]
        xs.append(x)
    r = analysis.seconds_to_error(xs, seconds=2.0, eps=0.01)
    tau, var = (1 + phi) / (2 * (1 - phi)), 1 / (1 - phi * phi)
    assert abs(r["tau_int"] - tau) < 0.1 * tau and abs(r["var"] - var) < 0.05 * var
    want = 2.0 * 2 * tau * var / (0.01 ** 2 * n * chains)
    assert abs(r["seconds_to_error"] - want) < 0.15 * want
    assert r["reliable"] and r["series_over_tau"] > 50
    r2 = analysis.seconds_to_error(xs, seconds=2.0, eps=0.005)
    assert abs(r2["seconds_to_error"] / r["seconds_to_error"] - 4.0) < 1e-9
    short = analysis.seconds_to_error([x[:20] for x in xs], seconds=1.0, eps=0.01)
    assert not short["reliable"]
