"""The multi-rank bench path on CPU: two gloo ranks (no data-path collective)
combine their timed regions by MAX and their iterations by SUM, agree on the
split of a batch of independent LPs without an exchange, and the reference arm
runs on rank 0 alone."""
import json
import os
import socket
import types

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, figures, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=len(figures))
    try:
        out[rank] = bench.combine_ranks(*figures[rank], len(figures))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_all_iterations():
    figures = [(1.25, 896), (1.5, 960)]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(_free_port(), figures, out), nprocs=2, join=True,
                           start_method="spawn")
        got = dict(out)
    assert got[0] == got[1] == (1.5, 1856.0)
    # whole-job throughput = units of every rank / the slowest rank's time
    assert got[0][1] / got[0][0] == pytest.approx(1856 / 1.5)


def test_one_rank_keeps_its_own_figures():
    assert bench.combine_ranks(2.0, 700, 1) == (2.0, 700.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    calls = []
    monkeypatch.setattr(bench, "cpu_oracle_sample", lambda iters: calls.append(iters) or
                        {"value": 50.0, "unit": bench.UNIT, "cores": 1, "kind": "oracle",
                         "sample": "stub"})
    args = types.SimpleNamespace(warmup=3, steps=2, cpu_sample_iters=40, gpus=2)
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(args)
    assert calls == [] and capsys.readouterr().out == ""
    monkeypatch.setenv("RANK", "0")
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip())
    assert calls == [40] * 5
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] == 50.0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0


def test_shard_by_nnz_is_a_balanced_partition():
    sizes = np.random.default_rng(5).integers(10_000, 2_000_000, 256).tolist()
    for ws in (1, 2, 3, 8):
        parts = bench.shard_by_nnz(sizes, ws)
        assert len(parts) == ws
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))          # each LP on exactly one rank
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)    # greedy bound
        assert parts == bench.shard_by_nnz(sizes, ws)   # the same split on every call
    # 9 -> rank 0, 7 -> rank 1, 5 -> rank 1 (load 7 < 9), 1 -> rank 0 (load 9 < 12)
    assert bench.shard_by_nnz([5, 9, 7, 1], 2) == [[1, 3], [0, 2]]


def _split_rank(rank, port, sizes, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        mine = bench.shard_by_nnz(sizes, 2)[rank]  # computed locally, no exchange
        got = [None, None]
        dist.all_gather_object(got, mine)      # gathered here only to check them
        out[rank] = got
    finally:
        dist.destroy_process_group()


def test_two_ranks_agree_on_the_split_without_an_exchange():
    sizes = np.random.default_rng(6).integers(1, 10**6, 37).tolist()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.start_processes(_split_rank, args=(_free_port(), sizes, out), nprocs=2, join=True,
                           start_method="spawn")
        got = dict(out)
    assert got[0] == got[1]
    a, b = got[0]
    assert not set(a) & set(b) and sorted(a + b) == list(range(37))


@pytest.mark.parametrize("argv", [["--workload", "energy"], ["--workload", "fp"], ["--kernels-only"]])
def test_single_gpu_workloads_leave_other_ranks_idle(argv):
    import subprocess
    import sys
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(os.path.dirname(bench.__file__), "bench.py"),
                          *argv], env=env, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout == ""


def test_all_core_oracle_sample_times_replicas_started_together():
    """The replicas wait for one wall-clock start; the rate is all their iterations over
    the span from the earliest start to the latest end, not a sum of separate rates."""
    d = bench.cpu_oracle_all_cores(iters=2, procs=2)
    assert d["cores"] == 2 and d["kind"] == "oracle" and d["value"] > 0
    assert "2 single-threaded replicas started together" in d["sample"]
    spread = float(d["sample"].split("starts spread over ")[1].split(" s")[0])
    assert spread < 0.5


def test_roofline_traffic_comes_from_the_committed_capture():
    """bench.py reads the DRAM bytes per launch of its roofline kernel from the committed
    ncu summary, and reports none for a kernel or precision that was not captured."""
    assert bench.ncu_traffic("dual_step", "bf16") == 7_759_360
    assert bench.ncu_traffic("primal_step", "bf16") == 11_005_056
    assert bench.ncu_traffic("dual_step", "fp32", "energy") == 116_110_080
    assert bench.ncu_traffic("dual_step", "fp64") is None
    assert bench.ncu_traffic("persistent_attempt", "bf16") is None
    assert bench.ncu_traffic("dual_step", "bf16", "batch") is None
    kt = {"primal_step": {"ms": 0.033, "bytes": 169598404.0},
          "dual_step": {"ms": 0.042, "bytes": 135255364.0}}
    roof = bench.kernel_roofline(kt, 6794.5, "measured", "energy", "fp32")
    assert roof["kernel"] == "dual_step" and roof["traffic"] == 116_110_080
    assert bench.kernel_roofline(kt, 6794.5, "measured")["traffic"] is None
