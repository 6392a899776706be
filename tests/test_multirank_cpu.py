"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas, no data-path
collective) reduce their step times to the maximum on every rank and report the
whole-job throughput; the reference arm runs on rank 0 only."""
import json
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_max, value = bench.reduce_step_time(1.0 + rank, world, 1_000_000)
    r_env = bench._rank_env()
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms_max, value, r_env))


def test_two_ranks_take_the_slowest_rank_and_sum_the_work():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms_max, value, env in res:
        assert ms_max == 2.0                              # the slowest rank's step time
        assert value == pytest.approx(2 * 1.0 / 2e-3)     # 2 x 1 Mpix per step over 2 ms
        assert env[0] == rank and env[1] == world


def test_reference_arm_is_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, gpus = 1, 1, 2

    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""


def test_json_line_takes_numpy_values():
    """The bench line carries counts and errors computed with numpy (int64, float32,
    arrays): they serialise as plain JSON numbers and lists."""
    import numpy as np
    import bench
    line = {"parity": {"bracketed_pixels": np.int64(7), "err": np.float32(0.25), "tiles": np.arange(3),
                       "unmatched": [(1, 2, np.float64(0.5), np.int64(6), True)]}}
    assert json.loads(bench._dumps(line)) == {"parity": {"bracketed_pixels": 7, "err": 0.25, "tiles": [0, 1, 2],
                                                         "unmatched": [[1, 2, 0.5, 6, True]]}}


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    """The reference arm (the FP64 oracle on the host cores, one stratified tile per step at
    a small primitive count) prints one JSON line with the bench contract's keys, its own
    e2e (no copies) and a cpu_baseline describing the run."""
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")

    class Args:
        steps, warmup, gpus, prims, ref_tiles = 1, 0, 1, 20000, 1

    assert bench.run_reference(Args()) == 0
    out = capsys.readouterr().out.strip().splitlines()
    assert len(out) == 1
    line = json.loads(out[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "e2e", "cpu_baseline"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True and line["n_gpus"] == 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
