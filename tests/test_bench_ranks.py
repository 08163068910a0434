"""The multi-rank path of bench.py on CPU (gloo, world size 2): each rank runs its own
replica, the job's time is the slowest rank's and its vehicle-steps are the sum over
ranks; the reference arm runs on rank 0 only and the other ranks leave without output."""
import importlib.util
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        b = _bench()
        # rank r took (r + 1) seconds for 100 (r + 1) vehicle-steps
        secs, vs = b.reduce_over_ranks(float(rank + 1), 100 * (rank + 1), world, "cpu")
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"secs": secs, "veh_steps": vs}, f)
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_two_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        got = json.load(open(tmp_path / f"rank{r}.json"))
        assert got == {"secs": 2.0, "veh_steps": 300.0}     # max of the times, sum of the work


def test_single_rank_is_identity():
    b = _bench()
    assert b.reduce_over_ranks(1.5, 42, 1, "cpu") == (1.5, 42)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    b = _bench()
    calls = []

    def fake_time_oracle(frac, steps, warmup, budget_s=None):
        calls.append((frac, steps, warmup))
        return dict(value=1.0e6, steps=steps, seconds=1.0, veh_steps=int(1e6), trips=300000)

    monkeypatch.setattr(b, "time_oracle", fake_time_oracle)
    args = b.argparse.Namespace(sample_frac=0.1, steps=3, warmup=1, gpus=2)
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    b.run_reference(args)
    assert calls == [] and capsys.readouterr().out == ""
    monkeypatch.setenv("RANK", "0")
    b.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip())
    assert calls == [(0.1, 3, 1)]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] == 1.0e6
    assert line["e2e"] == {"value": 1.0e6, "unit": line["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["cpu_baseline"]["kind"] == "oracle"
