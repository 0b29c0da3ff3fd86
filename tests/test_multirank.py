"""The multi-rank path of bench.py on CPU, as two gloo ranks. The path does not
shard, so under torchrun every rank runs an independent replica. The ranks meet
in a barrier and in a max-reduction of the timed region, and the job's value
counts every rank's nodes over the slowest rank's time. The oracle arm runs on
rank 0 alone: the other ranks return at once."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import contextlib
    import io

    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        bench.barrier(dist)
        ms = bench.max_over_ranks(dist, 10.0 + 5.0 * rank)  # rank r took 10 + 5r ms
        value = bench.job_mlups(world, 1000, 10, ms)
        buf = io.StringIO()
        rc = None
        if rank != 0:
            class A:  # the arguments the oracle arm reads before it checks the rank
                steps, warmup, gpus = 2, 3, world
            with contextlib.redirect_stdout(buf):
                rc = bench.reference_arm(A, rank, dist)
        bench.barrier(dist)
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"ms": ms, "value": value, "rc": rc, "printed": buf.getvalue()}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_by_the_slowest_and_count_every_rank(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for r in res:
        assert r["ms"] == 15.0                      # the slowest rank's time, on every rank
        assert abs(r["value"] - 2 * 1000 * 10 / 0.015 / 1e6) < 1e-12
    assert res[1]["rc"] == 0 and res[1]["printed"] == ""  # no oracle work, no line, off rank 0


def test_bench_run_record_appends_a_json_line(tmp_path, capsys):
    """bench.py --record: the printed line is also appended, with time and host,
    to a JSON-lines run log; a second run appends a second line."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import argparse
    import bench
    log = tmp_path / "runs.jsonl"
    args = argparse.Namespace(record=str(log))
    bench.emit(args, {"metric": "m", "value": 1.5})
    bench.emit(args, {"metric": "m", "value": 2.5})
    printed = [json.loads(x) for x in capsys.readouterr().out.strip().splitlines()]
    assert [p["value"] for p in printed] == [1.5, 2.5]
    recs = [json.loads(x) for x in log.read_text().splitlines()]
    assert [r["value"] for r in recs] == [1.5, 2.5]
    assert all("recorded_utc" in r and r["host"] == socket.gethostname() for r in recs)
