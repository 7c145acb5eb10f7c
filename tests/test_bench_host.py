"""Host logic of the benchmark's multi-process path, on CPU: under torchrun
each rank runs its own replica of the workload (the path has no data
exchange), the ranks meet at barriers around the timed region, the job's
time is the slowest rank's (a MAX all-reduce) and the reference arm runs on
rank 0 only.  Two ranks over gloo stand in for two GPUs over NCCL."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        w, r, local = bench._dist()
        bench._barrier(w)
        slowest = bench._max_over_ranks(10.0 + 5.0 * r, w)  # rank-dependent "times"
        bench._barrier(w)
        with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
            json.dump({"world": w, "rank": r, "local": local, "max": slowest}, f)
    finally:
        dist.destroy_process_group()


def test_two_ranks_agree_on_the_slowest_time(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, d in enumerate(res):
        assert d["world"] == world and d["rank"] == r and d["local"] == r
        assert d["max"] == 15.0


def test_single_process_needs_no_process_group(monkeypatch):
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench._dist() == (1, 0, 0)
    assert bench._max_over_ranks(3.5, 1) == 3.5
    bench._barrier(1)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import argparse

    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    bench.run_reference(argparse.Namespace(steps=1, warmup=0, level=9))
    assert capsys.readouterr().out == ""


def test_partme_counts_work_units_and_coarse_solves():
    """E_parTME = t n_c mu_sm / n (Sec. 5) with mu_sm = n / t_WU: the FMG time
    in work units; without the coarse grid it leaves out one coarse solve
    before the first level and one per cycle on each finer level."""
    import bench

    class FakeMesh:
        coarsest = 2

        def time_op(self, level, op, precision=0, reps=10):
            return {("residual", 0): 4.0, ("residual", 1): 2.0,
                    ("coarse_solve", 0): 1.0, ("coarse_solve", 1): 0.5}[(op, precision)]

    lb = bench.LevelBench.__new__(bench.LevelBench)
    lb.mesh, lb.level, lb.dofs = FakeMesh(), 9, 1000
    fmg = {"V22_fp64": {"ms": 400.0}, "2V22_fp64": {"ms": 800.0},
           "V22_fp32ir": {"ms": 200.0}, "2V22_fp32ir": {"ms": 300.0}}
    r = lb.partme(fmg)
    assert r["mu_sm_lups"]["fp64"] == pytest.approx(1000 / 4e-3)
    assert r["V22_fp64"]["E_parTME"] == pytest.approx(100.0)
    assert r["V22_fp64"]["E_parTME_wcg"] == pytest.approx((400.0 - 1.0 - 7 * 1.0) / 4.0)
    assert r["2V22_fp64"]["E_parTME_wcg"] == pytest.approx((800.0 - 1.0 - 14 * 1.0) / 4.0)
    # FP32 corrections: the first coarse solve is FP64, the cycles' are FP32
    assert r["V22_fp32ir"]["E_parTME"] == pytest.approx(100.0)
    assert r["2V22_fp32ir"]["E_parTME_wcg"] == pytest.approx((300.0 - 1.0 - 14 * 0.5) / 2.0)
