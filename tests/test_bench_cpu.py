"""Host logic of bench.py, on CPU: the multi-rank timing (replicas, one
process per GPU, max over ranks) with a world-size-2 gloo process group, the
whole-job value, and the CPU-oracle reference arm's JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(100.0 * (rank + 1), "cpu")  # rank 1 is the slow one
        with open(os.path.join(outdir, f"r{rank}"), "w") as f:
            f.write(repr(ms))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2(tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    got = [float(open(tmp_path / f"r{r}").read()) for r in range(2)]
    assert got == [200.0, 200.0]


def test_max_over_ranks_single_process():
    assert bench.max_over_ranks(123.5, "cpu") == 123.5


def test_job_value_counts_every_rank():
    # 2 ranks x 3 pencils of order 1024 in the slowest rank's 1.5 s
    v = bench.job_value(2, 3, 1024, 1500.0)
    assert v == pytest.approx(2 * 3 * (116.0 * 1024 ** 3 / 3.0) / 1.5 / 1e12, rel=1e-15)
    assert bench.job_value(1, 1, 16384, 1000.0) == pytest.approx(bench.f_nom(16384) / 1e12)


def _reference_arm(env_extra):
    env = dict(os.environ, **env_extra)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "128", "--cpu-sample", "48",
           "--steps", "1", "--warmup", "0"]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)


def test_reference_arm_prints_one_json_line():
    r = _reference_arm({"RANK": "0"})
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "TFLOP/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing():
    r = _reference_arm({"RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


@pytest.mark.parametrize("t_step,expect", [(40.0, (5, 20)), (66.0, (4, 20)), (72.0, (3, 19)), (400.0, (3, 1))])
def test_plan_steps_fits_the_budget(t_step, expect):
    """The wall-clock plan: the requested steps when they fit; else the
    warm-up shrinks to 3 (never below), then the timed steps (at least one);
    whatever it returns fits the budget when a timed step fits at all."""
    spent, budget, extra = 30.0 + t_step, 1700.0, 35.0
    w, k = bench.plan_steps(5, 20, t_step, spent, budget, extra)
    assert (w, k) == expect
    assert w >= 3 and k >= 1
    if t_step * 3 <= budget - spent - extra:
        assert spent + (w - 1 + k) * t_step + extra <= budget
