"""Host logic of the bench's multi-GPU path on CPU: two ranks over gloo (one
process per rank, rendezvous on 127.0.0.1), and the reference arm's rank
gating.  Ranks solve independent problems (weak scaling, no exchange on the
data path); the job's time is the slowest rank's and its rate counts every
rank's units."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    sys.path.insert(0, ROOT)
    import bench
    spec = bench.workload_spec("n128", rank)
    ms = bench.max_over_ranks(10.0 * (rank + 1), ws, "cpu")
    rate = bench.whole_job_rate(ws, 100, ms)
    with open(os.path.join(out_dir, "r%d.json" % rank), "w") as fh:
        json.dump({"spec": spec, "ms": ms, "rate": rate, "env": bench.dist_env()}, fh)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo_max_time_and_whole_job_rate(tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    r = [json.load(open(tmp_path / ("r%d.json" % k))) for k in range(2)]
    assert r[0]["ms"] == r[1]["ms"] == 20.0          # slowest rank
    assert r[0]["rate"] == pytest.approx(2 * 100 / 0.020)
    assert r[0]["env"] == [2, 0, 0] and r[1]["env"] == [2, 1, 1]
    s0, s1 = r[0]["spec"], r[1]["spec"]
    assert s0["seed"] != s1["seed"]                  # independent problems ...
    assert {k: v for k, v in s0.items() if k != "seed"} == {k: v for k, v in s1.items() if k != "seed"}


def _run_bench(args, env_extra, timeout=600):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT,
                          env=env, capture_output=True, text=True, timeout=timeout)


def test_reference_arm_other_ranks_exit_without_work():
    p = _run_bench(["--impl", "reference", "--gpus", "2", "--workload", "n32", "--steps", "5",
                    "--warmup", "1", "--ref-budget", "1"],
                   {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""


def test_reference_arm_prints_one_contract_line():
    # (5 oracle iterations at n = 32 take milliseconds; the budget only guards against a slow host)
    p = _run_bench(["--impl", "reference", "--workload", "n32", "--steps", "5", "--warmup", "1",
                    "--ref-budget", "20"], {"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["higher_is_better"] is True
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "dtype",
              "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    # one step is one oracle iteration: K of them when they fit the time budget
    assert d["steps"] == 5 and d["requested_steps"] == 5


def test_launch_counts_include_the_skipped_tail_of_a_loop_body():
    import bench
    # single image: 16 iterations per loop body; shared-A batch: 4
    # fixed-count runs launch exactly their iterations; a run stopped by tol at k of
    # max_iter = 5000 (312 bodies + 8) launches the rest of its body and the last 8
    assert [bench.loop_launch_iters(k) for k in (1, 16, 17, 300, 30000)] == [1, 16, 17, 300, 30000]
    assert [bench.loop_launch_iters(k, 5000) for k in (1, 16, 17, 2403, 4995, 5000)] == \
        [24, 24, 40, 2424, 5000, 5000]
    assert [bench.batch_launch_iters(k) for k in (1, 4, 7, 300)] == [4, 4, 8, 300]
    # a 128 x 128 batch (G's partial tiles added by the u-solve) against another side
    assert bench.batch_launches(300) == 5 * 300 + 14
    assert bench.batch_launches(7, g_in_usolve=False) == 6 * 8 + 12
