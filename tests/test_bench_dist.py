"""Host logic of bench.py for N > 1 ranks (replicas only), on CPU with gloo:
each rank times its own replica box; the job's time is the slowest rank's
and the value counts the nodes of every rank."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, local, ws = bench.dist_setup()          # gloo on a machine without CUDA
    bench.barrier(ws)
    t = bench.max_over_ranks(times[r], ws)
    v = bench.job_mlups(1000, 10, t, ws)
    out.put((r, ws, t, v))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_gloo_max_time_and_job_value():
    import torch
    import torch.multiprocessing as mp
    if torch.cuda.is_available():
        pytest.skip("exercises the CPU (gloo) path")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [12.5, 20.0]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, ws, t, v in res:
        assert ws == 2
        assert t == 20.0                          # slowest rank
        assert abs(v - 2 * 1000 * 10 / 0.020 / 1e6) < 1e-9


def test_single_rank_helpers():
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert abs(bench.job_mlups(512 ** 3, 50, 5000.0, 1) - 512 ** 3 * 50 / 5.0 / 1e6) < 1e-6
    args = bench.parse_args([])
    assert (args.gpus, args.steps, args.warmup, args.impl, args.size) == (1, 50, 5, "ours", 512)


# ---------------------------------------------------------------------------
# The source hash that ties a traffic record to its kernel


def _bench():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    return bench


def test_strip_comments_keeps_code_and_literals():
    b = _bench()
    src = ('int a = 1; // c\n/* x\n y */ char s[] = "a // b \\" /* c */";\n'
           "char q = '\"';\n\n  // only a comment\nint b;  \n")
    assert b.strip_comments(src) == ('int a = 1;\n  char s[] = "a // b \\" /* c */";\n'
                                     "char q = '\"';\nint b;")
    # a change of code changes the hash input, a change of comment does not
    assert b.strip_comments("x = 1; // one") == b.strip_comments("x = 1; // uno")
    assert b.strip_comments("x = 1;") != b.strip_comments("x = 2;")



def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference (the oracle on the host cores) prints one
    JSON line with the keys the benchmark contract names, on CPU."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True,
                         timeout=600, cwd=root, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "MLUPS"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"]
