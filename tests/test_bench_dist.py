"""The multi-replica (N > 1) host path of bench.py on CPU: two gloo ranks run
the same rendezvous, barrier and max-over-ranks helpers the GPU launch uses
(one process per GPU, replicas only: no data-path collective), and the
reference arm's rank handling under torchrun-style environments."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, sys
sys.path.insert(0, {root!r})
import bench
ws, rank, local = bench.dist_setup()
bench.dist_barrier(ws)
# per-rank timings: the job time is the slowest replica's
m = bench.dist_max(ws, 10.0 * rank + 1.5)
bench.dist_barrier(ws)
print(json.dumps({{"rank": rank, "local": local, "ws": ws, "max": m}}), flush=True)
import torch.distributed as dist
dist.destroy_process_group()
"""


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank: int, ws: int, port: int) -> dict:
    env = dict(os.environ)
    env.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
               LOCAL_RANK=str(rank), AC_BENCH_BACKEND="gloo", CUDA_VISIBLE_DEVICES="")
    return env


def test_two_gloo_ranks_agree_on_the_slowest_replica():
    port = _free_port()
    code = RANK_SCRIPT.format(root=ROOT)
    procs = [subprocess.Popen([sys.executable, "-c", code], env=_env(r, 2, port), cwd=ROOT,
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for r in range(2)]
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=180)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            pytest.fail("gloo ranks did not finish")
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["ws"] == 2 and o["local"] == o["rank"]
        assert o["max"] == pytest.approx(11.5)


def test_single_process_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.get(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    try:
        for k in env:
            os.environ.pop(k, None)
        ws, rank, local = bench.dist_setup()
        assert (ws, rank, local) == (1, 0, 0)
        bench.dist_barrier(ws)
        assert bench.dist_max(ws, 3.25) == 3.25
    finally:
        for k, v in env.items():
            if v is not None:
                os.environ[k] = v


def test_reference_arm_runs_on_rank_zero_only():
    # rank 1 of a two-rank launch leaves at once without output; rank 0 times
    # the oracle on a bounded sample and reports n_gpus = 2
    args = [sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--workload",
            "separation4096", "--ref-steps", "1", "--steps", "1", "--warmup", "0"]
    r1 = subprocess.run(args, env=_env(1, 2, _free_port()), cwd=ROOT, capture_output=True,
                        text=True, timeout=300)
    assert r1.returncode == 0, r1.stderr[-2000:]
    assert r1.stdout.strip() == ""
    r0 = subprocess.run(args, env=_env(0, 2, _free_port()), cwd=ROOT, capture_output=True,
                        text=True, timeout=300)
    assert r0.returncode == 0, r0.stderr[-2000:]
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
