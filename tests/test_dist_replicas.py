"""The bench's multi-GPU mode runs independent replicas ("replicas only": no data
is exchanged, thesis 5.2.2's screen-space sharding is not used on one-GPU machines).
Its host logic -- rendezvous, barrier, the max over ranks of the step time, the
whole-job value, and the reference arm printing on rank 0 only -- is checked
here with two gloo ranks on the CPU."""
import importlib.util
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    b = _bench()
    r, w, local = b.dist_env()
    b.dist_init(w, local)
    b.barrier(w)
    ms = b.max_over_ranks(1.0 + r, w)             # rank 1 is the slower one
    value = b.whole_job_value(1000.0, ms, w)
    b.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((r, w, ms, value))


def test_two_gloo_ranks_agree_on_the_slowest_step():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for r, w, ms, value in got:
        assert w == 2
        assert ms == 2.0                            # max over ranks
        assert value == pytest.approx(2 * 1000.0 / 2e-3 / 1e9)   # all ranks' units / slowest time


def test_single_rank_needs_no_process_group():
    b = _bench()
    assert b.max_over_ranks(3.5, 1) == 3.5
    assert b.whole_job_value(500.0, 2.0, 1) == pytest.approx(500.0 / 2e-3 / 1e9)


@pytest.mark.parametrize("rank", [0, 1])
def test_reference_arm_prints_on_rank_zero_only(rank):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--workload", "cfg1", "--steps", "2", "--warmup", "1"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    if rank != 0:
        assert lines == []
        return
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 1              # the steps asked for, well inside the time cap
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
