"""The N > 1 host logic of bench.py on CPU: two gloo ranks.

The path does not shard (each replica solves its own sequence), so the only
cross-rank steps are the barrier and the max over ranks of the timed regions.
These tests run them as two processes on the gloo backend; nothing here needs a
GPU."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
dist.init_process_group("gloo")
import bench
r = dist.get_rank()
# rank 0: 100 ms over 10 systems, 10 ms end to end; rank 1: 200 ms and 5 ms
ms, e2e = bench.reduce_over_ranks(100.0 * (r + 1), 5.0 * (2 - r), 10, dist.get_world_size(), "cpu")
dist.barrier()
print(json.dumps([r, ms, e2e]), flush=True)
dist.destroy_process_group()
"""


def free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def run_ranks(code, world, extra_env=None):
    port = free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        env.update(extra_env or {})
        procs.append(subprocess.Popen(code, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True, cwd=ROOT))
    outs = []
    try:
        for p in procs:
            out, err = p.communicate(timeout=180)
            outs.append((p.returncode, out, err))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    return outs


def test_max_over_ranks_gloo_world2():
    outs = run_ranks([sys.executable, "-c", WORKER.format(root=ROOT)], 2)
    got = {}
    for rc, out, err in outs:
        assert rc == 0, err[-2000:]
        r, ms, e2e = json.loads(out.strip().splitlines()[-1])
        got[r] = (ms, e2e)
    # the slowest replica ends the job: 200 ms for 2 x 10 systems; 10 ms end to end for 2
    assert got[0] == got[1] == (10.0, 5.0)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(84.0, 83.0, 4, 1, "cpu") == (21.0, 83.0)


def test_replica_seeds_are_distinct():
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    seeds = {bench.replica_rhs_seed(r, i) for r in range(8) for i in range(20)}
    assert len(seeds) == 8 * 20
    a, b = W.rhs(64, bench.replica_rhs_seed(0, 3)), W.rhs(64, bench.replica_rhs_seed(1, 3))
    assert not (a == b).all()


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun only rank 0 times the oracle; rank 1 prints nothing and exits 0."""
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(free_port()), CUDA_VISIBLE_DEVICES="")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""
