"""The multi-rank host path on CPU: rank layout, the partition of independent snapshots
over ranks, and the scalar reductions (slowest rank's time, units summed over ranks),
run as world_size-2 ``gloo`` process groups.

Each rank coarse-grains its own share of a small batch of snapshots with the oracle; the
gathered results must equal, bit for bit, the same snapshots coarse-grained in one
process, so the partition loses, duplicates and alters nothing.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from paper_1409_0001_gb300.ranks import dist_env, reduce_scalar, shard_by_cost

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_dist_env_layouts():
    assert dist_env({}) == (1, 0, 0)
    assert dist_env({"WORLD_SIZE": "4", "RANK": "3", "LOCAL_RANK": "3"}) == (4, 3, 3)
    with pytest.raises(ValueError):
        dist_env({"WORLD_SIZE": "2", "RANK": "2"})
    with pytest.raises(ValueError):
        dist_env({"WORLD_SIZE": "0"})


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_is_a_balanced_partition(world):
    rng = np.random.default_rng(world)
    costs = (rng.integers(32, 97, 64) ** 3).tolist()       # cells of 32^3..96^3 snapshots
    shards = [shard_by_cost(costs, world, r) for r in range(world)]
    flat = sorted(i for s in shards for i in s)
    assert flat == list(range(len(costs)))                 # every item once
    loads = [sum(costs[i] for i in s) for s in shards]
    assert max(loads) <= sum(costs) / world + max(costs)   # list-scheduling bound
    assert shards == [shard_by_cost(costs, world, r) for r in range(world)]   # deterministic


def test_shard_edge_cases():
    assert shard_by_cost([], 2, 0) == [] and shard_by_cost([], 2, 1) == []
    assert shard_by_cost([5.0], 3, 0) == [0] and shard_by_cost([5.0], 3, 2) == []
    assert sorted(shard_by_cost([1, 1, 1, 1], 2, 0) + shard_by_cost([1, 1, 1, 1], 2, 1)) == [0, 1, 2, 3]
    with pytest.raises(ValueError):
        shard_by_cost([1], 2, 2)


def test_reduce_without_process_group_is_identity():
    assert reduce_scalar(3.5, "max") == 3.5
    with pytest.raises(ValueError):
        reduce_scalar(1.0, "min")


WORKER = r"""
import json, os, sys, time
sys.path.insert(0, os.environ["REPO_ROOT"])
import numpy as np
import torch.distributed as dist
import oracle
import workloads as W
from paper_1409_0001_gb300.ranks import dist_env, reduce_scalar, shard_by_cost

ws, rank, local = dist_env()
dist.init_process_group("gloo")
oracle.build()
cases = W.batched_snapshots(n_snap=7, side_lo=5, side_hi=11, logn_lo=2.0, logn_hi=3.0, seed=3)
mine = shard_by_cost([c.ncells for c in cases], ws, rank)
t0 = time.perf_counter()
res, units = {}, 0.0
for i in mine:
    c = cases[i]
    _, eps, nout, _ = oracle.coarse_grain_structured(c.dims, c.origin, c.dx, c.pos, c.w, c.b,
                                                     c.nsteps)
    res[i] = eps.tobytes().hex()
    units += c.nsteps * c.ncells
dt = time.perf_counter() - t0
gathered = [None] * ws
dist.all_gather_object(gathered, res)
out = {"rank": rank, "mine": mine, "t": dt, "units": units,
       "t_max": reduce_scalar(dt, "max"), "units_sum": reduce_scalar(units, "sum"),
       "rank_max": reduce_scalar(rank + 1, "max"), "rank_sum": reduce_scalar(rank + 1, "sum")}
if rank == 0:
    merged = {}
    for g in gathered:
        merged.update(g)
    out["results"] = merged
with open(os.path.join(os.environ["OUT_DIR"], "rank%d.json" % rank), "w") as f:
    json.dump(out, f)
dist.barrier()
dist.destroy_process_group()
"""


def test_two_gloo_ranks_shard_snapshots(orc, tmp_path):
    import workloads as W

    script = tmp_path / "worker.py"
    script.write_text(WORKER)
    port = free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(r), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), REPO_ROOT=ROOT,
                   OUT_DIR=str(tmp_path))
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
    for p in procs:
        out, _ = p.communicate(timeout=240)
        assert p.returncode == 0, out.decode()[-2000:]
    r0 = json.loads((tmp_path / "rank0.json").read_text())
    r1 = json.loads((tmp_path / "rank1.json").read_text())
    assert sorted(r0["mine"] + r1["mine"]) == list(range(7))
    assert r0["rank_max"] == r1["rank_max"] == 2.0
    assert r0["rank_sum"] == r1["rank_sum"] == 3.0
    assert r0["t_max"] == r1["t_max"] == max(r0["t"], r1["t"])
    assert r0["units_sum"] == r1["units_sum"] == r0["units"] + r1["units"]

    cases = W.batched_snapshots(n_snap=7, side_lo=5, side_hi=11, logn_lo=2.0, logn_hi=3.0, seed=3)
    assert r0["units_sum"] == sum(c.nsteps * c.ncells for c in cases)
    assert sorted(int(k) for k in r0["results"]) == list(range(7))
    for i, c in enumerate(cases):
        _, eps, _, _ = orc.coarse_grain_structured(c.dims, c.origin, c.dx, c.pos, c.w, c.b,
                                                   c.nsteps)
        assert r0["results"][str(i)] == eps.tobytes().hex()


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       env=env, capture_output=True, timeout=120)
    assert p.returncode == 0
    assert p.stdout.strip() == b""
