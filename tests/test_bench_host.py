"""Host-side logic of bench.py on CPU: the multi-rank aggregation over a
world_size-2 gloo group, the algorithmic byte model, and the JSON contract of
the reference (oracle) arm."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sec, frames = bench.aggregate(1.0 + rank, 10 + rank, world)
    out.put((rank, sec, frames))
    bench.barrier(world)
    dist.destroy_process_group()


def test_aggregate_max_time_sum_frames_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, sec, frames in res:
        assert sec == 2.0 and frames == 21       # max over ranks, sum of frames


def test_stage_bytes_model():
    sys.path.insert(0, ROOT)
    import bench
    import scenes
    sc = scenes.config1()
    b = bench.stage_bytes(sc)
    R2, WH = 256 * 256, 256 * 256
    assert b["filter"] == R2 * 17 and b["bwd_filter"] == R2 * 28
    # the final antialiasing reads only its listed pixels; the shading writes the colour and the image
    assert b["final_antialias"] == 0 and b["shade"] == WH * 49 + 8 * R2 + 24 * sc["verts"].shape[0]
    listed = bench.stage_bytes(sc, [10, 20])
    assert listed["final_antialias"] == 20 * 52 and listed["sm_antialias"] == 10 * 36
    assert set(b) >= {"raster", "sm_antialias", "shade", "bwd_sm_interp", "bwd_sm_antialias", "bwd_shade", "setup"}


@pytest.mark.slow
def test_reference_arm_json_contract():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "config1", "--steps", "1", "--warmup", "3"], capture_output=True, text=True, env=env,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    d = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config",
              "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["e2e"]["h2d_bytes_per_step"] == 0 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"


def _partition_worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    import scenes
    dist.init_process_group("gloo", rank=rank, world_size=world)
    costs = [bench.scene_cost(sc) for sc in scenes.config4()]
    mine = bench.partition_scenes(costs, world)[rank]
    got = [None] * world
    dist.all_gather_object(got, mine)
    out.put((rank, got, costs))
    dist.destroy_process_group()


def test_config4_scene_partition_covers_every_scene_once_gloo():
    """Config 4's scenes split over two gloo ranks (the multi-GPU batch):
    each rank computes its own share; together they hold every scene exactly
    once, with costs within 5 % of each other."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_partition_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=300) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, parts0, costs), (_, parts1, _) = res
    assert parts0 == parts1                       # every rank derives the same split
    flat = sorted(k for part in parts0 for k in part)
    assert flat == list(range(len(costs)))
    loads = [sum(costs[k] for k in part) for part in parts0]
    assert max(loads) <= 1.05 * min(loads), loads


def test_partition_is_balanced_for_uneven_costs():
    sys.path.insert(0, ROOT)
    import bench
    costs = [100, 1, 1, 1, 50, 49]
    parts = bench.partition_scenes(costs, 2)
    assert sorted(parts[0] + parts[1]) == list(range(6))
    assert sorted(sum(costs[k] for k in p) for p in parts) == [101, 101]
