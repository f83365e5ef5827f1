"""Views spread over two ranks (gloo, CPU): the multi-process host logic of a multi-GPU run.

Each rank renders its slice of one batch of views (with the oracle standing in for the GPU path), the slices
together equal the single-process render of the whole batch, and the timing reduction takes the slowest rank.
"""
import importlib.util
import json
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
W, H, V, N = 64, 32, 5, 300


def _replicas():
    # loaded by path: the module needs only torch, not the CUDA library the package loads on import
    spec = importlib.util.spec_from_file_location("omnigs_replicas",
                                                  os.path.join(ROOT, "paper_2404_03202_gb300", "replicas.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _scene_and_poses():
    import synth
    return synth.shell_scene(N, 7), synth.random_viewmats(V, 8)


def _worker(rank, world, port, outdir):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        R = _replicas()
        scene, poses = _scene_and_poses()
        a, b = R.view_range(V, world, rank)
        img = oracle.render(scene, poses[a:b], W, H)["rgb"] if b > a else np.zeros((0, 3, H, W))
        # gather every rank's slice (variable length: pad to the largest slice)
        counts = [R.view_range(V, world, r)[1] - R.view_range(V, world, r)[0] for r in range(world)]
        buf = torch.zeros((max(counts), 3, H, W), dtype=torch.float64)
        buf[: b - a] = torch.from_numpy(np.asarray(img, dtype=np.float64))
        parts = [torch.zeros_like(buf) for _ in range(world)]
        dist.all_gather(parts, buf)
        slowest = R.max_over_ranks(10.0 + rank)
        if rank == 0:
            full = np.concatenate([parts[r][: counts[r]].numpy() for r in range(world)])
            np.save(os.path.join(outdir, "gathered.npy"), full)
        with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
            json.dump({"range": [a, b], "slowest": slowest}, f)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2])
def test_views_sharded_over_ranks_match_one_process(tmp_path, world, oracle_lib):
    import oracle
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert [g["range"] for g in got] == [[0, 3], [3, 5]]
    assert all(g["slowest"] == 10.0 + world - 1 for g in got)
    scene, poses = _scene_and_poses()
    whole = oracle.render(scene, poses, W, H)["rgb"]
    assert (whole > 0).mean() > 0.2  # the views are not blank
    assert np.array_equal(np.load(tmp_path / "gathered.npy"), whole)


def test_view_range_partitions_every_batch():
    R = _replicas()
    for views in range(0, 20):
        for world in range(1, 9):
            spans = [R.view_range(views, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == views
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        R.view_range(4, 2, 2)


def test_max_over_ranks_without_a_process_group():
    assert _replicas().max_over_ranks(3.25) == 3.25
