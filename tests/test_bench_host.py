"""Host-side bookkeeping of bench.py (no GPU): the box-row count behind bin_count's and bin_emit's algorithmic bytes,
and the radix-sort pass counts behind the sort stages."""
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import bench  # noqa: E402
import gpu_util  # noqa: E402
import oracle  # noqa: E402
import synth  # noqa: E402


def _brute_rows(py, ry, alive, T, H):
    """Tile rows a box [floor(py) - ry, floor(py) + ry] overlaps, one tile row at a time."""
    rows = 0
    for y, r, a in zip(py, ry, alive):
        if not a:
            continue
        iy = int(np.floor(y))
        rows += sum(1 for t in range(H // T) if t * T <= iy + r and (t + 1) * T - 1 >= iy - r)
    return rows


def test_box_rows_counts_the_tile_rows_of_every_box():
    W, H, T = 256, 128, 16
    sc = synth.shell_scene(1500, seed=5)
    vm = np.concatenate([synth.identity_viewmats(1), synth.random_viewmats(1, 8)])
    sp = oracle.splats_from_records(oracle.preprocess(sc, vm, W, H))
    packed = gpu_util.pack_splats(sp)
    rad = packed[:, 6].view(np.int32)
    ry, rx = (rad >> 16) & 0xFFFF, rad & 0xFFFF
    want = _brute_rows(packed[:, 1], ry, rx != 0, T, H)
    assert bench.box_rows(torch.from_numpy(packed), T, H) == want
    # boxes reaching past the top and bottom edges are clipped to the image
    edge = packed.copy()
    edge[:4, 1] = [0.2, -3.0, H - 0.5, H + 7.0]
    edge[:4, 6] = np.array([(40 << 16) | 1] * 4, np.int32).view(np.float32)
    want = _brute_rows(edge[:, 1], (edge[:, 6].view(np.int32) >> 16) & 0xFFFF,
                       (edge[:, 6].view(np.int32) & 0xFFFF) != 0, T, H)
    assert bench.box_rows(torch.from_numpy(edge), T, H) == want


def test_sort_pass_counts():
    # 9-bit digits at most, an even number of passes (the sorted keys land back in the first buffer)
    assert bench._sort_passes(16) == 2
    assert bench._sort_passes(13) == 2
    assert bench._sort_passes(35) == 4
    assert bench._sort_passes(19) == 4
    assert bench._sort_passes(1) == 2


def test_stage_bytes_packed_depth_sort_only_when_the_index_fits():
    sb = bench.stage_bytes(1_000_000, 8, 2048, 1024, 16, 10_000, 1_000)
    assert sb["depth_sort"] == 4 * 8_000_000 * 24 - 8_000_000 * 4
    assert sb["preprocess_fwd"] == 1_000_000 * 236 + 8_000_000 * (48 + 8)  # the projection writes the packed keys
    sb = bench.stage_bytes(1_000_000, 8, 2048, 1024, 16, 10_000, 1_000, equirect=False)
    assert sb["depth_sort"] == 4 * 8_000_000 * 32
    assert sb["preprocess_fwd"] == 1_000_000 * 236 + 8_000_000 * 48


def test_oracle_pool_times_a_bounded_sample_on_several_cores():
    """The cpu_baseline leg: spawned workers build the workload once and each time a bounded oracle sample at the
    same time; the step time is the mean per-core time divided by the core count."""
    pool = bench.OraclePool("shell-small", cores=2)
    try:
        ms, ms_core, desc = pool.round(0.5)
        ms2, _, _ = pool.round(0.5)
    finally:
        pool.close()
    assert pool.cores == 2
    assert ms > 0 and ms2 > 0 and abs(ms * 2 - ms_core) <= 1e-9 * ms_core
    assert "view 0 of 1" in desc and "tiles" in desc


def test_whole_oracle_step_on_one_and_several_cores():
    """The unsampled leg: shell-small (config 1) as one whole oracle step, single-threaded (every stage timed) and
    split over two spawned processes by tile rows."""
    out = bench.oracle_small_configs(2, names=("shell-small",))
    r = out["shell-small"]
    assert r["single_thread_ms"] > 0 and r["all_cores_ms"] > 0 and r["cores"] == 2
    assert set(r["single_thread_stages_ms"]) == {"preprocess", "bin_sort", "blend_fwd_bwd", "preprocess_bwd"}
    assert abs(sum(r["single_thread_stages_ms"].values()) - r["single_thread_ms"]) <= 1e-6 * r["single_thread_ms"]


def test_render_bwd_traffic_figure_belongs_to_the_current_adjoint():
    """The bench reports the adjoint's measured DRAM traffic only while the adjoint's source is the one it was
    measured on; this fails when the kernel changes without a new capture."""
    import hashlib
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "paper_2404_03202_gb300", "csrc", "render.cu")) as f:
        src = bench.render_bwd_source(f.read())
    assert hashlib.sha256(src.encode()).hexdigest() == bench.RENDER_BWD_TRAFFIC["source_sha256"]
