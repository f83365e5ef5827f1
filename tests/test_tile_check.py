"""Pins of the tile-list validity check (tests/tile_check.py) on the CPU.

The check decides whether a list that leaves (Gaussian, tile) pairs out of the oracle's instance-box lists is still
a correct binning (Sec. 3.3, Eq. 8). Here it is given lists built in Python: the box lists culled by the stated rule
in FP64 (it must accept them), the uncut box lists (it must reject them: they keep pairs far out of reach), and
lists broken by hand, one mistake each (it must reject every one, naming the rule).
"""
import numpy as np
import pytest

import oracle
import synth
from tests import tile_check as tc


def _lists(ranges, lst):
    return [list(lst[a:b]) for a, b in np.asarray(ranges)]


def _as_ranges(lists):
    sizes = np.array([len(L) for L in lists], np.int64)
    return np.stack([np.cumsum(sizes) - sizes, np.cumsum(sizes)], 1), np.array([i for L in lists for i in L], np.int64)


def _fp64_culled(sp, V, W, H, T, ranges, lst, camera=None):
    """The box lists with the stated row culling taken in FP64: a pair stays when its splat keeps whole rows (box
    over every column or, equirectangular, rx + T > W / 2; or det <= 1e-3 c0 c2) or when the ellipse grown to
    q (1.001) + 1e-3 reaches the tile's pixel-centre rectangle widened by one pixel in x."""
    TX = W // T
    tiles = np.arange(len(ranges), dtype=np.int64)
    t, _, s = tc._gather(np.asarray(ranges), lst, tiles)
    px, rx = np.asarray(sp["px"], np.float64), np.asarray(sp["rx"], np.int64)
    ix = np.floor(px).astype(np.int64)
    x0, x1 = np.floor_divide(ix - rx, T), np.floor_divide(ix + rx, T)
    wide = x1 - x0 + 1 >= TX
    if camera is not None:
        x0, x1 = np.maximum(x0, 0), np.minimum(x1, TX - 1)
        wide = x1 - x0 + 1 >= TX
    else:
        wide |= 2 * (rx + T) > W
    c0, c1, c2 = (np.asarray(sp[k], np.float64) for k in ("c0", "c1", "c2"))
    whole = wide | ~((c0 > 0) & (c2 > 0)) | (c0 * c2 - c1 * c1 <= 1e-3 * c0 * c2)
    q = oracle.splat_q(sp)
    keep = whole[s] | (tc.pair_reach(sp, s, t, W, H, T, 1.0, camera) <= q[s] * 1.001 + 1e-3)
    counts = np.bincount(t[keep], minlength=len(ranges))
    new_ranges = np.stack([np.cumsum(counts) - counts, np.cumsum(counts)], 1)
    return new_ranges, s[keep]


def _case(V=2, n=400, W=256, H=128, T=16, seed=5):
    sp = synth.random_splats(V, n, W, H, seed=seed, max_radius=30, wide_frac=0.05)
    sp = {k: (np.asarray(v, np.float64) if np.asarray(v).dtype.kind == "f" else v) for k, v in sp.items()}
    ranges, lst = oracle.bin_sort(sp, V, W, H, T)
    got_r, got_l = _fp64_culled(sp, V, W, H, T, ranges, lst)
    return sp, (V, W, H, T), (ranges, lst), (got_r, got_l)


def test_min_form_on_rect_against_dense_grid():
    rng = np.random.default_rng(0)
    for _ in range(200):
        sx, sy, rho = rng.uniform(0.5, 5), rng.uniform(0.5, 5), rng.uniform(-0.95, 0.95)
        s00, s11, s01 = sx * sx, sy * sy, rho * sx * sy
        det = s00 * s11 - s01 * s01
        c0, c1, c2 = s11 / det, -s01 / det, s00 / det
        x0, y0 = rng.uniform(-20, 20, 2)
        x1, y1 = x0 + rng.uniform(0, 10), y0 + rng.uniform(0, 10)
        u, v = np.meshgrid(np.linspace(x0, x1, 401), np.linspace(y0, y1, 401))
        dense = (c0 * u * u + 2 * c1 * u * v + c2 * v * v).min()
        got = float(tc.min_form_on_rect(np.float64(c0), c1, c2, x0, x1, y0, y1))
        assert got <= dense + 1e-12 and dense - got <= 1e-3 * max(1.0, dense)


@pytest.mark.parametrize("T", [8, 16, 32])
def test_fp64_culled_lists_pass_and_box_lists_fail(oracle_lib, T):
    sp, (V, W, H, T), (ranges, lst), (gr, gl) = _case(T=T, seed=10 + T)
    st = tc.check_tile_lists(sp, V, W, H, T, gr, gl, ranges, lst)
    assert st["dropped"] > 0.05 * st["box_pairs"] and st["kept_checked"] > 0.5 * st["kept"], st
    assert st["whole_row_pairs"] > 0, st
    # the box lists keep pairs far out of reach: rule 3
    with pytest.raises(AssertionError, match="rule 3"):
        tc.check_tile_lists(sp, V, W, H, T, ranges, lst, ranges, lst)


def test_dropping_a_reaching_pair_fails(oracle_lib):
    sp, (V, W, H, T), (ranges, lst), (gr, gl) = _case()
    lists = _lists(gr, gl)
    q = oracle.splat_q(sp)
    tiles = np.repeat(np.arange(len(gr)), gr[:, 1] - gr[:, 0])
    # a kept pair with a pixel centre of alpha >= 1/255 (unwidened reach below q) of a culled splat
    reach = tc.pair_reach(sp, gl, tiles, W, H, T, 0.0)
    _, culls = tc.splat_classes(sp, W, T)
    k = int(np.nonzero((reach < 0.5 * q[gl]) & culls[gl])[0][0])
    lists[tiles[k]].remove(gl[k])
    with pytest.raises(AssertionError, match="rule 2"):
        tc.check_tile_lists(sp, V, W, H, T, *_as_ranges(lists), ranges, lst)


def test_swapped_order_fails(oracle_lib):
    sp, (V, W, H, T), (ranges, lst), (gr, gl) = _case()
    lists = _lists(gr, gl)
    t = next(i for i, L in enumerate(lists) if len(L) >= 3)
    lists[t][0], lists[t][1] = lists[t][1], lists[t][0]
    with pytest.raises(AssertionError, match="order"):
        tc.check_tile_lists(sp, V, W, H, T, *_as_ranges(lists), ranges, lst)


def test_duplicated_entry_fails(oracle_lib):
    sp, (V, W, H, T), (ranges, lst), (gr, gl) = _case()
    lists = _lists(gr, gl)
    t = next(i for i, L in enumerate(lists) if len(L) >= 2)
    lists[t].insert(1, lists[t][0])
    with pytest.raises(AssertionError, match="rule 1"):
        tc.check_tile_lists(sp, V, W, H, T, *_as_ranges(lists), ranges, lst)


def test_pair_outside_the_box_fails(oracle_lib):
    sp, (V, W, H, T), (ranges, lst), (gr, gl) = _case()
    lists = _lists(gr, gl)
    box = _lists(ranges, lst)
    t = next(i for i, L in enumerate(lists) if len(L) >= 1)
    n = len(sp["px"]) // V
    stranger = next(i for i in range((t // ((W // T) * (H // T))) * n, len(sp["px"])) if i not in box[t])
    lists[t].append(stranger)
    with pytest.raises(AssertionError, match="rule 1"):
        tc.check_tile_lists(sp, V, W, H, T, *_as_ranges(lists), ranges, lst)


def _single(px, py, c0, c1, c2, q, rx, ry):
    o = np.exp(q / 2) / 255.0
    return dict(px=np.array([px]), py=np.array([py]), c0=np.array([c0]), c1=np.array([c1]), c2=np.array([c2]),
                q=np.array([q]), opacity=np.array([o]), r=np.ones(1), g=np.ones(1), b=np.ones(1),
                depth=np.ones(1), rx=np.array([rx], np.int32), ry=np.array([ry], np.int32))


def test_hand_computed_row_culling_and_margin(oracle_lib):
    """A circle of radius sqrt(q / c0) = 12 px (q = 9, c0 = c2 = 1/16) at (108.4, 50) on 16 px tiles, with a box of
    half-extent 60. Grown by the stated widening (q = 9.01: radius 12.007) and one pixel, its widest chord in tile
    row 3 (pixel centres 48.5 .. 63.5) spans 95.39 .. 121.41: columns 5 (last centre 95.5) to 7. In tile row 2
    (centres 32.5 .. 47.5) the widest chord is at y = 47.5, 108.4 -+ sqrt(144.16 - 2.5^2) = 108.4 -+ 11.74; less
    one pixel its left end is 95.66 > 95.5, so the row keeps columns 6-7. Every other row of the box is out of
    reach."""
    W, H, T = 256, 128, 16
    sp = _single(108.4, 50.0, 1 / 16, 0.0, 1 / 16, 9.0, 60, 60)
    ranges, lst = oracle.bin_sort(sp, 1, W, H, T)
    TX = W // T
    expect = [[] for _ in range(len(ranges))]
    for ty, cols in [(2, (6, 7)), (3, (5, 6, 7))]:
        for c in cols:
            expect[ty * TX + c] = [0]
    st = tc.check_tile_lists(sp, 1, W, H, T, *_as_ranges(expect), ranges, lst)
    assert st["kept"] == 5 and st["dropped"] == st["box_pairs"] - 5
    gr, gl = _fp64_culled(sp, 1, W, H, T, ranges, lst)
    assert np.array_equal(gr, _as_ranges(expect)[0])
    # column 5 of row 3 is kept by the widening alone (its last pixel centre, 95.5, is 12.9 px from the centre):
    # leaving it out is allowed; keeping column 5 of row 2 as well is allowed (within the widening plus rounding);
    # leaving out column 6 of row 3, which the circle covers, is not
    expect[3 * TX + 5] = []
    tc.check_tile_lists(sp, 1, W, H, T, *_as_ranges(expect), ranges, lst)
    expect[2 * TX + 5] = [0]
    tc.check_tile_lists(sp, 1, W, H, T, *_as_ranges(expect), ranges, lst)
    expect[3 * TX + 6] = []
    with pytest.raises(AssertionError, match="rule 2"):
        tc.check_tile_lists(sp, 1, W, H, T, *_as_ranges(expect), ranges, lst)


def test_margin_is_enforced(oracle_lib):
    """The circle's edge 12.0013 px from column 5's last pixel centre: no pixel of column 5 reaches alpha >= 1/255
    (form 9.0019 > q = 9), but the rectangle grown by 1/2 px reaches it, so leaving the pair out breaks the stated
    margin (rule 2)."""
    W, H, T = 256, 128, 16
    sp = _single(95.5 + 12.0013, 56.0, 1 / 16, 0.0, 1 / 16, 9.0, 14, 14)
    ranges, lst = oracle.bin_sort(sp, 1, W, H, T)
    TX = W // T
    lists = _lists(ranges, lst)
    assert lists[3 * TX + 5] == [0]
    reach = tc.pair_reach(sp, np.array([0]), np.array([3 * TX + 5]), W, H, T, 0.0)[0]
    assert 9.0 < reach < 9.0 * 1.0005
    lists[3 * TX + 5] = []
    with pytest.raises(AssertionError, match="rule 2"):
        tc.check_tile_lists(sp, 1, W, H, T, *_as_ranges(lists), ranges, lst)


def test_whole_row_splats_may_not_drop(oracle_lib):
    """A needle conic (det = 1e-5 c0 c2) and a box wider than the image keep every tile of their boxes, even those
    out of reach (rule 4)."""
    W, H, T = 256, 128, 16
    TX = W // T
    c0, c2 = 1 / 16, 1 / 16
    needle = _single(100.0, 60.0, c0, np.sqrt(c0 * c2 * (1 - 1e-5)), c2, 9.0, 40, 40)
    ranges, lst = oracle.bin_sort(needle, 1, W, H, T)
    tc.check_tile_lists(needle, 1, W, H, T, ranges, lst, ranges, lst)
    lists = _lists(ranges, lst)
    t = next(i for i, L in enumerate(lists) if L)
    lists[t] = []
    with pytest.raises(AssertionError, match="rule 4"):
        tc.check_tile_lists(needle, 1, W, H, T, *_as_ranges(lists), ranges, lst)
    wide = _single(100.0, 60.0, 1 / 16, 0.0, 1 / 16, 9.0, 200, 20)
    ranges, lst = oracle.bin_sort(wide, 1, W, H, T)
    lists = _lists(ranges, lst)
    assert sum(len(L) for L in lists) == TX * 4  # pixel rows 40 .. 80: tile rows 2 .. 5
    tc.check_tile_lists(wide, 1, W, H, T, ranges, lst, ranges, lst)
    lists[3 * TX + 0] = []
    with pytest.raises(AssertionError, match="rule 4"):
        tc.check_tile_lists(wide, 1, W, H, T, *_as_ranges(lists), ranges, lst)


def test_half_width_boxes_keep_whole_rows(oracle_lib):
    """Equirectangular: a box of half-width rx = 114 on a 256 px image (16 px tiles) spans 15 of the 16 tile columns
    (x = 6 .. 234), yet rx + T > W / 2, so its column offsets can differ from the blend's minimal-image dx: its rows
    are kept whole (rule 4). The uncut box lists pass; leaving out a far column does not."""
    W, H, T = 256, 128, 16
    TX = W // T
    sp = _single(120.3, 60.0, 1 / 16, 0.0, 1 / 16, 9.0, 114, 20)
    ranges, lst = oracle.bin_sort(sp, 1, W, H, T)
    lists = _lists(ranges, lst)
    assert sum(len(L) for L in lists) == 15 * 4  # columns 0 .. 14; pixel rows 40 .. 80: tile rows 2 .. 5
    tc.check_tile_lists(sp, 1, W, H, T, ranges, lst, ranges, lst)
    lists[3 * TX + 0] = []
    with pytest.raises(AssertionError, match="rule 4"):
        tc.check_tile_lists(sp, 1, W, H, T, *_as_ranges(lists), ranges, lst)


def test_a_flat_ellipse_short_of_the_needle_threshold_is_culled(oracle_lib):
    """det = 5e-3 c0 c2 is a flat ellipse but no needle (the threshold is 1e-3): its rows are culled like any other,
    so its FP64-culled lists pass and drop pairs of its box."""
    W, H, T = 256, 128, 16
    c0, c2 = 1 / 16, 1 / 64
    c1 = np.sqrt(c0 * c2 * (1 - 5e-3))
    sp = _single(128.3, 64.0, c0, c1, c2, 9.0, 80, 40)
    ranges, lst = oracle.bin_sort(sp, 1, W, H, T)
    gr, gl = _fp64_culled(sp, 1, W, H, T, ranges, lst)
    st = tc.check_tile_lists(sp, 1, W, H, T, gr, gl, ranges, lst)
    assert st["dropped"] > 0 and st["whole_row_pairs"] == 0, st


@pytest.mark.parametrize("side", [-1, 1])
def test_half_pixel_widening_on_either_side(oracle_lib, side):
    """A circle (radius 12, q = 9) whose edge stops 0.3 px short of a tile's outer pixel centres, on its left
    (side -1: the circle lies left of column 6, whose first centre is x = 96.5) or on its right (side 1: right of
    column 5, last centre 95.5). No pixel centre of that tile reaches alpha >= 1/255 (form 9.46 > q (1 + 5e-4) +
    5e-4), but the tile's rectangle grown by 1/2 px does: leaving the pair out breaks rule 2."""
    W, H, T = 256, 128, 16
    TX = W // T
    col, centre = (6, 96.5 - 12.3) if side < 0 else (5, 95.5 + 12.3)
    sp = _single(centre, 56.0, 1 / 16, 0.0, 1 / 16, 9.0, 14, 14)
    ranges, lst = oracle.bin_sort(sp, 1, W, H, T)
    lists = _lists(ranges, lst)
    assert lists[3 * TX + col] == [0]
    reach = tc.pair_reach(sp, np.array([0]), np.array([3 * TX + col]), W, H, T, 0.0)[0]
    assert reach > 9.0 * (1 + 5e-4) + 5e-4
    lists[3 * TX + col] = []
    with pytest.raises(AssertionError, match="rule 2"):
        tc.check_tile_lists(sp, 1, W, H, T, *_as_ranges(lists), ranges, lst)


def test_seam_copy_counts_for_the_equirectangular_camera_only(oracle_lib):
    """A circle centred 2 px right of the seam reaches the last tile column through its copy at -W: leaving that tile
    out breaks rule 2 on the equirectangular camera; with a pinhole camera (no wrap) the box is clipped at column 0
    and the last column is no tile of it."""
    W, H, T = 256, 128, 16
    TX = W // T
    sp = _single(2.0, 60.0, 1 / 16, 0.0, 1 / 16, 9.0, 13, 13)
    ranges, lst = oracle.bin_sort(sp, 1, W, H, T)
    lists = _lists(ranges, lst)
    assert lists[3 * TX + TX - 1] == [0]
    lists[3 * TX + TX - 1] = []
    with pytest.raises(AssertionError, match="rule 2"):
        tc.check_tile_lists(sp, 1, W, H, T, *_as_ranges(lists), ranges, lst)
    cam = oracle.pinhole(200.0, 200.0, W / 2, H / 2)
    ranges_p, lst_p = oracle.bin_sort(sp, 1, W, H, T, camera=cam)
    assert not _lists(ranges_p, lst_p)[3 * TX + TX - 1]
    gr, gl = _fp64_culled(sp, 1, W, H, T, ranges_p, lst_p, camera=cam)
    tc.check_tile_lists(sp, 1, W, H, T, gr, gl, ranges_p, lst_p, camera=cam)


def test_minimal_image_across_the_seam(oracle_lib):
    """A splat of the egocentric workload (2048 x 1024, 16 px tiles) whose box, 1006 px either side of x = 1702.9,
    nearly wraps: in tile row 3 its sheared ellipse reaches x = 2744, the far copy of tile column 43, but the blend
    evaluates column 43's pixels at their minimal image dx = +999 .. +1014, out of reach, so leaving tile 43 out is
    valid; column 41 (pixels 656 .. 671, minimal image dx = -1017 .. -1002) is reached and may not be left out."""
    W, H, T = 2048, 1024, 16
    TX = W // T
    sp = _single(1702.8888, 20.02848, 2.3068576e-05, -3.3590427e-04, 0.0079759015, 10.253982, 1006, 58)
    ranges, lst = oracle.bin_sort(sp, 1, W, H, T)
    assert _lists(ranges, lst)[3 * TX + 43] == [0] and _lists(ranges, lst)[3 * TX + 41] == [0]
    reach = tc.pair_reach(sp, np.array([0, 0]), np.array([3 * TX + 43, 3 * TX + 41]), W, H, T, 0.0)
    assert reach[0] > 4 * 10.253982 and reach[1] < 10.253982
    lists = _lists(*_fp64_culled(sp, 1, W, H, T, ranges, lst))
    assert lists[3 * TX + 43] == [] and lists[3 * TX + 41] == [0]
    tc.check_tile_lists(sp, 1, W, H, T, *_as_ranges(lists), ranges, lst)
    lists[3 * TX + 41] = []
    with pytest.raises(AssertionError, match="rule 2"):
        tc.check_tile_lists(sp, 1, W, H, T, *_as_ranges(lists), ranges, lst)
