"""Validity of tile lists that leave out (Gaussian, tile) pairs, checked against the oracle's box lists (FP64, CPU).

Test infrastructure. The oracle lists one instance for every tile of a Gaussian's instance box (Sec. 3.3, "one
instance per influence"; the box is that of the alpha >= 1/255 region). A pair may be left out when no pixel centre
of the tile can receive alpha >= 1/255 from the Gaussian (Eq. 8): every pixel of the tile skips it, so no image
changes. The CUDA binning leaves pairs out row by row, with a stated widening: the ellipse dp^T conic dp <= q
(q = 2 ln(255 o), the alpha = 1/255 level) is grown to q (1.001) + 1e-3, and by one pixel on each side in x. Rows of
a box that spans every tile column, of a box with rx + T > W / 2 (equirectangular: beyond that the box's column
offsets can differ from the blend's minimal-image dx), and Gaussians whose conic is a needle (det <= 1e-3 c0 c2,
where the row bounds lose precision), keep the whole row.

A list is valid when, tile by tile:
  1. it is an order-preserving subsequence of the oracle's list: no pair from outside the instance box, and the
     (t_r, index) order kept;
  2. every pair it leaves out is out of reach by at least half the stated widening: over the tile's rectangle of
     pixel centres widened by 1/2 px on each side in x, min dp^T conic dp > q (1 + 5e-4) + 5e-4, with dx the minimal
     image across the longitude seam that the blend uses. In particular no pixel centre of the tile gets
     alpha >= 1/255 from it;
  3. every pair it keeps comes within the stated widening, up to single-precision rounding: over the rectangle
     widened by 3/2 px in x, min dp^T conic dp <= q (1.002) + 2e-3;
  4. a Gaussian whose box spans every tile column, or (equirectangular) whose box half-width rx + T exceeds W / 2,
     or whose conic is a needle, leaves out no pair, and 3 does not apply to it. Within 0.1 % of the needle
     threshold either decision is accepted (the implementation takes it in single precision).
"""
from __future__ import annotations

import numpy as np

DROP_Q_SCALE, DROP_Q_ADD, DROP_DX = 1.0 + 5e-4, 5e-4, 0.5
KEEP_Q_SCALE, KEEP_Q_ADD, KEEP_DX = 1.002, 2e-3, 1.5
NEEDLE = 1e-3


def min_form_on_rect(c0, c1, c2, x0, x1, y0, y1):
    """min of c0 u^2 + 2 c1 u v + c2 v^2 over [x0, x1] x [y0, y1], elementwise, for positive definite forms: 0 when
    the rectangle holds the origin, else the least of the four edge minima (a convex quadratic on a segment)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        best = np.full(np.broadcast(c0, x0).shape, np.inf)
        su, sv = -c1 / c0, -c1 / c2
        for v in (y0, y1):
            u = np.clip(su * v, x0, x1)
            best = np.minimum(best, (c0 * u + 2 * c1 * v) * u + c2 * v * v)
        for u in (x0, x1):
            v = np.clip(sv * u, y0, y1)
            best = np.minimum(best, c0 * u * u + (2 * c1 * u + c2 * v) * v)
    inside = (x0 <= 0) & (x1 >= 0) & (y0 <= 0) & (y1 >= 0)
    return np.where(inside, 0.0, best)


def _gather(ranges, lst, tiles):
    """Entries of the given tiles: (tile of each entry, position within its tile, splat)."""
    a, b = ranges[tiles, 0].astype(np.int64), ranges[tiles, 1].astype(np.int64)
    lens = b - a
    off = np.cumsum(lens) - lens
    total = int(lens.sum())
    within = np.arange(total, dtype=np.int64) - np.repeat(off, lens)
    pos = np.repeat(a, lens) + within
    return np.repeat(tiles, lens), within, np.asarray(lst, np.int64)[pos]


def splat_classes(sp, W, T, camera=None):
    """Per splat: (whole_rows, culls) booleans. whole_rows: the box spans every tile column, or (equirectangular)
    rx + T > W / 2, or the conic is a needle (with a 0.1 % band that is neither); culls: the rows may be culled
    (clearly not a needle, box narrower than that)."""
    TX = W // T
    px = np.asarray(sp["px"], np.float64)
    rx = np.asarray(sp["rx"], np.int64)
    ix = np.floor(px).astype(np.int64)
    x0, x1 = np.floor_divide(ix - rx, T), np.floor_divide(ix + rx, T)
    if camera is not None:
        x0, x1 = np.maximum(x0, 0), np.minimum(x1, TX - 1)
        wide = x1 - x0 + 1 >= TX
    else:
        wide = (x1 - x0 + 1 >= TX) | (2 * (rx + T) > W)
    c0, c1, c2 = (np.asarray(sp[k], np.float64) for k in ("c0", "c1", "c2"))
    det = c0 * c2 - c1 * c1
    pos = (c0 > 0) & (c2 > 0)
    needle = ~pos | (det <= NEEDLE * (1 - 1e-3) * c0 * c2)
    clear = pos & (det > NEEDLE * (1 + 1e-3) * c0 * c2)
    return wide | needle, ~wide & clear


def pair_reach(sp, splat, tile, W, H, T, dx_widen, camera=None):
    """min dp^T conic dp over the pixel-centre rectangle of each (splat, tile) pair, widened by dx_widen px on each
    side in x. Equirectangular: each x offset u = x - p_x is taken as the minimal image the blend uses (u in
    (-W/2, W/2], dx = -u in [-W/2, W/2)); a rectangle that straddles u = W/2 is split there into its two images."""
    TX, TY = W // T, H // T
    tt = tile % (TX * TY)
    ty, tx = tt // TX, tt % TX
    px = np.asarray(sp["px"], np.float64)[splat]
    py = np.asarray(sp["py"], np.float64)[splat]
    c0, c1, c2 = (np.asarray(sp[k], np.float64)[splat] for k in ("c0", "c1", "c2"))
    xa = tx * T + 0.5 - dx_widen - px
    xb = tx * T + T - 0.5 + dx_widen - px
    ya = ty * T + 0.5 - py
    yb = ty * T + T - 0.5 - py
    if camera is not None:
        return min_form_on_rect(c0, c1, c2, xa, xb, ya, yb)
    half = 0.5 * W
    ka = np.ceil((xa - half) / W)  # xa - ka W lies in (-W/2, W/2]
    kb = np.ceil((xb - half) / W)
    m = min_form_on_rect(c0, c1, c2, xa - ka * W, np.where(ka == kb, xb - ka * W, half), ya, yb)
    k = np.nonzero(kb > ka)[0]
    if len(k):
        m[k] = np.minimum(m[k], min_form_on_rect(c0[k], c1[k], c2[k], -half, xb[k] - kb[k] * W, ya[k], yb[k]))
    return m


def check_tile_lists(sp, V, W, H, T, got_ranges, got_list, ref_ranges, ref_list, tiles=None, camera=None,
                     q=None) -> dict:
    """Assert rules 1-4 of the module docstring on the given tiles (default: all). sp: splat fields (px, py, c0, c1,
    c2, rx, and q or opacity); lists hold splat indices v * n + g. Returns counts of the pairs checked."""
    import oracle
    TX, TY = W // T, H // T
    nt = V * TX * TY
    tiles = np.arange(nt, dtype=np.int64) if tiles is None else np.asarray(tiles, np.int64)
    q = oracle.splat_q(sp) if q is None else np.asarray(q, np.float64)
    M = len(q)
    got_ranges = np.asarray(got_ranges, np.int64).reshape(-1, 2)
    ref_ranges = np.asarray(ref_ranges, np.int64).reshape(-1, 2)
    gt, gpos, gs = _gather(got_ranges, got_list, tiles)
    rt, rpos, rs = _gather(ref_ranges, ref_list, tiles)
    gkey, rkey = gt * M + gs, rt * M + rs

    # 1. subsequence of the oracle's list, order kept
    order = np.argsort(rkey, kind="stable")
    sk = rkey[order]
    at = np.searchsorted(sk, gkey)
    found = (at < len(sk)) & (sk[np.minimum(at, len(sk) - 1)] == gkey)
    if not found.all():
        k = int(np.nonzero(~found)[0][0])
        raise AssertionError(f"rule 1: tile {gt[k]} lists splat {gs[k]}, which its instance box does not reach")
    refpos = rpos[order[at]]
    same = gt[1:] == gt[:-1]
    bad = same & (np.diff(refpos) <= 0)
    if bad.any():
        k = int(np.nonzero(bad)[0][0])
        raise AssertionError(f"rule 1: tile {gt[k]} lists splats {gs[k]}, {gs[k + 1]} out of (t_r, index) order "
                             f"(or twice)")

    whole, culls = splat_classes(sp, W, T, camera)
    # 2. and 4. every left-out pair is out of reach; whole-row splats leave none out
    dropped = np.ones(len(rkey), bool)
    dropped[order[at]] = False
    ds, dt = rs[dropped], rt[dropped]
    w = whole[ds]
    if w.any():
        k = int(np.nonzero(w)[0][0])
        raise AssertionError(f"rule 4: splat {ds[k]} keeps whole rows but tile {dt[k]} is left out")
    m = pair_reach(sp, ds, dt, W, H, T, DROP_DX, camera)
    lim = q[ds] * DROP_Q_SCALE + DROP_Q_ADD
    bad = ~(m > lim)
    if bad.any():
        k = int(np.nonzero(bad)[0][0])
        raise AssertionError(f"rule 2: splat {ds[k]} left out of tile {dt[k]} comes within reach "
                             f"(min form {m[k]:.6g} <= {lim[k]:.6g})")
    # 3. every kept pair of a culled splat is within the widening
    kc = culls[gs]
    ks, kt = gs[kc], gt[kc]
    m = pair_reach(sp, ks, kt, W, H, T, KEEP_DX, camera)
    lim = q[ks] * KEEP_Q_SCALE + KEEP_Q_ADD
    bad = ~(m <= lim)
    if bad.any():
        k = int(np.nonzero(bad)[0][0])
        raise AssertionError(f"rule 3: splat {ks[k]} kept in tile {kt[k]} stays out of reach "
                             f"(min form {m[k]:.6g} > {lim[k]:.6g})")
    return dict(box_pairs=int(len(rs)), kept=int(len(gs)), dropped=int(dropped.sum()), kept_checked=int(kc.sum()),
                whole_row_pairs=int(whole[gs].sum()))
