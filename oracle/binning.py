"""Discrete stages on float32 records: macro-tile binning, segment order and
batch split, in plain integer arithmetic.

Records per gaussian (what the projection hands to partitioning):
    mx, my     float32 screen position (pixel centre convention)
    radius     int, 0 for a culled gaussian
    key        uint32 depth key (float32 depth bits, Sec. 4.3)

Binning test (Sec. 3.2 / 4.3, "conservative" gaussian-to-macro-tile test).
Reading: the baseline test is the 3-sigma rectangle in integers,
    x0 = floor(mx), tile-x range = [floor((x0 - r) / Bx), floor((x0 + r) / Bx)]
clamped to the grid (same for y), Bx the tile or macro-tile width in pixels.
It contains every pixel of the q <= 9 support (a supported pixel x satisfies
x0 - r <= x <= x0 + r).

Ellipse test (Sec. 3.2 per-row ellipse scan at macro granularity with an
opacity-aware threshold, Sec. 4.3).  The paper gives no formula; reading: a
gaussian is paired with a macro-tile of its rectangle when the ellipse
    (L0 dx + L1 dy)^2 + (L2 dy)^2 <= E_bin
(L the Cholesky factors of the conic prescaled by sqrt(log2(e) / 2), so the
left side is q log2(e) / 2) meets the pixel centres of the tile, evaluated
per macro row band in float32 with a fixed operation order and fixed margins
so that it is reproducible bit for bit:
    E_bin  = min(9 log2(e) / 2, lb(255 o)) + 2^-12, where lb is an upper bound
             of log2 from frexp (z = m 2^k, m in [0.5, 1)):
             lb(z) = k + (B m + A), A = -475/256, B = 123/64, a line above
             log2(m) on [0.5, 1] (log2 m <= B m + A - 0.00098; gap <= 0.105)
    band   rows [ya, yb] of the macro row; it meets the ellipse when
           [ya - my, yb - my] meets +-(hy (1 + 2^-10) + 2^-6), hy = sqrt(E) / L2
    x span the extremes of (-L1 dy -+ sqrt(E - (L2 dy)^2)) / L0 over the
           band's part of [-hy, hy]: at the ellipse's leftmost / rightmost
           point when the band holds it, else at the band end nearer to it
           (the edges are convex / concave), widened by 2^-6 + 2^-10 |offset|
           pixels, clamped to +-2^30 (see ellipse_span for the op order)
    cols   [floor(ceil(xl) / Bx), floor(floor(xr) / Bx)] within the rectangle
It is conservative for the blend test (q <= 9 and alpha >= 1/255, i.e.
q log2(e) / 2 <= min(9 log2(e) / 2, log2(255 o))): the margins cover float32
rounding.  Gaussians with degenerate factors, and rectangles of one macro
cell or of more than 64 cells (the test is stored as a 64-bit cell mask),
keep their whole rectangle.

Segments (Sec. 3.3): one per (view, macro-tile); the segment id is
view * N_M + my * gx + mx.  Order inside a segment: ascending (key, id)
(reading: the paper sorts by the 32-bit depth key only and is silent on ties;
ties are broken by gaussian id).

Batches (Sec. 3.1): a segment of n pairs splits into ceil(n / B_r) batches of
consecutive sorted positions [j B_r, min((j+1) B_r, n)).
"""
from __future__ import annotations

import numpy as np


def grid_dims(width: int, height: int, bw: int, bh: int):
    return -(-width // bw), -(-height // bh)


def rect_ranges(mx32, my32, radius, width, height, bw, bh):
    """Inclusive clamped tile ranges (tx0, tx1, ty0, ty1) per gaussian and
    the number of cells; cells = 0 when the range is empty or radius = 0."""
    gw, gh = grid_dims(width, height, bw, bh)
    x0 = np.floor(np.asarray(mx32, np.float32).astype(np.float64)).astype(np.int64)
    y0 = np.floor(np.asarray(my32, np.float32).astype(np.float64)).astype(np.int64)
    r = np.asarray(radius, np.int64)
    tx0 = np.maximum(np.floor_divide(x0 - r, bw), 0)
    tx1 = np.minimum(np.floor_divide(x0 + r, bw), gw - 1)
    ty0 = np.maximum(np.floor_divide(y0 - r, bh), 0)
    ty1 = np.minimum(np.floor_divide(y0 + r, bh), gh - 1)
    nx = np.maximum(tx1 - tx0 + 1, 0)
    ny = np.maximum(ty1 - ty0 + 1, 0)
    cells = np.where(r > 0, nx * ny, 0)
    return tx0, tx1, ty0, ty1, cells, gw, gh


F32 = np.float32
ELL_A = F32(-475.0 / 256.0)
ELL_B = F32(123.0 / 64.0)
ELL_MARGIN_E = F32(2.0 ** -12)
ELL_PAD = F32(2.0 ** -6)
ELL_REL = F32(2.0 ** -10)
SUPPORT_E = F32(4.5 * np.log2(np.e))        # q = 9 in units of q log2(e) / 2
PRESCALE = F32(np.sqrt(np.log2(np.e) / 2.0))


def log2_upper(z32):
    """lb(z) >= log2(z) for float32 z > 0 (see the module docstring)."""
    z = np.asarray(z32, F32)
    m, k = np.frexp(z)
    return k.astype(F32) + (ELL_B * m.astype(F32) + ELL_A)


def ellipse_level(o32):
    """E_bin of the ellipse test for float32 opacities."""
    z = F32(255.0) * np.asarray(o32, F32)
    return np.minimum(SUPPORT_E, log2_upper(z)) + ELL_MARGIN_E


def cholesky_from_conic(conic32):
    """Prescaled Cholesky factors (L0, L1, L2) of float32 conics (A, B, C),
    q = A dx^2 + 2 B dx dy + C dy^2 = (l0 dx + l1 dy)^2 + (l2 dy)^2:
    l0 = sqrt(A), l1 = B / l0, l2 = sqrt(C - l1^2), each op rounded to float32."""
    c = np.asarray(conic32, F32)
    l0 = np.sqrt(np.maximum(c[:, 0], F32(0)))
    safe = np.where(l0 > 0, l0, F32(1))
    l1 = np.where(l0 > 0, c[:, 1] / safe, F32(0)).astype(F32)
    l2 = np.sqrt(np.maximum(c[:, 2] - l1 * l1, F32(0)))
    return l0 * PRESCALE, l1 * PRESCALE, l2 * PRESCALE


def ellipse_span(mx, my, L0, L1, L2, E, ya, yb):
    """x span [xl, xr] (pixel-centre coordinates, widened) of the ellipse
    over the rows [ya, yb] (float32 arrays, one entry per (gaussian, band)).
    Returns (xl, xr, meet, ok): meet = False when the band misses the
    ellipse, ok = False for degenerate factors.

    Per gaussian: sE = sqrt(E), hy = sE / L2 (the ellipse's y half-extent),
    the leftmost point at dy_l = L1 sE / (L2 sqrt(L1^2 + L2^2)) (the rightmost
    at -dy_l) and its offset x_l = (-L1 dy_l - h(dy_l)) / L0, x_r = -x_l,
    h(dy) = sqrt(max(0, E - (L2 dy)^2)).  Per band: the band meets the
    ellipse when it meets [-hy', hy'] (hy' = hy (1 + 2^-10) + 2^-6); the
    left edge (-L1 dy - h(dy)) / L0 is convex in dy, so over the band's part
    [a, b] of [-hy, hy] its minimum is at dy_l when dy_l is in [a, b], else at
    the end nearer to dy_l (likewise the right edge, concave, with -dy_l).  A
    band that meets only the widened range is evaluated at the tip (a = b =
    -+hy).  Divisions by L0 and L2 are products with their reciprocals."""
    mx, my, L0, L1, L2, E = (np.asarray(v, F32) for v in (mx, my, L0, L1, L2, E))
    ya, yb = np.asarray(ya, F32), np.asarray(yb, F32)
    ok = (L0 > 0) & (L2 > 0)
    L0s = np.where(ok, L0, F32(1))
    L2s = np.where(ok, L2, F32(1))
    live = E > 0
    Ep = np.maximum(E, F32(0))
    sE = np.sqrt(Ep)
    iL0 = F32(1) / L0s
    iL2 = F32(1) / L2s
    hy = sE * iL2
    hyw = hy * F32(1.0 + 2.0 ** -10) + ELL_PAD
    ra, rb = ya - my, yb - my
    meet = live & (np.maximum(ra, -hyw) <= np.minimum(rb, hyw))

    def half(dy):
        t = L2s * dy
        return np.sqrt(np.maximum(F32(0), Ep - t * t))

    nrm = np.sqrt(L1 * L1 + L2s * L2s)
    dyl = (L1 * sE) / (L2s * nrm)
    x_l = (-L1 * dyl - half(dyl)) * iL0
    x_r = (L1 * dyl + half(dyl)) * iL0
    a = np.maximum(ra, -hy)
    b = np.minimum(rb, hy)
    tip = np.where(rb < -hy, -hy, hy)
    inside = a <= b
    a = np.where(inside, a, tip)
    b = np.where(inside, b, tip)
    dlo = np.where(dyl < a, a, b)
    lo = np.where((dyl >= a) & (dyl <= b), x_l, (-L1 * dlo - half(dlo)) * iL0)
    dhi = np.where(-dyl < a, a, b)
    hi = np.where((-dyl >= a) & (-dyl <= b), x_r, (-L1 * dhi + half(dhi)) * iL0)
    xl = (mx + lo) - (np.abs(lo) * ELL_REL + ELL_PAD)
    xr = (mx + hi) + (np.abs(hi) * ELL_REL + ELL_PAD)
    # far outside any image; keeps the integer conversion in range
    lim = F32(2.0 ** 30)
    xl = np.minimum(np.maximum(xl, -lim), lim)
    xr = np.minimum(np.maximum(xr, -lim), lim)
    return xl, xr, meet, ok


def ellipse_cols(mx, my, L0, L1, L2, E, ya, yb, bw):
    """Macro columns [c0, c1] where the ellipse meets the row band [ya, yb];
    c0 > c1 when it misses.  Returns (c0, c1, ok)."""
    xl, xr, meet, ok = ellipse_span(mx, my, L0, L1, L2, E, ya, yb)
    with np.errstate(invalid="ignore"):
        c0 = np.floor_divide(np.ceil(np.where(meet, xl, 0)).astype(np.int64), bw)
        c1 = np.floor_divide(np.floor(np.where(meet, xr, 0)).astype(np.int64), bw)
    c1 = np.where(meet, c1, c0 - 1)
    return c0, c1, ok


def _cells_from_rows(g, row, c0, c1, gw):
    """Expand (gaussian, macro row, [c0, c1]) into (gaussian, segment)."""
    n = np.maximum(c1 - c0 + 1, 0)
    ids = np.repeat(g, n)
    k = np.arange(int(n.sum()), dtype=np.int64) - np.repeat(np.cumsum(n) - n, n)
    seg = np.repeat(row, n) * gw + np.repeat(c0, n) + k
    return ids, seg


def bin_pairs(mx32, my32, radius, key, width, height, bw, bh, seg_base: int = 0, ellipse=None):
    """Unordered (segment, key, id) pairs of one view.  ellipse = (L0, L1,
    L2, o) float32 arrays selects the ellipse test, else the rectangle."""
    tx0, tx1, ty0, ty1, cells, gw, gh = rect_ranges(mx32, my32, radius, width, height, bw, bh)
    if ellipse is None:
        ids = np.repeat(np.arange(len(cells), dtype=np.int64), cells)
        k = np.arange(int(cells.sum()), dtype=np.int64) - np.repeat(np.cumsum(cells) - cells, cells)
        nx = np.repeat(tx1 - tx0 + 1, cells)
        seg = (np.repeat(ty0, cells) + k // np.maximum(nx, 1)) * gw + np.repeat(tx0, cells) + k % np.maximum(nx, 1)
        return seg + seg_base, np.asarray(key, np.uint32)[ids], ids, gw * gh
    L0, L1, L2, o = (np.asarray(v, F32) for v in ellipse)
    refine = (cells > 1) & (cells <= 64)
    ny = np.where(cells > 0, ty1 - ty0 + 1, 0)
    g = np.repeat(np.arange(len(cells), dtype=np.int64), ny)
    row = np.repeat(ty0, ny) + (np.arange(int(ny.sum()), dtype=np.int64) - np.repeat(np.cumsum(ny) - ny, ny))
    ya = (row * bh).astype(F32)
    yb = (row * bh + bh - 1).astype(F32)
    E = ellipse_level(o)[g]
    c0, c1, ok = ellipse_cols(np.asarray(mx32, F32)[g], np.asarray(my32, F32)[g], L0[g], L1[g], L2[g], E, ya, yb,
                              bw)
    use = ok & refine[g]
    c0 = np.where(use, np.maximum(c0, tx0[g]), tx0[g])
    c1 = np.where(use, np.minimum(c1, tx1[g]), tx1[g])
    ids, seg = _cells_from_rows(g, row, c0, c1, gw)
    return seg + seg_base, np.asarray(key, np.uint32)[ids], ids, gw * gh


def segments(views, width_height, bw, bh):
    """Segmented, sorted pair list over several views.

    views: list of (mx32, my32, radius, key) tuples, or (mx32, my32,
    radius, key, (L0, L1, L2, o)) for the ellipse test (one per view, all
    with the same gaussian count); width_height: list of (W, H) per view.
    Returns dict with seg_off [S+1] (int64), keys [P] uint32, ids [P] int64,
    n_macro per view and the segment base per view.
    """
    segs, keys, ids, bases, nms = [], [], [], [], []
    base = 0
    for vw, (w, h) in zip(views, width_height):
        mx, my, r, key = vw[:4]
        s, k, i, nm = bin_pairs(mx, my, r, key, w, h, bw, bh, base, ellipse=vw[4] if len(vw) > 4 else None)
        segs.append(s), keys.append(k), ids.append(i), bases.append(base), nms.append(nm)
        base += nm
    seg = np.concatenate(segs) if segs else np.zeros(0, np.int64)
    key = np.concatenate(keys) if keys else np.zeros(0, np.uint32)
    gid = np.concatenate(ids) if ids else np.zeros(0, np.int64)
    o = np.lexsort((gid, key, seg))
    seg, key, gid = seg[o], key[o], gid[o]
    seg_off = np.searchsorted(seg, np.arange(base + 1)).astype(np.int64)
    return {"seg_off": seg_off, "keys": key, "ids": gid, "n_macro": nms,
            "seg_base": bases, "n_seg": base}


def plain_tile_pairs(views, width_height, tile: int = 8):
    """Discrete stages of the plain per-tile path (the single-tile-size
    baseline of Sec. 2 and 5): every (render tile, gaussian) pair of the
    integer 3-sigma rectangle test at tile x tile pixels, over all views;
    the global tile of view v is (tiles of views < v) + ty gw + tx.  Pairs
    are ordered by the 64-bit key (global tile << 32 | depth key), then by
    the record index v n + i (n gaussians per view).

    views: list of (mx32, my32, radius, key); width_height: (W, H) per view.
    Returns keys64 uint64 [P], ids int64 [P] (v n + i) and ranges int64
    [tiles, 2]: [start, end) of each tile's pairs, (0, 0) for an empty tile.
    """
    seg, key, rid, base = [], [], [], 0
    for v, (vw, (w, h)) in enumerate(zip(views, width_height)):
        mx, my, r, k = vw[:4]
        s, kk, i, nt = bin_pairs(mx, my, r, k, w, h, tile, tile, base)
        seg.append(s), key.append(kk), rid.append(i + v * len(r))
        base += nt
    seg = np.concatenate(seg) if seg else np.zeros(0, np.int64)
    key = np.concatenate(key) if key else np.zeros(0, np.uint32)
    rid = np.concatenate(rid) if rid else np.zeros(0, np.int64)
    o = np.lexsort((rid, key, seg))
    seg, key, rid = seg[o], key[o], rid[o]
    keys64 = (seg.astype(np.uint64) << np.uint64(32)) | key.astype(np.uint64)
    start = np.searchsorted(seg, np.arange(base), side="left")
    end = np.searchsorted(seg, np.arange(base), side="right")
    ranges = np.stack([np.where(end > start, start, 0), np.where(end > start, end, 0)], axis=1)
    return keys64, rid, ranges.astype(np.int64)


def batches(seg_off: np.ndarray, cap: int):
    """Batch table [(segment, start, count)] in segment-major order and the
    first batch index of every segment (length S+1)."""
    n = np.diff(np.asarray(seg_off, np.int64))
    nb = -(-n // cap)
    first = np.concatenate([[0], np.cumsum(nb)]).astype(np.int64)
    seg = np.repeat(np.arange(len(n), dtype=np.int64), nb)
    j = np.arange(int(nb.sum()), dtype=np.int64) - np.repeat(first[:-1], nb)
    start = seg_off[seg] + j * cap
    count = np.minimum(cap, seg_off[seg + 1] - start)
    return np.stack([seg, start, count], axis=1), first


def tile_pair_count(mx32, my32, radius, width, height, tile=8):
    """Number of (render tile, gaussian) pairs of the rect test."""
    return int(rect_ranges(mx32, my32, radius, width, height, tile, tile)[4].sum())


def per_tile_counts(mx32, my32, radius, width, height, tile=8):
    """Gaussians per render tile under the rect test, [gh, gw] (the load
    statistic of the paper's teaser figure)."""
    tx0, tx1, ty0, ty1, cells, gw, gh = rect_ranges(mx32, my32, radius, width, height, tile, tile)
    diff = np.zeros((gh + 1, gw + 1), np.int64)
    m = cells > 0
    np.add.at(diff, (ty0[m], tx0[m]), 1)
    np.add.at(diff, (ty0[m], tx1[m] + 1), -1)
    np.add.at(diff, (ty1[m] + 1, tx0[m]), -1)
    np.add.at(diff, (ty1[m] + 1, tx1[m] + 1), 1)
    return np.cumsum(np.cumsum(diff, 0), 1)[:gh, :gw]


def records_f32(proj: dict):
    """float32 records of an oracle projection (what partitioning consumes)."""
    return (proj["mean2d"][:, 0].astype(np.float32), proj["mean2d"][:, 1].astype(np.float32),
            proj["radius"].astype(np.int64), proj["depth_key"].astype(np.uint32))
