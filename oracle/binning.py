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


def bin_pairs(mx32, my32, radius, key, width, height, bw, bh, seg_base: int = 0):
    """Unordered (segment, key, id) pairs of one view."""
    tx0, tx1, ty0, ty1, cells, gw, gh = rect_ranges(mx32, my32, radius, width, height, bw, bh)
    ids = np.repeat(np.arange(len(cells), dtype=np.int64), cells)
    k = np.arange(int(cells.sum()), dtype=np.int64) - np.repeat(np.cumsum(cells) - cells, cells)
    nx = np.repeat(tx1 - tx0 + 1, cells)
    seg = (np.repeat(ty0, cells) + k // np.maximum(nx, 1)) * gw + np.repeat(tx0, cells) + k % np.maximum(nx, 1)
    return seg + seg_base, np.asarray(key, np.uint32)[ids], ids, gw * gh


def segments(views, width_height, bw, bh):
    """Segmented, sorted pair list over several views.

    views: list of (mx32, my32, radius, key) tuples (one per view, all with
    the same gaussian count); width_height: list of (W, H) per view.
    Returns dict with seg_off [S+1] (int64), keys [P] uint32, ids [P] int64,
    n_macro per view and the segment base per view.
    """
    segs, keys, ids, bases, nms = [], [], [], [], []
    base = 0
    for (mx, my, r, key), (w, h) in zip(views, width_height):
        s, k, i, nm = bin_pairs(mx, my, r, key, w, h, bw, bh, base)
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
